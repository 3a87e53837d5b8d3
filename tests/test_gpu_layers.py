"""Multi-layer states: L independent shallow-water layers advanced on one
mesh, sharing every mesh-table load (the paper's speed-up runs repeat the
computation for 100 layers).  Each layer sees exactly the arithmetic of a
single-layer state, so L copies of one state reproduce the single-layer
result bit for bit, and different layers each match the FP64 oracle."""
import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def sphw():
    return W.workload("scvt_2562")


def perturbed(w, L, seed=3):
    rng = np.random.default_rng(seed)
    h = np.stack([w.h0 * (1.0 + 1e-3 * k * rng.standard_normal(w.nCells)) for k in range(L)])
    u = np.stack([w.u0 * (1.0 + 0.1 * k) for k in range(L)])
    return h, u


def run(w, h0, u0, n, precision, layers=1, **kw):
    with lts.Model(w.mesh, w.fine_mask, w.M, h0, u0, w.dt, w.g, precision=precision,
                   layers=layers, **kw) as m:
        m.step(n)
        return m.read()


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
@pytest.mark.parametrize("L", [2, 5, 33])
def test_identical_layers_equal_single_layer_bitwise(sphw, precision, L):
    h1, u1, d1 = run(sphw, sphw.h0, sphw.u0, 4, precision)
    hL, uL, dL = run(sphw, np.tile(sphw.h0, (L, 1)), np.tile(sphw.u0, (L, 1)), 4, precision, layers=L)
    assert hL.shape == (L, sphw.nCells) and uL.shape == (L, int(sphw.mesh["nEdges"]))
    for k in range(L):
        assert np.array_equal(hL[k], h1) and np.array_equal(uL[k], u1), k
    assert abs(dL["mass"] - L * d1["mass"]) <= 1e-13 * L * d1["mass"]


@pytest.mark.parametrize("precision,comp", [(lts.LTS_FP64, False), (lts.LTS_FP32, True), (lts.LTS_FP32, False)])
@pytest.mark.parametrize("L", [3, 4, 6, 8])
def test_different_layers_equal_their_single_layer_runs_bitwise(sphw, precision, comp, L):
    """Each layer of a state whose layers differ equals the single-layer run
    from that layer's initial state, bit for bit, so a swapped or shifted
    lane would fail here.  Even L runs pairs of layers through two-word
    accesses (L = 6 also has a thread with a single pair, layers 4 and 5);
    with L a multiple of four the FP32 vertex and edge passes run a thread's
    four layers through four-word accesses (L = 8: two groups per element);
    odd L runs every layer through the single-layer code."""
    h0, u0 = perturbed(sphw, L)
    hL, uL, _ = run(sphw, h0, u0, 4, precision, layers=L, compensated=comp)
    for k in range(L):
        h1, u1, _ = run(sphw, h0[k], u0[k], 4, precision, compensated=comp)
        assert np.array_equal(hL[k], h1) and np.array_equal(uL[k], u1), k


@pytest.mark.parametrize("L", [3, 4])
def test_layers_match_oracle_each(sphw, L):
    n = 10
    h0, u0 = perturbed(sphw, L)
    hL, uL, _ = run(sphw, h0, u0, n, lts.LTS_FP64, layers=L)
    o = oracle.Oracle(sphw.mesh)
    cl, el = o.regions(sphw.fine_mask)
    for k in range(L):
        rh, ru = o.lts3(h0[k], u0[k], cl, el, sphw.M, sphw.dt, n, g=sphw.g)
        assert rel(hL[k], rh) <= 1e-12 and rel(uL[k], ru) <= 1e-12, k


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
@pytest.mark.parametrize("mode,order", [(lts.LTS_MODE_LTS, 2), (lts.LTS_MODE_SSPRK3, 3)])
def test_layers_other_integrators(sphw, mode, order, precision):
    L = 4
    dt = sphw.dt / (2 * sphw.M)
    h0, u0 = perturbed(sphw, L)
    with lts.Model(sphw.mesh, sphw.fine_mask, sphw.M, h0, u0, dt, sphw.g, precision=precision,
                   mode=mode, order=order, layers=L) as m:
        m.step(3)
        hL, uL, _ = m.read()
    for k in range(L):
        with lts.Model(sphw.mesh, sphw.fine_mask, sphw.M, h0[k], u0[k], dt, sphw.g,
                       precision=precision, mode=mode, order=order) as m:
            m.step(3)
            h1, u1, _ = m.read()
        assert np.array_equal(hL[k], h1) and np.array_equal(uL[k], u1), k


def test_layers_write_read_roundtrip_and_checks(sphw):
    L = 3
    h0, u0 = perturbed(sphw, L)
    with lts.Model(sphw.mesh, sphw.fine_mask, sphw.M, h0, u0, sphw.dt, sphw.g,
                   precision=lts.LTS_FP64, layers=L) as m:
        h, u, _ = m.read()
        assert np.array_equal(h, h0) and np.array_equal(u, u0)
        m.write(h0[::-1].copy(), u0[::-1].copy())
        h, u, _ = m.read()
        assert np.array_equal(h, h0[::-1]) and np.array_equal(u, u0[::-1])
    with pytest.raises(lts.LtsError) as ei:   # layers need the three-launch path
        lts.Model(sphw.mesh, sphw.fine_mask, sphw.M, h0, u0, sphw.dt, sphw.g,
                  precision=lts.LTS_FP32, layers=L, kernel_path=lts.PATH_FUSED)
    assert ei.value.code == lts.LTS_EINVAL
