"""The second-order path on the GPU (Algorithm 2.2 with its LTS2 branches,
Algorithm 2.1 as SSPRK2) through the C ABI, against the FP64 oracle.

LTS2's stability limit is below LTS3's, so these runs use half the LTS3
coarse step of the workload (the paper's LTS2 runs use smaller steps too)."""
import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_H = 2e-5
TOL32_U = 1e-4


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def sphw():
    return W.workload("scvt_2562")


def gpu(w, n, precision, M=None, dt=None, mode=lts.LTS_MODE_LTS, order=2, **kw):
    with lts.Model(w.mesh, w.fine_mask, M or w.M, w.h0, w.u0, dt or w.dt / 2, w.g,
                   precision=precision, mode=mode, order=order, **kw) as m:
        m.step(n)
        h, u, _ = m.read()
    return h, u


@pytest.fixture(scope="module")
def ref50(sphw):
    o = oracle.Oracle(sphw.mesh)
    cl, el = o.regions(sphw.fine_mask)
    return o.lts2(sphw.h0, sphw.u0, cl, el, sphw.M, sphw.dt / 2, 50, g=sphw.g)


def test_lts2_fp64_matches_oracle(sphw, ref50):
    h, u = gpu(sphw, 50, lts.LTS_FP64)
    assert rel(h, ref50[0]) <= TOL64 and rel(u, ref50[1]) <= TOL64


def test_lts2_fp32_matches_oracle(sphw, ref50):
    h, u = gpu(sphw, 50, lts.LTS_FP32)
    assert rel(h, ref50[0]) <= TOL32_H and rel(u, ref50[1]) <= TOL32_U


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
def test_lts2_m1_equals_ssprk2_bitwise(sphw, precision):
    dt = sphw.dt / (2 * sphw.M)
    a = gpu(sphw, 10, precision, M=1, dt=dt)
    b = gpu(sphw, 10, precision, M=1, dt=dt, mode=lts.LTS_MODE_SSPRK2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_ssprk2_fp64_matches_oracle(sphw):
    dt = sphw.dt / (2 * sphw.M)
    h, u = gpu(sphw, 30, lts.LTS_FP64, dt=dt, mode=lts.LTS_MODE_SSPRK2)
    rh, ru = oracle.Oracle(sphw.mesh).ssprk2(sphw.h0, sphw.u0, dt, 30, g=sphw.g)
    assert rel(h, rh) <= TOL64 and rel(u, ru) <= TOL64


def test_lts2_schedules_and_launch_modes_identical(sphw):
    a = gpu(sphw, 6, lts.LTS_FP32)
    for kw in ({"coarse_schedule": lts.LTS_COARSE_SERIAL}, {"use_graph": False}, {"profile": 1}):
        b = gpu(sphw, 6, lts.LTS_FP32, **kw)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), kw


def test_lts2_rejects_fused_path(sphw):
    with pytest.raises(lts.LtsError) as ei:
        gpu(sphw, 1, lts.LTS_FP32, kernel_path=lts.PATH_FUSED)
    assert ei.value.code == lts.LTS_EINVAL
