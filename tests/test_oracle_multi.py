"""Pins of the oracle's several-regions LTS3 (disjoint fine regions, each with
its own M, sharing the coarse step): the closed form on a decoupled linear
system (each region's fine sets P3(z/M_r)^M_r, every other set P3(z)), one
region reproducing or_lts3 bit for bit, two regions of equal M reproducing
the single-region run on their union, M = 1 everywhere reproducing SSPRK3,
and mass conservation."""
import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import workloads as W


def P3(z):
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0


@pytest.fixture(scope="module")
def two():
    """32x32 periodic hexagons with two fine disks 160 km apart."""
    w = W.workload("hex_1024")
    x, y = w.mesh["xCell"], w.mesh["yCell"]
    Lx, Ly = w.mesh["period_x"], w.mesh["period_y"]
    rof = np.zeros(w.nCells, np.int8)
    for r, (cx, cy) in enumerate([(0.25 * Lx, 0.25 * Ly), (0.75 * Lx, 0.75 * Ly)], start=1):
        dx = (x - cx) - Lx * np.round((x - cx) / Lx)
        dy = (y - cy) - Ly * np.round((y - cy) / Ly)
        rof[dx * dx + dy * dy <= 35e3 ** 2] = r
    return w, rof


def _linear(mesh, seed=0):
    rng = np.random.default_rng(seed)
    lam_c = -rng.uniform(1e-5, 2e-3, mesh["nCells"])
    lam_e = -rng.uniform(1e-5, 2e-3, mesh["nEdges"])
    return lam_c, lam_e, rng.uniform(1, 2, mesh["nCells"]), rng.uniform(-1, 1, mesh["nEdges"])


@pytest.mark.parametrize("Ms", [(2, 3), (4, 1), (5, 2)])
def test_multi_linear_closed_form(two, Ms):
    w, rof = two
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions((rof > 0).astype(np.int8))
    creg, ereg = o.region_ids(rof, cl, el)
    lam_c, lam_e, h0, u0 = _linear(w.mesh, seed=sum(Ms))
    dt = 120.0
    h, u = o.lts3_multi(h0, u0, rof, Ms, dt, 1, lam_c=lam_c, lam_e=lam_e)
    zc, ze = lam_c * dt, lam_e * dt
    Mc = np.where(creg > 0, np.array((1,) + tuple(Ms))[creg], 1)
    Me = np.where(ereg > 0, np.array((1,) + tuple(Ms))[ereg], 1)
    exp_h = np.where(cl <= 2, P3(zc / Mc) ** Mc, P3(zc)) * h0
    exp_u = np.where(el <= 1, P3(ze / Me) ** Me, P3(ze)) * u0
    assert np.allclose(h, exp_h, rtol=2e-14)
    assert np.allclose(u, exp_u, rtol=2e-14, atol=1e-16)


def test_one_region_is_lts3_bitwise(two):
    w, rof = two
    o = oracle.Oracle(w.mesh)
    one = (rof == 1).astype(np.int8)
    cl, el = o.regions(one)
    a = o.lts3(w.h0, w.u0, cl, el, 3, w.dt, 4)
    b = o.lts3_multi(w.h0, w.u0, one, [3], w.dt, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_equal_m_regions_equal_union_run_bitwise(two):
    w, rof = two
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions((rof > 0).astype(np.int8))
    a = o.lts3(w.h0, w.u0, cl, el, 2, w.dt, 4)
    b = o.lts3_multi(w.h0, w.u0, rof, [2, 2], w.dt, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_all_m1_is_ssprk3_bitwise(two):
    w, rof = two
    o = oracle.Oracle(w.mesh)
    a = o.lts3_multi(w.h0, w.u0, rof, [1, 1], w.dt, 4)
    b = o.ssprk3(w.h0, w.u0, w.dt, 4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_multi_mass_conservation(two):
    w, rof = two
    o = oracle.Oracle(w.mesh)
    m0 = o.mass(w.h0)
    h, _ = o.lts3_multi(w.h0, w.u0, rof, [4, 2], w.dt, 10)
    assert abs(o.mass(h) - m0) < 1e-13 * m0
    assert np.max(np.abs(h - w.h0)) > 1e-4


def test_touching_regions_are_rejected(two):
    w, _ = two
    o = oracle.Oracle(w.mesh)
    rof = np.zeros(w.nCells, np.int8)
    rof[:40] = 1
    rof[40:80] = 2
    cl, el = o.regions((rof > 0).astype(np.int8))
    with pytest.raises(ValueError):
        o.region_ids(rof, cl, el)
