"""Several disjoint fine regions with their own M sharing the coarse step,
on the GPU through the C ABI, against the FP64 oracle (or_lts3_multi), and
the identities the oracle's pins fix: one region as the ordinary LTS3 path,
two regions of equal M as the single-region run on their union, M = 1
everywhere as SSPRK3, and every launch schedule alike."""
import math

import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.fixture(scope="module")
def hexrid():
    w = W.workload("hex_1024")
    x, y = w.mesh["xCell"], w.mesh["yCell"]
    Lx, Ly = w.mesh["period_x"], w.mesh["period_y"]
    rid = np.zeros(w.nCells, np.int8)
    for r, (cx, cy) in enumerate([(0.25 * Lx, 0.25 * Ly), (0.75 * Lx, 0.75 * Ly)], start=1):
        dx = (x - cx) - Lx * np.round((x - cx) / Lx)
        dy = (y - cy) - Ly * np.round((y - cy) / Ly)
        rid[dx * dx + dy * dy <= 25e3 ** 2] = r
    # a bump over region 1 so both regions and the coarse cells move
    return w, rid


@pytest.fixture(scope="module")
def sphrid():
    """Sphere with two refined caps of different ratio (8:1 and 4:1)."""
    caps = [(1.5 * math.pi, math.pi / 6, math.radians(12), math.radians(4), 8.0),
            (0.5 * math.pi, -math.pi / 6, math.radians(12), math.radians(4), 4.0)]
    mesh = W.scvt_mesh(6000, 21, caps, 60)
    h0, u0, b = W.zonal_state(mesh)
    mesh["bottom"] = b
    lon, lat = W._lonlat(mesh["xCell"], mesh["yCell"], mesh["zCell"])
    rid = np.zeros(mesh["nCells"], np.int8)
    for r, (lo, la, rad, wid, ratio) in enumerate(caps, start=1):
        d = W._great_circle(lon, lat, lo, la)
        s = 1.0 / ratio + (1.0 - 1.0 / ratio) * 0.5 * (1.0 + np.tanh((d - rad) / wid))
        rid[s < 0.9] = r
    dt, _, _ = W._cfl_dt(mesh, h0, u0, rid == 0, 0.5)
    return mesh, h0, u0, rid, dt


def gpu(mesh, rid, Ms, h0, u0, dt, n, precision, **kw):
    with lts.Model(mesh, rid, list(Ms), h0, u0, dt, 9.81, precision=precision, **kw) as m:
        m.step(n)
        return m.read()


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
def test_two_hex_regions_match_oracle(hexrid, precision):
    w, rid = hexrid
    n, Ms = 20, (4, 2)
    h, u, _ = gpu(w.mesh, rid, Ms, w.h0, w.u0, w.dt, n, precision)
    rh, ru = oracle.Oracle(w.mesh).lts3_multi(w.h0, w.u0, rid, Ms, w.dt, n, g=w.g)
    # u of the small hex bump sits near the FP64 conditioning floor
    # g eps H T / d_min of two correct evaluation orders (as in the
    # single-region hex test)
    floor = 9.81 * 2.0 ** -53 * float(w.h0.max()) * n * w.dt / float(w.mesh["dcEdge"].min())
    floor /= float(np.abs(ru).max())
    if precision == lts.LTS_FP64:
        assert rel(h, rh) <= 1e-12 and rel(u, ru) <= max(1e-12, floor), (rel(h, rh), rel(u, ru))
    else:
        assert rel(h, rh) <= 2e-5 and rel(u, ru) <= 1e-4, (rel(h, rh), rel(u, ru))


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
def test_two_sphere_caps_match_oracle(sphrid, precision):
    mesh, h0, u0, rid, dt = sphrid
    n, Ms = 10, (8, 4)
    h, u, _ = gpu(mesh, rid, Ms, h0, u0, dt, n, precision)
    rh, ru = oracle.Oracle(mesh).lts3_multi(h0, u0, rid, Ms, dt, n)
    th, tu = (1e-12, 1e-12) if precision == lts.LTS_FP64 else (2e-5, 1e-4)
    assert rel(h, rh) <= th and rel(u, ru) <= tu, (rel(h, rh), rel(u, ru))


def test_one_region_equals_plain_path(hexrid):
    w, rid = hexrid
    one = (rid == 1).astype(np.int8)
    a = gpu(w.mesh, one, [3], w.h0, w.u0, w.dt, 5, lts.LTS_FP64)
    with lts.Model(w.mesh, one, 3, w.h0, w.u0, w.dt, 9.81, precision=lts.LTS_FP64) as m:
        m.step(5)
        b = m.read()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
def test_equal_m_equals_union_run(hexrid, precision):
    w, rid = hexrid
    a = gpu(w.mesh, rid, [2, 2], w.h0, w.u0, w.dt, 6, precision)
    with lts.Model(w.mesh, (rid > 0).astype(np.int8), 2, w.h0, w.u0, w.dt, 9.81,
                   precision=precision) as m:
        m.step(6)
        b = m.read()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_all_m1_is_ssprk3(hexrid):
    w, rid = hexrid
    a = gpu(w.mesh, rid, [1, 1], w.h0, w.u0, w.dt, 5, lts.LTS_FP64)
    with lts.Model(w.mesh, rid > 0, 1, w.h0, w.u0, w.dt, 9.81, precision=lts.LTS_FP64,
                   mode=lts.LTS_MODE_SSPRK3) as m:
        m.step(5)
        b = m.read()
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_multi_schedules_identical(sphrid):
    mesh, h0, u0, rid, dt = sphrid
    a = gpu(mesh, rid, (8, 4), h0, u0, dt, 4, lts.LTS_FP32)
    for kw in ({"coarse_schedule": lts.LTS_COARSE_FAR}, {"coarse_schedule": lts.LTS_COARSE_SERIAL},
               {"use_graph": False}, {"pdl": False}):
        b = gpu(mesh, rid, (8, 4), h0, u0, dt, 4, lts.LTS_FP32, **kw)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]), kw
