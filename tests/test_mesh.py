"""Pins of the seeded mesh generators (inputs of both the oracle and the GPU
path): Euler characteristic, total area, circumcentre property, orientation
conventions of Appendix B, and closed forms of the regular hexagon."""
import math

import numpy as np
import pytest

from paper_2106_07154_gb300 import workloads as W


@pytest.fixture(scope="module")
def hexm():
    return W.hex_mesh(8, 6, 10e3, 1e-4)


@pytest.fixture(scope="module")
def sph():
    cap = (1.5 * math.pi, math.pi / 6, math.radians(20), math.radians(6), 3.0)
    return W.scvt_mesh(642, 3, [cap], 30, cache=False)


def test_hex_closed_forms(hexm):
    dc = 10e3
    n, e, v = hexm["nCells"], hexm["nEdges"], hexm["nVertices"]
    assert (n, e, v) == (48, 144, 96)
    assert v - e + n == 0                                   # torus
    assert np.allclose(hexm["areaCell"], math.sqrt(3) / 2 * dc * dc, rtol=1e-13)
    assert np.allclose(hexm["areaTriangle"], math.sqrt(3) / 4 * dc * dc, rtol=1e-13)
    assert np.allclose(hexm["kiteAreasOnVertex"], math.sqrt(3) / 12 * dc * dc, rtol=1e-13)
    assert np.allclose(hexm["dcEdge"], dc, rtol=1e-13)
    assert np.allclose(hexm["dvEdge"], dc / math.sqrt(3), rtol=1e-12)
    assert np.isclose(hexm["areaCell"].sum(), hexm["period_x"] * hexm["period_y"], rtol=1e-13)


def test_orientation_rule(hexm, sph):
    for m in (hexm, sph):
        coe = m["cellsOnEdge"]
        # Remark of Appendix B: i1 > i2 => n_{e,i1} = 1, i.e. n_e leaves the larger index
        assert np.all(coe[:, 0] > coe[:, 1])


def _unit(a):
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _sph_tri_area(a, b, c):
    """L'Huilier's theorem from the three arc lengths (independent of the builder)."""
    ang = lambda x, y: np.arccos(np.clip(np.sum(x * y, -1), -1, 1))
    A, B, Cc = ang(b, c), ang(c, a), ang(a, b)
    s = 0.5 * (A + B + Cc)
    t = np.tan(s / 2) * np.tan((s - A) / 2) * np.tan((s - B) / 2) * np.tan((s - Cc) / 2)
    return 4 * np.arctan(np.sqrt(np.maximum(t, 0)))


def test_scvt_invariants(sph):
    R = sph["radius"]
    n, e, v = sph["nCells"], sph["nEdges"], sph["nVertices"]
    assert v - e + n == 2                                    # sphere
    assert e == 3 * n - 6 and v == 2 * n - 4
    assert np.isclose(sph["areaCell"].sum(), 4 * math.pi * R * R, rtol=1e-12)
    assert np.isclose(sph["areaTriangle"].sum(), 4 * math.pi * R * R, rtol=1e-12)
    xc = np.stack([sph["xCell"], sph["yCell"], sph["zCell"]], 1) / R
    xv = np.stack([sph["xVertex"], sph["yVertex"], sph["zVertex"]], 1) / R
    cov = sph["cellsOnVertex"]
    # circumcentre: each vertex equidistant from its three cells
    d = np.stack([np.sum(xv * xc[cov[:, k]], 1) for k in range(3)], 1)
    assert np.max(np.abs(d - d[:, :1])) < 1e-12
    # A_v equals the spherical area of the Delaunay triangle (L'Huilier)
    area = _sph_tri_area(xc[cov[:, 0]], xc[cov[:, 1]], xc[cov[:, 2]]) * R * R
    assert np.allclose(sph["areaTriangle"], area, rtol=1e-9)
    # kites: per vertex sum = A_v, per cell sum = A_i
    assert np.allclose(sph["kiteAreasOnVertex"].sum(1), sph["areaTriangle"], rtol=1e-12)
    ka = np.zeros(n)
    np.add.at(ka, cov.ravel(), sph["kiteAreasOnVertex"].ravel())
    assert np.allclose(ka, sph["areaCell"], rtol=1e-12)
    # lengths
    coe, voe = sph["cellsOnEdge"], sph["verticesOnEdge"]
    dc = R * np.arccos(np.clip(np.sum(xc[coe[:, 0]] * xc[coe[:, 1]], 1), -1, 1))
    assert np.allclose(sph["dcEdge"], dc, rtol=1e-9)
    dv = R * np.arccos(np.clip(np.sum(xv[voe[:, 0]] * xv[voe[:, 1]], 1), -1, 1))
    assert np.allclose(sph["dvEdge"], dv, rtol=1e-6, atol=1e-3)
    # verticesOnEdge[:,1] lies in the direction k x n_e (t_{e,v} = +1)
    xe = _unit(np.stack([sph["xEdge"], sph["yEdge"], sph["zEdge"]], 1))
    nvec = xc[coe[:, 1]] - xc[coe[:, 0]]
    kxn = np.cross(xe, nvec)
    side = np.sum((xv[voe[:, 1]] - xv[voe[:, 0]]) * kxn, 1)
    assert np.all(side >= -1e-15)
    # f_v = 2 Omega sin(lat_v)
    assert np.allclose(sph["fVertex"], 2 * W.OMEGA * xv[:, 2], rtol=1e-12)


def test_rings_counter_clockwise(sph):
    R = sph["radius"]
    xc = np.stack([sph["xCell"], sph["yCell"], sph["zCell"]], 1) / R
    coc, noc, eoc, voc = sph["cellsOnCell"], sph["nEdgesOnCell"], sph["edgesOnCell"], sph["verticesOnCell"]
    coe, voe = sph["cellsOnEdge"], sph["verticesOnEdge"]
    for i in range(sph["nCells"]):
        k = noc[i]
        for j in range(k):
            a, b = xc[coc[i, j]], xc[coc[i, (j + 1) % k]]
            assert np.dot(np.cross(a - xc[i], b - xc[i]), xc[i]) > 0
            e = eoc[i, j]
            assert set(coe[e]) == {i, coc[i, j]}
            # vertex j between edge j and edge j+1
            e2 = eoc[i, (j + 1) % k]
            assert voc[i, j] in set(voe[e]) and voc[i, j] in set(voe[e2])


def test_scvt_density_refines_cap():
    """Cells in the cap are smaller by about the requested ratio."""
    cap = (0.0, 0.0, math.radians(25), math.radians(5), 3.0)
    m = W.scvt_mesh(2562, 5, [cap], 80, cache=False)
    R = m["radius"]
    xc = np.stack([m["xCell"], m["yCell"], m["zCell"]], 1) / R
    ang = np.arccos(np.clip(xc[:, 0], -1, 1))
    inner = np.sqrt(m["areaCell"][ang < math.radians(15)]).mean()
    outer = np.sqrt(m["areaCell"][ang > math.radians(50)]).mean()
    assert 2.4 < outer / inner < 3.6


def test_scvt_deterministic():
    a = W.scvt_mesh(162, 9, [], 10, cache=False)
    b = W.scvt_mesh(162, 9, [], 10, cache=False)
    assert np.array_equal(a["cellsOnEdge"], b["cellsOnEdge"])
    assert np.array_equal(a["areaCell"], b["areaCell"])
