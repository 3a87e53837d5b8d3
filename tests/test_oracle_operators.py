"""Pins of the oracle's TRiSK operators (Appendix B) against what the
mathematics fixes: closed forms on regular hexagons, antisymmetry of the
weights, discrete adjointness, curl of a gradient, energy neutrality of the
potential-vorticity flux, the lake at rest, the sign of the vorticity, and the
energy diagnostic (a closed form and the conservation the semi-discrete
system has)."""
import math

import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import workloads as W


@pytest.fixture(scope="module")
def hexm():
    return W.hex_mesh(8, 8, 10e3, 1e-4)


@pytest.fixture(scope="module")
def sph():
    cap = (1.5 * math.pi, math.pi / 6, math.radians(20), math.radians(6), 3.0)
    m = W.scvt_mesh(642, 3, [cap], 30, cache=False)
    rng = np.random.default_rng(0)
    m["bottom"] = rng.uniform(0, 500, m["nCells"])
    return m


def _normals_plane(m):
    coe = m["cellsOnEdge"]
    dx = m["xCell"][coe[:, 1]] - m["xCell"][coe[:, 0]]
    dy = m["yCell"][coe[:, 1]] - m["yCell"][coe[:, 0]]
    dx -= m["period_x"] * np.round(dx / m["period_x"])
    dy -= m["period_y"] * np.round(dy / m["period_y"])
    n = np.stack([dx, dy], 1)
    return n / np.linalg.norm(n, axis=1, keepdims=True)


def test_weights_regular_hexagon(hexm):
    """T5b: on regular hexagons every kite is A_i/6, so the weights take the
    values {+-1/3, +-1/6, 0} and each edge has 10 neighbours."""
    o = oracle.Oracle(hexm)
    n, eoe, w = o.weights()
    assert np.all(n == 10)
    vals = w[:, :10]
    allowed = np.array([-1 / 3, -1 / 6, 0.0, 1 / 6, 1 / 3])
    dist = np.abs(vals[..., None] - allowed).min(-1)
    assert dist.max() < 1e-14
    # each cell contributes one of each magnitude 1/3,1/6,0,1/6,1/3
    for half in (vals[:, :5], vals[:, 5:]):
        assert np.allclose(np.sort(np.abs(half), 1), [0, 1 / 6, 1 / 6, 1 / 3, 1 / 3], atol=1e-14)


def test_weights_antisymmetric(sph):
    """T5a: w_{e,e'} = -w_{e',e} (needed for energy conservation)."""
    o = oracle.Oracle(sph)
    n, eoe, w = o.weights()
    tab = {}
    for e in range(sph["nEdges"]):
        for j in range(n[e]):
            tab[(e, eoe[e, j])] = w[e, j]
    worst = max(abs(v + tab[(b, a)]) for (a, b), v in tab.items())
    assert worst < 1e-14


def test_tangential_reconstruction_uniform(hexm):
    """T5c: for a uniform flux F on regular hexagons, F_e^perp of Eq.
    (Feperp) equals the normal component of F^perp = k x F (Appendix A)."""
    o = oracle.Oracle(hexm)
    nrm = _normals_plane(hexm)
    for F in ([1.0, 0.0], [0.3, -2.0], [-1.5, 0.7]):
        Fe = nrm @ np.array(F)
        kxF = np.array([-F[1], F[0]])
        Fperp = o.tangential(Fe)
        assert np.allclose(Fperp, nrm @ kxF, atol=1e-13)


def test_kinetic_energy_uniform(hexm):
    """K_i = |u|^2/2 exactly for a uniform velocity on regular hexagons."""
    o = oracle.Oracle(hexm)
    nrm = _normals_plane(hexm)
    U = np.array([3.0, -4.0])
    K = o.kinetic(nrm @ U)
    assert np.allclose(K, 12.5, rtol=1e-13)
    assert np.allclose(o.divergence(nrm @ U), 0.0, atol=1e-16)


def test_divergence_sums_to_zero(sph):
    """T5d: sum_i A_i [div F]_i = 0 (every flux enters one cell and leaves the other)."""
    o = oracle.Oracle(sph)
    F = np.random.default_rng(1).normal(size=sph["nEdges"])
    d = o.divergence(F)
    A = sph["areaCell"]
    assert abs(np.sum(A * d)) < 1e-13 * np.sum(np.abs(A * d))


def test_adjointness(sph):
    """T5e: sum_i A_i phi_i [div F]_i = - sum_e l_e d_e F_e [grad phi]_e."""
    o = oracle.Oracle(sph)
    rng = np.random.default_rng(2)
    F = rng.normal(size=sph["nEdges"])
    phi = rng.normal(size=sph["nCells"])
    lhs = np.sum(sph["areaCell"] * phi * o.divergence(F))
    rhs = -np.sum(sph["dvEdge"] * sph["dcEdge"] * F * o.gradient(phi))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_curl_of_gradient(sph):
    """T5f: the vorticity of a discrete gradient vanishes."""
    o = oracle.Oracle(sph)
    phi = np.random.default_rng(3).normal(size=sph["nCells"])
    g = o.gradient(phi)
    z = o.vorticity(g)
    scale = np.abs(g).max() * sph["dcEdge"].max() * 3 / sph["areaTriangle"].min()
    assert np.abs(z).max() < 1e-13 * scale


def test_pv_flux_energy_neutral(sph):
    """T5g: sum_e l_e d_e F_e (F^perp [q])_e = 0 for any F and q."""
    o = oracle.Oracle(sph)
    rng = np.random.default_rng(4)
    F = rng.normal(size=sph["nEdges"])
    qe = rng.normal(size=sph["nEdges"])
    pv = o.pv_flux(F, qe)
    w = sph["dvEdge"] * sph["dcEdge"] * F
    assert abs(np.sum(w * pv)) < 1e-13 * np.sum(np.abs(w * pv))


def test_lake_at_rest(sph):
    """T5h: u = 0 and h + b constant -> H = U = 0 exactly."""
    o = oracle.Oracle(sph)
    b = np.floor(sph["bottom"])           # integers: h = C - b is exact
    m = dict(sph)
    m["bottom"] = b
    o = oracle.Oracle(m)
    h = 4000.0 - b
    H, U = o.rhs(h, np.zeros(sph["nEdges"]))
    assert np.all(H == 0.0) and np.all(U == 0.0)


def test_vorticity_sign_solid_body():
    """zeta_v of u = u0 cos(lat) approaches the exact 2 u0 sin(lat)/R (pins t_{e,v})."""
    m = W.scvt_mesh(2562, 11, [], 40, cache=False)
    _, u, _ = W.zonal_state(m, u0=20.0, mountain_height=0.0)
    o = oracle.Oracle(m)
    z = o.vorticity(u)
    R = m["radius"]
    lat = np.arcsin(m["zVertex"] / R)
    exact = 2 * 20.0 * np.sin(lat) / R
    assert np.abs(z - exact).max() < 0.05 * np.abs(exact).max()


def test_geostrophic_balance_pv_vs_gradient():
    """For the balanced zonal state the PV flux and the gradient of K + g(h+b)
    nearly cancel (Appendix A balance), so |U| is a small fraction of either."""
    m = W.scvt_mesh(2562, 11, [], 40, cache=False)
    h, u, b = W.zonal_state(m, u0=20.0, mountain_height=0.0)
    m["bottom"] = b
    o = oracle.Oracle(m)
    H, U = o.rhs(h, u)
    g_term = o.gradient(9.81 * (h + b))
    q = o.pv_vertex(h, u)
    voe = m["verticesOnEdge"]
    pv = o.pv_flux(o.thickness_flux(h, u), 0.5 * (q[voe[:, 0]] + q[voe[:, 1]]))
    # discretisation residual of the balance (coarse 480 km mesh): < 20% ...
    assert np.abs(U).max() < 0.2 * np.abs(g_term).max()
    # ... whereas the PV flux with the opposite sign would double the tendency
    assert np.abs(U + 2 * pv).max() > 1.5 * np.abs(g_term).max()
    assert np.abs(H).max() * 3600 < 5.0    # < 5 m/hour thickness tendency


@pytest.mark.parametrize("bottom", [0.0, 250.0])
def test_energy_uniform_flow_closed_form(hexm, bottom):
    """Energy (reading R8) of a uniform flow U at constant thickness h over a
    constant bottom b on regular hexagons: K = |U|^2/2 in every cell, so
    E = (total area) h (|U|^2/2 + g (h/2 + b)), a single number the per-cell
    sum must reproduce.  A missing 1/2, a wrong g or a wrong area weighting
    fails it."""
    m = dict(hexm)
    m["bottom"] = np.full(hexm["nCells"], bottom)
    o = oracle.Oracle(m)
    nrm = _normals_plane(hexm)
    U = np.array([3.0, -4.0])
    h0, g = 800.0, 9.81
    area = hexm["period_x"] * hexm["period_y"]
    assert abs(np.sum(hexm["areaCell"]) - area) < 1e-9 * area
    E = o.energy(np.full(hexm["nCells"], h0), nrm @ U, g)
    exact = area * h0 * (0.5 * 25.0 + g * (0.5 * h0 + bottom))
    assert abs(E - exact) < 1e-13 * exact


def test_energy_conserved_along_the_flow(sph):
    """The TRiSK system of Eq. (1) conserves the energy of reading R8 in
    continuous time (Appendix B: the PV flux does no work and the divergence
    is the negative adjoint of the gradient).  So the derivative of the
    oracle's energy along its own right-hand side, taken by a centred
    difference, vanishes relative to the rate at which potential and kinetic
    energy trade.  Negative controls: doubling K or the g h term in the
    energy breaks it by orders of magnitude."""
    o = oracle.Oracle(sph)
    rng = np.random.default_rng(5)
    b = sph["bottom"]
    h = 5000.0 - b + rng.uniform(-20.0, 20.0, sph["nCells"])
    u = rng.normal(0.0, 10.0, sph["nEdges"])
    g = 9.81
    H, U = o.rhs(h, u, g)
    A = sph["areaCell"]
    # the rate of exchange between the two energy forms (the scale)
    exchange = abs(np.sum(A * (o.kinetic(u) + g * (h + b)) * H))
    eps = 1.0

    def ddt(energy):
        return (energy(h + eps * H, u + eps * U) - energy(h - eps * H, u - eps * U)) / (2 * eps)

    assert abs(ddt(lambda hh, uu: o.energy(hh, uu, g))) < 1e-6 * exchange
    twice_k = lambda hh, uu: np.sum(A * hh * (2.0 * o.kinetic(uu) + g * (0.5 * hh + b)))
    full_gh = lambda hh, uu: np.sum(A * hh * (o.kinetic(uu) + g * (hh + b)))
    assert abs(ddt(twice_k)) > 0.1 * exchange
    assert abs(ddt(full_gh)) > 0.1 * exchange
