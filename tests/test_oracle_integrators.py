"""Pins of the oracle's time integrators (Algorithms 2.1 and 2.2) and of the
index sets of Eqs. (3)-(5) against closed forms, brute force and the
properties the paper states (M = 1 identity, mass conservation, order 3)."""
import math

import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import workloads as W


def P3(z):
    """SSPRK3 stability polynomial (third-order Taylor polynomial of e^z)."""
    return 1 + z + z * z / 2 + z ** 3 / 6


@pytest.fixture(scope="module")
def hexw():
    return W.hex_bump(nx=16, ny=16, radius=35e3, M=2, seed=3)


@pytest.fixture(scope="module")
def sphw():
    w = W.workload("scvt_2562", cache=False, lloyd_iters=40, M=4)
    return w


# ------------------------------------------------------------------ regions

def _bfs_labels(mesh, fine, layers=1):
    """Independent restatement of Eqs. (3)-(5) by breadth-first distances
    (interfaces `layers` cells thick: I1 = distance 1..L, I2 = L+1..2L)."""
    n = mesh["nCells"]
    coc, noc = mesh["cellsOnCell"], mesh["nEdgesOnCell"]
    nb = [list(coc[i, :noc[i]]) for i in range(n)]
    INF = 10 ** 9

    def bfs(sources, allowed):
        d = np.full(n, INF)
        frontier = list(sources)
        for s in frontier:
            d[s] = 0
        while frontier:
            nxt = []
            for i in frontier:
                for j in nb[i]:
                    if allowed[j] and d[j] == INF:
                        d[j] = d[i] + 1
                        nxt.append(j)
            frontier = nxt
        return d

    isF = fine.astype(bool)
    dout = bfs(np.nonzero(isF)[0], ~isF | True)        # distance from F
    din = bfs(np.nonzero(~isF)[0], isF | True)          # distance from outside F
    cl = np.full(n, 5, np.int8)
    cl[(dout >= 1) & (dout <= layers)] = 3
    cl[(dout > layers) & (dout <= 2 * layers)] = 4
    cl[isF] = 0
    cl[isF & (din == 2)] = 1
    cl[isF & (din == 1) & np.array([any((not isF[j]) and dout[j] == 1 for j in nb[i]) for i in range(n)])] = 2
    rank = np.where(cl <= 0, 0, np.where(cl <= 2, 1, cl))
    coe = mesh["cellsOnEdge"]
    el = np.minimum(rank[coe[:, 0]], rank[coe[:, 1]]).astype(np.int8)
    return cl, el


@pytest.mark.parametrize("which", ["hex", "sph"])
@pytest.mark.parametrize("layers", [1, 2, 3])
def test_regions_match_brute_force(which, layers, hexw, sphw):
    w = hexw if which == "hex" else sphw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask, layers)
    bcl, bel = _bfs_labels(w.mesh, w.fine_mask, layers)
    assert np.array_equal(cl, bcl)
    assert np.array_equal(el, bel)
    # the sets form a disjoint cover and are all present
    assert set(np.unique(cl)) == {0, 1, 2, 3, 4, 5}
    assert set(np.unique(el)) == {0, 1, 3, 4, 5}


# ------------------------------------------------------------ linear system

def _linear(mesh, seed=0):
    rng = np.random.default_rng(seed)
    lam_c = -rng.uniform(1e-5, 2e-3, mesh["nCells"])
    lam_e = -rng.uniform(1e-5, 2e-3, mesh["nEdges"])
    h0 = rng.uniform(1, 2, mesh["nCells"])
    u0 = rng.uniform(-1, 1, mesh["nEdges"])
    return lam_c, lam_e, h0, u0


def test_ssprk3_linear_closed_form(hexw):
    """T6a: one SSPRK3 step of y' = lam y multiplies y by 1 + z + z^2/2 + z^3/6."""
    o = oracle.Oracle(hexw.mesh)
    lam_c, lam_e, h0, u0 = _linear(hexw.mesh)
    dt = 100.0
    h, u = o.ssprk3(h0, u0, dt, 1, lam_c=lam_c, lam_e=lam_e)
    assert np.allclose(h, h0 * P3(lam_c * dt), rtol=1e-14)
    assert np.allclose(u, u0 * P3(lam_e * dt), rtol=1e-14, atol=1e-16)


def test_rk4_linear_closed_form(hexw):
    o = oracle.Oracle(hexw.mesh)
    lam_c, lam_e, h0, u0 = _linear(hexw.mesh)
    dt = 100.0
    z = lam_c * dt
    h, _ = o.rk4(h0, u0, dt, 1, lam_c=lam_c, lam_e=lam_e)
    assert np.allclose(h, h0 * (P3(z) + z ** 4 / 24), rtol=1e-14)


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_lts3_linear_closed_form(hexw, M):
    """On decoupled linear ODEs Algorithm 2.2 gives P3(z/M)^M on the fine sets
    (M SSPRK3 substeps) and P3(z) on every other set; on I1 this holds only
    because the predictions and theta-weights integrate the quadratic
    interpolant exactly (a consequence of the alpha/beta/gamma formulas)."""
    w = hexw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    lam_c, lam_e, h0, u0 = _linear(w.mesh, seed=M)
    dt = 120.0
    h, u = o.lts3(h0, u0, cl, el, M, dt, 1, lam_c=lam_c, lam_e=lam_e)
    zc, ze = lam_c * dt, lam_e * dt
    fine_c, fine_e = cl <= 2, el <= 1
    exp_h = np.where(fine_c, P3(zc / M) ** M, P3(zc)) * h0
    exp_u = np.where(fine_e, P3(ze / M) ** M, P3(ze)) * u0
    assert np.allclose(h, exp_h, rtol=2e-15 * 10)
    assert np.allclose(u, exp_u, rtol=2e-14, atol=1e-16)


@pytest.mark.parametrize("M", [1, 2, 4, 7])
def test_prediction_reproduces_fine_stage_inputs(M):
    """T9: for y' = lam y, old = 1, 1st = 1 + z, 2nd = 1 + z/2 + z^2/4 (the
    coarse stages); the predictions of Steps 3.x.1 must equal, up to O(z^3),
    the value the fine SSPRK3 holds at that stage of substep k."""
    for k in range(M):
        # fine solution at t_k, as a polynomial in z up to z^2: exp(k z / M)
        base = np.array([1.0, k / M, (k / M) ** 2 / 2])
        targets = {
            1: base,
            2: np.convolve(base, [1.0, 1.0 / M])[:3],                       # Euler stage
            3: np.convolve(base, [1.0, 1.0 / (2 * M), 1.0 / (4 * M * M)])[:3],  # SSP stage 2
        }
        for stage in (1, 2, 3):
            c = oracle.predict_coeffs(k, M, stage)
            poly = c[0] * np.array([1, 0, 0]) + c[1] * np.array([1, 1, 0]) + c[2] * np.array(
                [1, 0.5, 0.25])
            assert np.allclose(poly, targets[stage], atol=1e-15), (k, stage)


# -------------------------------------------------------------- SWE system

def _sw(w, ncoarse, M=None, step5=0):
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    return o.lts3(w.h0, w.u0, cl, el, M or w.M, w.dt, ncoarse, step5_form=step5)


@pytest.mark.parametrize("which", ["hex", "sph"])
def test_lts3_m1_is_ssprk3_bitwise(which, hexw, sphw):
    """T1 (Remark in Section 2.2): with M = 1, LTS3 reproduces SSPRK3; with
    the replay form of Step 5 the agreement is bit for bit."""
    w = hexw if which == "hex" else sphw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    h1, u1 = o.lts3(w.h0, w.u0, cl, el, 1, w.dt, 5)
    h2, u2 = o.ssprk3(w.h0, w.u0, w.dt, 5)
    assert np.array_equal(h1, h2) and np.array_equal(u1, u2)
    # the Step 5 form printed in the paper agrees up to roundoff only
    h3, u3 = o.lts3(w.h0, w.u0, cl, el, 1, w.dt, 5, step5_form=1)
    assert np.max(np.abs(h3 - h2)) < 1e-12 * np.abs(h2).max()
    assert np.max(np.abs(u3 - u2)) < 1e-10 * np.abs(u2).max() + 1e-14


def test_step5_forms_agree(sphw):
    """The replay reading of Step 5 and the printed increment form agree to roundoff for M > 1."""
    a = _sw(sphw, 3, M=4, step5=0)
    b = _sw(sphw, 3, M=4, step5=1)
    assert np.max(np.abs(a[0] - b[0])) < 1e-11 * np.abs(a[0]).max()
    assert np.max(np.abs(a[1] - b[1])) < 1e-9 * np.abs(a[1]).max()


def test_mass_conservation(sphw):
    """T2: LTS3 conserves sum_i A_i h_i to roundoff (the role of interface 2)."""
    o = oracle.Oracle(sphw.mesh)
    cl, el = o.regions(sphw.fine_mask)
    m0 = o.mass(sphw.h0)
    h, u = o.lts3(sphw.h0, sphw.u0, cl, el, 4, sphw.dt, 10)
    assert abs(o.mass(h) - m0) < 1e-13 * m0
    assert np.max(np.abs(h - sphw.h0)) > 1e-3          # the state did move


def test_mass_conservation_breaks_without_interface_2(sphw):
    """Control: with interface 2 merged into the coarse set (labels 4 -> 5),
    the corrected interface no longer matches the coarse fluxes and mass
    drifts far above roundoff, so the pin above has teeth."""
    o = oracle.Oracle(sphw.mesh)
    cl, el = o.regions(sphw.fine_mask)
    cl2, el2 = cl.copy(), el.copy()
    cl2[cl2 == 4] = 5
    el2[el2 == 4] = 5
    m0 = o.mass(sphw.h0)
    h, _ = o.lts3(sphw.h0, sphw.u0, cl2, el2, 4, sphw.dt, 10)
    assert abs(o.mass(h) - m0) > 1e-10 * m0


def _err(a, b):
    return max(np.max(np.abs(a[0] - b[0])) / np.abs(b[0]).max(),
               np.max(np.abs(a[1] - b[1])) / (np.abs(b[1]).max() + 1e-300))


def test_convergence_order_three(hexw):
    """T3 (Section 3.2): LTS3 errors against an RK4 reference with a tiny step
    fall by ~8 per halving of the coarse step."""
    w = hexw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    T = 1200.0
    ref = o.rk4(w.h0, w.u0, T / 1920, 1920)
    errs = []
    for dt in (30.0, 15.0, 7.5):
        n = int(round(T / dt))
        res = o.lts3(w.h0, w.u0, cl, el, 2, dt, n)
        errs.append(np.max(np.abs(res[0] - ref[0])))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 2.7, (errs, orders)


def test_lts_vs_fine_ssprk3(hexw):
    """T7: LTS3(dt, M) and global SSPRK3(dt/M) approach each other at order 3."""
    w = hexw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    T = 1200.0
    d = []
    for dt in (30.0, 15.0):
        n = int(round(T / dt))
        a = o.lts3(w.h0, w.u0, cl, el, 2, dt, n)
        b = o.ssprk3(w.h0, w.u0, dt / 2, 2 * n)
        d.append(np.max(np.abs(a[0] - b[0])))
    assert math.log2(d[0] / d[1]) > 2.6, d


def _steady_drift(n, T=7200.0):
    w = W.workload("scvt_2562", n=n, cache=False, lloyd_iters=60, M=2, mountain=False)
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    nco = int(math.ceil(T / w.dt))
    dt = T / nco
    a = o.lts3(w.h0, w.u0, cl, el, 2, dt, nco)
    b = o.ssprk3(w.h0, w.u0, dt / 2, 2 * nco)
    return np.max(np.abs(b[0] - w.h0)), np.max(np.abs(a[0] - b[0]))


def test_balanced_flow_stays_steady():
    """T8: a balanced zonal flow (b = 0) only adjusts by its discretisation
    residual, which shrinks under mesh refinement; the time-stepping
    difference LTS3 - fine SSPRK3 is far smaller than that adjustment."""
    drift_c, diff_c = _steady_drift(2562)
    drift_f, _ = _steady_drift(10242)
    assert drift_c < 5e-3 * 6000.0
    assert drift_f < 0.6 * drift_c, (drift_c, drift_f)
    assert diff_c < 0.05 * drift_c, (diff_c, drift_c)


@pytest.mark.parametrize("layers", [2, 3])
def test_thick_interfaces_conserve_mass_and_reduce_to_ssprk3(sphw, layers):
    """Interfaces L cells thick (the speed-up runs of Section 3): mass stays
    conserved to roundoff, and M = 1 is SSPRK3 bit for bit."""
    w = sphw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask, layers)
    c1, _ = o.regions(w.fine_mask, 1)
    assert (cl == 3).sum() > (c1 == 3).sum() and (cl == 4).sum() > (c1 == 4).sum()
    h, u = o.lts3(w.h0, w.u0, cl, el, w.M, w.dt, 5, g=w.g)
    m0 = o.mass(w.h0)
    assert abs(o.mass(h) - m0) <= 1e-13 * m0
    dt1 = w.dt / w.M
    ha, ua = o.lts3(w.h0, w.u0, cl, el, 1, dt1, 4, g=w.g)
    hb, ub = o.ssprk3(w.h0, w.u0, dt1, 4, g=w.g)
    assert np.array_equal(ha, hb) and np.array_equal(ua, ub)
    with pytest.raises(ValueError):
        o.regions(w.fine_mask, 0)


def test_energy_drift_is_third_order():
    """SSPRK3 (Algorithm 2.1) applied to the energy-conserving TRiSK system
    changes the energy of reading R8 only through its time error, so the
    drift over a fixed time falls eight-fold when dt halves (order 3).  An
    energy diagnostic that the semi-discrete system does not conserve would
    drift by the same amount at every dt."""
    m = W.scvt_mesh(642, 3, [], 30, cache=False)
    h, u, b = W.zonal_state(m, u0=20.0, mountain_height=2000.0)
    m["bottom"] = b
    o = oracle.Oracle(m)
    E0 = o.energy(h, u)
    T = 6 * 3600.0
    drift = []
    for dt in (600.0, 300.0, 150.0):
        h1, u1 = o.ssprk3(h, u, dt, int(round(T / dt)))
        drift.append(abs(o.energy(h1, u1) - E0) / E0)
    assert drift[0] > 1e-10   # well above roundoff
    for a, c in zip(drift, drift[1:]):
        assert 6.0 < a / c < 10.0
