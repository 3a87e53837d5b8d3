"""Pins of the oracle's second-order branch: SSPRK2 (Algorithm 2.1) and
LTS2 (Algorithm 2.2 with its LTS2 branches), against what the method and
the mathematics fix: the stability polynomial 1 + z + z^2/2 on a linear
ODE, the closed form of one LTS2 step on a decoupled linear system, the
M = 1 identity with SSPRK2 (Remark in Section 2.2), mass conservation,
second-order convergence against RK4 and against SSPRK2 at the fine step."""
import math

import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import workloads as W


def P2(z):
    """SSPRK2 stability polynomial (second-order Taylor polynomial of e^z)."""
    return 1.0 + z + z * z / 2.0


@pytest.fixture(scope="module")
def hexw():
    return W.workload("hex_1024")


@pytest.fixture(scope="module")
def sphw():
    return W.workload("scvt_2562", cache=False, lloyd_iters=40, M=4)


def _linear(mesh, seed=0):
    rng = np.random.default_rng(seed)
    lam_c = -rng.uniform(1e-5, 2e-3, mesh["nCells"])
    lam_e = -rng.uniform(1e-5, 2e-3, mesh["nEdges"])
    h0 = rng.uniform(1, 2, mesh["nCells"])
    u0 = rng.uniform(-1, 1, mesh["nEdges"])
    return lam_c, lam_e, h0, u0


def test_ssprk2_linear_closed_form(hexw):
    o = oracle.Oracle(hexw.mesh)
    lam_c, lam_e, h0, u0 = _linear(hexw.mesh)
    dt = 100.0
    h, u = o.ssprk2(h0, u0, dt, 1, lam_c=lam_c, lam_e=lam_e)
    assert np.allclose(h, h0 * P2(lam_c * dt), rtol=1e-14)
    assert np.allclose(u, u0 * P2(lam_e * dt), rtol=1e-14, atol=1e-16)


@pytest.mark.parametrize("M", [1, 2, 3, 5])
def test_lts2_linear_closed_form(hexw, M):
    """One LTS2 step of decoupled y' = lam y: P2(z/M)^M on the fine sets, and
    P2(z) on I1 (the linear predictions and theta = 1/2, 1/2 integrate the
    linear interpolant exactly), I2 and C."""
    w = hexw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    lam_c, lam_e, h0, u0 = _linear(w.mesh, seed=M)
    dt = 120.0
    h, u = o.lts2(h0, u0, cl, el, M, dt, 1, lam_c=lam_c, lam_e=lam_e)
    zc, ze = lam_c * dt, lam_e * dt
    exp_h = np.where(cl <= 2, P2(zc / M) ** M, P2(zc)) * h0
    exp_u = np.where(el <= 1, P2(ze / M) ** M, P2(ze)) * u0
    assert np.allclose(h, exp_h, rtol=2e-14)
    assert np.allclose(u, exp_u, rtol=2e-14, atol=1e-16)


@pytest.mark.parametrize("M", [1, 2, 5])
def test_lts2_predictions_are_linear_interpolation(M):
    """Steps 3.1.1 / 3.2.1 with alpha~ = beta~ = 0: the value at t_k and
    t_{k+1} on the line through x_old (t = 0) and x_1st (t = dt)."""
    for k in range(M):
        assert np.allclose(oracle.predict_coeffs(k, M, 1, order=2), [1 - k / M, k / M, 0.0], atol=0)
        assert np.allclose(oracle.predict_coeffs(k, M, 2, order=2),
                           [1 - (k + 1) / M, (k + 1) / M, 0.0], atol=1e-16)


@pytest.mark.parametrize("which", ["hex", "sph"])
def test_lts2_m1_is_ssprk2_bitwise(which, hexw, sphw):
    w = hexw if which == "hex" else sphw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    dt = w.dt / 2
    a = o.lts2(w.h0, w.u0, cl, el, 1, dt, 5)
    b = o.ssprk2(w.h0, w.u0, dt, 5)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    c = o.lts2(w.h0, w.u0, cl, el, 1, dt, 5, step5_form=1)     # printed Step 5: roundoff
    assert np.max(np.abs(c[0] - b[0])) < 1e-12 * np.abs(b[0]).max()


def test_lts2_mass_conservation(sphw):
    o = oracle.Oracle(sphw.mesh)
    cl, el = o.regions(sphw.fine_mask)
    m0 = o.mass(sphw.h0)
    h, _ = o.lts2(sphw.h0, sphw.u0, cl, el, 4, sphw.dt / 2, 10)
    assert abs(o.mass(h) - m0) < 1e-13 * m0
    assert np.max(np.abs(h - sphw.h0)) > 1e-3


def _err(a, b):
    return np.max(np.abs(a[0] - b[0]))


def test_lts2_convergence_order_two(hexw):
    w = hexw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    T = 1200.0
    ref = o.rk4(w.h0, w.u0, T / 1920, 1920)
    errs = []
    for dt in (20.0, 10.0, 5.0):
        n = int(round(T / dt))
        errs.append(_err(o.lts2(w.h0, w.u0, cl, el, 2, dt, n), ref))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert min(orders) > 1.8, (errs, orders)


def test_lts2_vs_fine_ssprk2(hexw):
    w = hexw
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    T = 1200.0
    d = []
    for dt in (20.0, 10.0):
        n = int(round(T / dt))
        a = o.lts2(w.h0, w.u0, cl, el, 2, dt, n)
        b = o.ssprk2(w.h0, w.u0, dt / 2, 2 * n)
        d.append(_err(a, b))
    assert math.log2(d[0] / d[1]) > 1.7, d
