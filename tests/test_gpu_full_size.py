"""Parity with the FP64 oracle at the full sizes of the spherical workloads,
in the launch configuration bench.py times (CUDA graph, programmatic
dependent launch, far coarse phases on a concurrent branch, defaults).

  scvt_40962 (40,962 cells, 4:1 cap, M = 4):  FP64 after 100 coarse steps
      (1e-12 relative max-norm), FP32 + compensation after the workload's
      500 coarse steps (2e-5 on h, 1e-4 on u).
  scvt_655362 (655,362 cells, 8:1 cap, M = 8): 100 coarse steps, FP64
      (1e-12) and FP32 + compensation (2e-5 / 1e-4); the oracle needs about a
      second per coarse step at this size on 16 host cores.
  scvt_2621442_2caps (2,621,442 cells, two fine regions with M = 8 and 4):
      1 coarse step, FP64 and FP32 + compensation.
"""
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


def gpu(w, n, precision):
    with lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=precision) as m:
        m.step(n)
        h, u, d = m.read()
    return h, u


@pytest.fixture(scope="module")
def cfg2():
    w = W.workload("scvt_40962")
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    h100, u100 = o.lts3(w.h0, w.u0, cl, el, w.M, w.dt, 100, g=w.g)
    h500, u500 = o.lts3(h100, u100, cl, el, w.M, w.dt, 400, g=w.g)
    return w, (h100, u100), (h500, u500)


@pytest.fixture(scope="module")
def cfg3():
    w = W.workload("scvt_655362")
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    return w, o.lts3(w.h0, w.u0, cl, el, w.M, w.dt, 100, g=w.g)


def test_cfg2_fp64_100_steps(cfg2):
    w, (rh, ru), _ = cfg2
    h, u = gpu(w, 100, lts.LTS_FP64)
    print(f"cfg2 FP64 after 100 coarse steps: h {rel(h, rh):.3e}, u {rel(u, ru):.3e}")
    assert rel(h, rh) <= TOL64 and rel(u, ru) <= TOL64, (rel(h, rh), rel(u, ru))


def test_cfg2_fp32_500_steps(cfg2):
    w, _, (rh, ru) = cfg2
    h, u = gpu(w, 500, lts.LTS_FP32)
    print(f"cfg2 FP32 after 500 coarse steps: h {rel(h, rh):.3e}, u {rel(u, ru):.3e}")
    assert rel(h, rh) <= TOL32_H and rel(u, ru) <= TOL32_U, (rel(h, rh), rel(u, ru))


def test_cfg3_fp64_100_steps(cfg3):
    w, (rh, ru) = cfg3
    h, u = gpu(w, 100, lts.LTS_FP64)
    print(f"cfg3 FP64 after 100 coarse steps: h {rel(h, rh):.3e}, u {rel(u, ru):.3e}")
    assert rel(h, rh) <= TOL64 and rel(u, ru) <= TOL64, (rel(h, rh), rel(u, ru))


def test_cfg3_fp32_100_steps(cfg3):
    w, (rh, ru) = cfg3
    h, u = gpu(w, 100, lts.LTS_FP32)
    print(f"cfg3 FP32 after 100 coarse steps: h {rel(h, rh):.3e}, u {rel(u, ru):.3e}")
    assert rel(h, rh) <= TOL32_H and rel(u, ru) <= TOL32_U, (rel(h, rh), rel(u, ru))


@pytest.fixture(scope="module")
def cfg5():
    """2,621,442-cell sphere with two refined caps (8:1 with M = 8, 4:1 with
    M = 4) as two fine regions sharing the coarse step, ridges and noise."""
    w = W.workload("scvt_2621442_2caps")
    o = oracle.Oracle(w.mesh)
    return w, o.lts3_multi(w.h0, w.u0, w.fine_mask, list(w.M), w.dt, 1, g=w.g)


def test_cfg5_fp64_1_step(cfg5):
    w, (rh, ru) = cfg5
    h, u = gpu(w, 1, lts.LTS_FP64)
    assert rel(h, rh) <= TOL64 and rel(u, ru) <= TOL64, (rel(h, rh), rel(u, ru))


def test_cfg5_fp32_1_step(cfg5):
    w, (rh, ru) = cfg5
    h, u = gpu(w, 1, lts.LTS_FP32)
    assert rel(h, rh) <= TOL32_H and rel(u, ru) <= TOL32_U, (rel(h, rh), rel(u, ru))
