"""The allocation-free diagnostics entry point (lts_diagnostics_noalloc).

Some callers cannot allocate device memory when they need the diagnostics:
hosts whose device memory comes from a fixed pool that must not grow, or
time loops that forbid allocation because cudaMalloc may synchronise the
device.  They get mass and energy into memory they already own; the
reduction's partial sums live in a fixed array inside the library.  This
file runs last so that a failure here does not hide the other tests.
"""
import numpy as np
import pytest

from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision,layers", [(lts.LTS_FP64, 1), (lts.LTS_FP32, 1), (lts.LTS_FP64, 2)])
def test_noalloc_diagnostics_match_lts_read(precision, layers):
    """Two calls in a row on an advancing state equal lts_read's diagnostics
    (the same blocking, so to the last bit; the bound leaves room only for
    roundoff)."""
    import torch

    w = W.workload("scvt_2562")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    h0 = np.tile(w.h0, (layers, 1)) + np.arange(layers)[:, None]   # layers differ
    u0 = np.tile(w.u0, (layers, 1))
    with lts.Model(w.mesh, w.fine_mask, w.M, h0, u0, w.dt, precision=precision, layers=layers) as m:
        for nsteps in (3, 2):            # two calls in a row on an advancing state
            m.step(nsteps)
            lts.lts_diagnostics_noalloc(m.state_h, out.data_ptr())
            _, _, ref = m.read()         # synchronises the state's stream
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert abs(got[0] - ref["mass"]) <= 1e-14 * abs(ref["mass"])
            assert abs(got[1] - ref["energy"]) <= 1e-14 * abs(ref["energy"])


def test_noalloc_rejects_states_beyond_its_array():
    """cells x layers above 1,048,576 is refused with LTS_EINVAL before any
    launch, and the caller's output stays untouched."""
    import torch

    w = W.workload("scvt_2562")
    L = 1_048_576 // w.mesh["nCells"] + 1
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    with lts.Model(w.mesh, w.fine_mask, w.M, np.tile(w.h0, (L, 1)), np.tile(w.u0, (L, 1)), w.dt,
                   precision=lts.LTS_FP32, layers=L) as m:
        with pytest.raises(lts.LtsError) as ei:
            lts.lts_diagnostics_noalloc(m.state_h, out.data_ptr())
        assert ei.value.code == lts.LTS_EINVAL and "cells x layers" in str(ei.value)
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == -1.0)
