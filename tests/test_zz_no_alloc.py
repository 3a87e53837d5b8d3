"""The allocation-free diagnostics entry point (lts_diagnostics_noalloc).

Callers that cannot allocate device memory when they need the diagnostics
(inside a stream capture, or with a pool that must not grow) get mass and
energy into memory they already own; the reduction's partial sums live in a
fixed array inside the library.  This file runs last so that a failure here
does not hide the other tests.
"""
import numpy as np
import pytest

from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
def test_noalloc_diagnostics_match_lts_read(precision):
    import torch

    w = W.workload("scvt_2562")
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, precision=precision) as m:
        for nsteps in (3, 2):            # two calls in a row on an advancing state
            m.step(nsteps)
            lts.lts_diagnostics_noalloc(m.state_h, out.data_ptr())
            _, _, ref = m.read()         # synchronises the state's stream
            got = out.cpu().numpy()
            assert np.isfinite(got).all()
            assert abs(got[0] - ref["mass"]) <= 1e-14 * abs(ref["mass"])
            assert abs(got[1] - ref["energy"]) <= 1e-14 * abs(ref["energy"])
