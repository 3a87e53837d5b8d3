"""Host I/O through the C ABI: lts_write, lts_read_async and lts_sync.
Copies run on their own streams and overlap the state's work, so these
tests check that every read sees exactly the state as it stood when it was
enqueued and every write replaces it in order (bitwise against the
synchronous write / step / read loop)."""
import numpy as np
import pytest

from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def sphw():
    return W.workload("scvt_2562")


def pinned(n):
    return torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()


def model(w, precision=lts.LTS_FP32):
    return lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=precision)


def inputs(w, k):
    rng = np.random.default_rng(100 + k)
    return w.h0 * (1.0 + 1e-4 * rng.standard_normal(w.nCells)), w.u0 * (1.0 + 0.05 * k)


@pytest.mark.parametrize("precision", [lts.LTS_FP32, lts.LTS_FP64])
def test_streamed_states_equal_round_trips(sphw, precision):
    """write(state k) / step / read_async for 6 different states with one
    sync at the end equals write / step / read per state."""
    nC, nE, n = sphw.nCells, int(sphw.mesh["nEdges"]), 6
    ref = []
    with model(sphw, precision) as m:
        for k in range(n):
            h, u = inputs(sphw, k)
            m.write(h, u)
            m.step(2)
            hr, ur, dr = m.read()
            ref.append((hr.copy(), ur.copy(), dr))
    hin = [pinned(nC) for _ in range(n)]
    uin = [pinned(nE) for _ in range(n)]
    hout = [pinned(nC) for _ in range(n)]
    uout = [pinned(nE) for _ in range(n)]
    with model(sphw, precision) as m:
        for k in range(n):
            hin[k][:], uin[k][:] = inputs(sphw, k)
            m.write(hin[k], uin[k])
            m.step(2)
            m.read_async(hout[k], uout[k], diag=True)
        diags = m.sync()
    assert len(diags) == n
    for k in range(n):
        assert np.array_equal(hout[k], ref[k][0]) and np.array_equal(uout[k], ref[k][1]), k
        assert diags[k]["mass"] == ref[k][2]["mass"] and diags[k]["energy"] == ref[k][2]["energy"]


def test_read_sees_the_state_when_enqueued(sphw):
    """A read enqueued before more steps returns the earlier state."""
    nC, nE = sphw.nCells, int(sphw.mesh["nEdges"])
    with model(sphw) as m:
        m.step(3)
        h3, u3, _ = m.read()
    with model(sphw) as m:
        ha, ua = pinned(nC), pinned(nE)
        m.step(3)
        m.read_async(ha, ua)
        m.step(4)
        m.sync()
        h7, _, _ = m.read()
    assert np.array_equal(ha, h3) and np.array_equal(ua, u3)
    assert not np.array_equal(h7, h3)


def test_writes_apply_in_order(sphw):
    """Two writes in a row: the later one wins, as if the first never came."""
    ha, ua = inputs(sphw, 1)
    hb, ub = inputs(sphw, 2)
    with model(sphw) as m:
        m.write(hb, ub)
        m.step(2)
        ref = m.read()
    with model(sphw) as m:
        m.write(ha, ua)
        m.write(hb, ub)
        m.step(2)
        got = m.read()
    assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1])


def test_too_many_pending_diagnostics_is_an_error(sphw):
    with model(sphw) as m:
        for _ in range(16):
            m.read_async(diag=True)
        with pytest.raises(lts.LtsError) as ei:
            m.read_async(diag=True)
        assert ei.value.code == lts.LTS_EINVAL
        assert len(m.sync()) == 16


def test_nonfinite_is_reported_by_sync(sphw):
    h0 = sphw.h0.copy()
    h0[10] = -5.0
    with lts.Model(sphw.mesh, sphw.fine_mask, sphw.M, h0, sphw.u0, sphw.dt, precision=lts.LTS_FP32) as m:
        m.step(1)
        m.read_async(pinned(sphw.nCells), None)
        with pytest.raises(lts.LtsError) as ei:
            m.sync()
        assert ei.value.code == lts.LTS_ENONFINITE
        m.write(sphw.h0, sphw.u0)
        m.step(1)
        m.sync()     # the flag was cleared by the failing sync


@pytest.mark.parametrize("precision", [lts.LTS_FP32, lts.LTS_FP64])
def test_snapshot_diagnostics_equal_state_diagnostics(sphw, precision):
    """lts_read's diagnostics run over an FP64 snapshot of the state beside
    the following work; they equal the reduction over the state itself
    (lts_diagnostics_noalloc, same blocking) to the last bit."""
    out = torch.zeros(2, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    with model(sphw, precision) as m:
        m.step(3)
        lts.lts_diagnostics_noalloc(m.state_h, out.data_ptr())
        _, _, d = m.read()
        got = out.cpu().numpy()
    assert got[0] == d["mass"] and got[1] == d["energy"]


def test_async_diagnostics_kept_by_the_binding(sphw):
    """Model.read_async keeps the diagnostics record alive until sync()."""
    with model(sphw, lts.LTS_FP64) as m:
        m.step(2)
        _, _, ref = m.read()
        for _ in range(3):
            m.read_async(diag=True)           # return value dropped
        import gc
        gc.collect()
        ds = m.sync()
    assert len(ds) == 3 and all(d["mass"] == ref["mass"] and d["energy"] == ref["energy"] for d in ds)
