"""Ensembles of independent meshes (lts_ensemble_*) through the C ABI.

Every member of an ensemble sees exactly the arithmetic of its own
stand-alone coarse step (same kernels, same per-element operation order;
only the index space is packed), so each member's state after n ensemble
steps must equal the member stepped alone, bit for bit.  The members here
have uneven sizes, different M (2, 4, 8) and dt, a planar hexagon mesh among
spheres, and one member without fine cells.  One member is also compared
with the FP64 oracle at the FP64 tolerance.
"""
import numpy as np
import pytest

import oracle
from paper_2106_07154_gb300 import lts
from paper_2106_07154_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def members():
    ws = [
        W.workload("scvt_2562"),                                                  # 4:1, M = 4
        W.sphere_cap(n=1500, ratio=2.0, M=2, seed=3, lloyd_iters=60, name="e1"),  # 2:1, M = 2
        W.sphere_cap(n=3000, ratio=8.0, M=8, seed=5, lloyd_iters=60, name="e2"),  # 8:1, M = 8
        W.workload("hex_1024"),                                                   # plane, M = 2
    ]
    nofine = W.workload("scvt_2562")
    nofine.fine_mask = np.zeros(nofine.nCells, np.int8)
    nofine.dt = nofine.dt / nofine.M          # coarse SSPRK3 on the refined cap: its fine CFL
    ws.append(nofine)
    return ws


def models(ws, precision, **kw):
    return [lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=precision, **kw)
            for w in ws]


def alone(ws, precision, n):
    out = []
    for m in models(ws, precision):
        m.step(n)
        out.append(m.read())
        m.close()
    return out


def rel(a, b):
    return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))


@pytest.mark.parametrize("precision", [lts.LTS_FP64, lts.LTS_FP32])
def test_ensemble_members_equal_standalone_bitwise(members, precision):
    n1, n2 = 3, 2
    ref1 = alone(members, precision, n1)
    ref2 = alone(members, precision, n1 + n2)
    ms = models(members, precision)
    with lts.Ensemble(ms) as e:
        st = e.stats()
        assert st["cells"] == sum(w.nCells for w in members)
        e.step(n1)
        for i, w in enumerate(members):        # read, then keep stepping
            h, u, d = e.read(i)
            assert np.array_equal(h, ref1[i][0]) and np.array_equal(u, ref1[i][1]), f"member {i}"
            assert d["steps"] == n1 and abs(d["time"] - n1 * w.dt) <= 1e-9 * n1 * w.dt
            assert d["mass"] == ref1[i][2]["mass"]
        e.step(n2)
        for i in range(len(members)):
            h, u, _ = e.read(i)
            assert np.array_equal(h, ref2[i][0]) and np.array_equal(u, ref2[i][1]), f"member {i}"
    for m in ms:
        m.close()


@pytest.mark.parametrize("use_graph,persistent,pdl", [(False, False, True), (True, True, True),
                                                      (False, True, False), (True, False, False)])
def test_ensemble_launch_modes_identical(members, use_graph, persistent, pdl):
    ref = alone(members, lts.LTS_FP32, 4)
    ms = models(members, lts.LTS_FP32)
    with lts.Ensemble(ms, use_graph=use_graph, persistent=persistent, pdl=pdl) as e:
        e.step(4)
        for i in range(len(members)):
            h, u, _ = e.read(i)
            assert np.array_equal(h, ref[i][0]) and np.array_equal(u, ref[i][1]), f"member {i}"
    for m in ms:
        m.close()


def test_ensemble_member_matches_oracle(members):
    w = members[2]                      # M = 8 member
    n = 10
    ms = models(members, lts.LTS_FP64)
    with lts.Ensemble(ms) as e:
        e.step(n)
        h, u, _ = e.read(2)
    for m in ms:
        m.close()
    o = oracle.Oracle(w.mesh)
    cl, el = o.regions(w.fine_mask)
    rh, ru = o.lts3(w.h0, w.u0, cl, el, w.M, w.dt, n, g=w.g)
    assert rel(h, rh) <= 1e-12 and rel(u, ru) <= 1e-12


def test_ensemble_rejects_mixed_precision(members):
    a = models(members[:1], lts.LTS_FP64)
    b = models(members[1:2], lts.LTS_FP32)
    with pytest.raises(lts.LtsError) as ei:
        lts.Ensemble(a + b)
    assert ei.value.code == lts.LTS_EINVAL
    with pytest.raises(lts.LtsError):
        lts.Ensemble(a + a)             # a member twice
    for m in a + b:
        m.close()


def test_ensemble_write_restarts_one_member(members):
    ref = alone(members, lts.LTS_FP64, 2)
    ms = models(members, lts.LTS_FP64)
    with lts.Ensemble(ms) as e:
        e.step(3)
        w = members[1]
        e.write(1, w.h0, w.u0, 0.0, 0)           # member 1 starts over
        e.step(2)
        h, u, d = e.read(1)
        assert np.array_equal(h, ref[1][0]) and np.array_equal(u, ref[1][1])
        assert d["steps"] == 2 and abs(d["time"] - 2 * w.dt) <= 1e-9 * w.dt
        h0, u0, d0 = e.read(0)                   # the others went on
        assert d0["steps"] == 5
    for m in ms:
        m.close()


def test_ensemble_pinned_round_trips(members):
    """Every member written from pinned memory, stepped, read back into the
    same buffers and written again (I/O is ordered by events, not host
    synchronisation): the results equal the standalone runs bit for bit."""
    torch = pytest.importorskip("torch")
    ref2 = alone(members, lts.LTS_FP64, 2)
    ref3 = alone(members, lts.LTS_FP64, 3)
    bufs = []
    for w in members:
        hb = torch.empty(w.nCells, dtype=torch.float64, pin_memory=True).numpy()
        ub = torch.empty(int(w.mesh["nEdges"]), dtype=torch.float64, pin_memory=True).numpy()
        hb[:] = w.h0
        ub[:] = w.u0
        bufs.append((hb, ub))
    ms = models(members, lts.LTS_FP64)
    with lts.Ensemble(ms) as e:
        e.step(4)                                # state to be replaced
        for i, (hb, ub) in enumerate(bufs):
            e.write(i, hb, ub, 0.0, 0)
        e.step(2)
        for i, (hb, ub) in enumerate(bufs):
            e.read(i, hb, ub)
            assert np.array_equal(hb, ref2[i][0]) and np.array_equal(ub, ref2[i][1]), i
        for i, (hb, ub) in enumerate(bufs):
            e.write(i, hb, ub, 0.0, 2)
        e.step(1)
        for i, (hb, ub) in enumerate(bufs):
            e.read(i, hb, ub)
            assert np.array_equal(hb, ref3[i][0]) and np.array_equal(ub, ref3[i][1]), i
    for m in ms:
        m.close()


def test_ensemble_async_reads(members):
    """lts_ensemble_read_async + lts_ensemble_sync: each read sees its member
    as it stood when the read was enqueued, even when the same member is
    read again after more steps before the sync; the values and diagnostics
    equal synchronous reads bit for bit."""
    torch = pytest.importorskip("torch")
    ms = models(members, lts.LTS_FP64)
    ref = alone(members, lts.LTS_FP64, 2)
    ref3 = alone(members, lts.LTS_FP64, 3)
    pin = lambda n: torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
    with lts.Ensemble(ms) as e:
        e.step(2)
        outs, diags = [], []
        for i, w in enumerate(members):
            hb, ub = pin(w.nCells), pin(int(w.mesh["nEdges"]))
            diags.append(e.read_async(i, hb, ub, diag=True))
            outs.append((hb, ub))
        e.step(1)
        h3, u3 = pin(members[0].nCells), pin(int(members[0].mesh["nEdges"]))
        e.read_async(0, h3, u3)
        e.sync()
        for i in range(len(members)):
            assert np.array_equal(outs[i][0], ref[i][0]) and np.array_equal(outs[i][1], ref[i][1]), i
            assert diags[i].mass == ref[i][2]["mass"] and diags[i].energy == ref[i][2]["energy"]
            assert diags[i].steps == 2
        assert np.array_equal(h3, ref3[0][0]) and np.array_equal(u3, ref3[0][1])
    for m in ms:
        m.close()


def test_ensemble_async_diagnostics_kept_by_the_binding(members):
    """The binding keeps each asynchronous read's diagnostics record alive
    until the sync (the library writes it then), so a caller may drop it."""
    ms = models(members, lts.LTS_FP64)
    ref = alone(members, lts.LTS_FP64, 1)
    with lts.Ensemble(ms) as e:
        e.step(1)
        for i in range(len(members)):
            e.read_async(i, diag=True)        # return value dropped
        import gc
        gc.collect()
        ds = e.sync()
        assert len(ds) == len(members)
        for i, d in enumerate(ds):
            assert d["mass"] == ref[i][2]["mass"] and d["energy"] == ref[i][2]["energy"], i
    for m in ms:
        m.close()
