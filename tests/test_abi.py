"""The C ABI: liblts.so loads without a GPU and exports every function that
include/lts.h declares; host-only entry points work without a GPU."""
import ctypes
import re
from pathlib import Path

import numpy as np

from paper_2106_07154_gb300 import lts

HEADER = Path(__file__).resolve().parent.parent / "include" / "lts.h"


def declared_functions():
    text = HEADER.read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lts_[a-z0-9_]+)\s*\(", text, re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("lts_mesh_create", "lts_regions_set", "lts_state_create", "lts_step", "lts_read",
                     "lts_build_scvt", "lts_build_hex_periodic", "lts_last_error"):
        assert required in names


def test_library_exports_every_declared_function():
    L = ctypes.CDLL(str(lts.LIB_PATH))
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_errors_without_gpu_are_reported_not_raised():
    mesh = lts.lts_build_hex_periodic(8, 8, 10e3, 1e-4)
    mh = lts.lts_mesh_create(mesh)
    rh = lts.lts_regions_set(mh, np.zeros(mesh["nCells"], np.int8), 3, 2)
    try:
        # bad arguments are rejected before any device work
        try:
            lts.lts_regions_set(mh, np.zeros(mesh["nCells"], np.int8), 4, 2)
            assert False, "order 4 should be rejected"
        except lts.LtsError as e:
            assert e.code == lts.LTS_EINVAL and "order" in str(e)
        r2 = lts.lts_regions_set(mh, np.zeros(mesh["nCells"], np.int8), 2, 2)   # LTS2
        lts.lts_regions_destroy(r2)
        try:
            lts.lts_regions_set(mh, np.zeros(mesh["nCells"], np.int8), 3, 0)
            assert False, "M = 0 should be rejected"
        except lts.LtsError as e:
            assert e.code == lts.LTS_EINVAL
    finally:
        lts.lts_regions_destroy(rh)
        lts.lts_mesh_destroy(mh)


def test_mesh_validation_rejects_clockwise_rings():
    mesh = lts.lts_build_hex_periodic(8, 8, 10e3, 1e-4)
    bad = dict(mesh)
    # reverse the ring of cell 0 (edges, neighbours and vertices)
    n = int(bad["nEdgesOnCell"][0])
    for k in ("edgesOnCell", "cellsOnCell"):
        a = bad[k].copy()
        a[0, :n] = a[0, :n][::-1]
        bad[k] = a
    v = bad["verticesOnCell"].copy()
    v[0, :n] = np.roll(v[0, :n][::-1], -1)
    bad["verticesOnCell"] = v
    try:
        lts.lts_mesh_create(bad)
        assert False, "a clockwise ring should be rejected"
    except lts.LtsError as e:
        assert e.code == lts.LTS_EINVAL and "counter-clockwise" in str(e)


def test_regions_labels_match_band_counts():
    mesh = lts.lts_build_hex_periodic(16, 16, 10e3, 1e-4)
    fine = np.zeros(mesh["nCells"], np.int8)
    fine[:40] = 1
    mh = lts.lts_mesh_create(mesh)
    rh = lts.lts_regions_set(mh, fine, 3, 2)
    try:
        cl, el = lts.lts_regions_labels(rh, mesh["nCells"], mesh["nEdges"])
        c, e, v = lts.lts_regions_counts(rh)
        assert c.sum() == mesh["nCells"] and e.sum() == mesh["nEdges"] and v.sum() == mesh["nVertices"]
        assert len(c) == lts.NBANDS == len(lts.BAND_NAMES)
        # label 5 (coarse) = bands C1..C5 and C rest; label 3 = I1; 4 = I2
        assert (cl == 3).sum() == c[4] and (cl == 4).sum() == c[5] and (cl == 5).sum() == c[6:].sum()
        pc, pe, pv = lts.lts_regions_permutation(rh, mesh["nCells"], mesh["nEdges"], mesh["nVertices"])
        assert sorted(pc.tolist()) == list(range(mesh["nCells"]))
        assert sorted(pe.tolist()) == list(range(mesh["nEdges"]))
        assert sorted(pv.tolist()) == list(range(mesh["nVertices"]))
        # band order: labels are non-decreasing along the permutation
        assert np.all(np.diff(np.minimum(cl[pc], 5)) >= 0)
    finally:
        lts.lts_regions_destroy(rh)
        lts.lts_mesh_destroy(mh)


def test_regions_ordering_index_keeps_mesh_order_inside_bands():
    mesh = lts.lts_build_hex_periodic(16, 16, 10e3, 1e-4)
    fine = np.zeros(mesh["nCells"], np.int8)
    fine[100:140] = 1
    mh = lts.lts_mesh_create(mesh)
    rh = lts.lts_regions_set(mh, fine, 3, 2)
    try:
        nC, nE, nV = mesh["nCells"], mesh["nEdges"], mesh["nVertices"]
        c0, _, _ = lts.lts_regions_counts(rh)
        pc0, _, _ = lts.lts_regions_permutation(rh, nC, nE, nV)
        lts.lts_regions_ordering(rh, lts.LTS_ORDER_INDEX)
        c1, _, _ = lts.lts_regions_counts(rh)
        pc1, pe1, pv1 = lts.lts_regions_permutation(rh, nC, nE, nV)
        assert np.array_equal(c0, c1)                       # the bands do not move
        off = np.concatenate([[0], np.cumsum(c1)])
        for b in range(len(c1)):                            # mesh order inside each band
            seg = pc1[off[b]:off[b + 1]]
            assert np.all(np.diff(seg) > 0)
            assert sorted(seg.tolist()) == sorted(pc0[off[b]:off[b + 1]].tolist())
        assert not np.array_equal(pc0, pc1)                 # Hilbert order differs
        assert sorted(pe1.tolist()) == list(range(nE)) and sorted(pv1.tolist()) == list(range(nV))
        lts.lts_regions_ordering(rh, lts.LTS_ORDER_HILBERT)
        pc2, _, _ = lts.lts_regions_permutation(rh, nC, nE, nV)
        assert np.array_equal(pc0, pc2)
        try:
            lts.lts_regions_ordering(rh, 5)
            assert False, "ordering 5 should be rejected"
        except lts.LtsError as e:
            assert e.code == lts.LTS_EINVAL
    finally:
        lts.lts_regions_destroy(rh)
        lts.lts_mesh_destroy(mh)


def _two_disks(mesh, radius):
    x, y = mesh["xCell"], mesh["yCell"]
    Lx, Ly = mesh["period_x"], mesh["period_y"]
    rid = np.zeros(mesh["nCells"], np.int8)
    for r, (cx, cy) in enumerate([(0.25 * Lx, 0.25 * Ly), (0.75 * Lx, 0.75 * Ly)], start=1):
        dx = (x - cx) - Lx * np.round((x - cx) / Lx)
        dy = (y - cy) - Ly * np.round((y - cy) / Ly)
        rid[dx * dx + dy * dy <= radius ** 2] = r
    return rid


def test_regions_multi_blocks_and_rejection():
    """Several fine regions (host only): every region's near bands form one
    contiguous block in the band-ordered arrays, the far coarse cells the
    last; the band counts equal those of the union; regions whose fine,
    interface and first coarse layers touch are rejected."""
    mesh = lts.lts_build_hex_periodic(32, 32, 10e3, 1e-4)
    rid = _two_disks(mesh, 25e3)
    mh = lts.lts_mesh_create(mesh)
    try:
        r2 = lts.lts_regions_set_multi(mh, rid, [4, 2])
        r1 = lts.lts_regions_set(mh, (rid > 0).astype(np.int8), 3, 4)
        c2, _, _ = lts.lts_regions_counts(r2)
        c1, _, _ = lts.lts_regions_counts(r1)
        assert np.array_equal(c1, c2)
        l2, _ = lts.lts_regions_labels(r2, mesh["nCells"], mesh["nEdges"])
        l1, _ = lts.lts_regions_labels(r1, mesh["nCells"], mesh["nEdges"])
        assert np.array_equal(l1, l2)
        pc, _, _ = lts.lts_regions_permutation(r2, mesh["nCells"], mesh["nEdges"], mesh["nVertices"])
        # new order: region 1's fine cells all come before region 2's
        pos = np.empty(mesh["nCells"], np.int64)
        pos[pc] = np.arange(mesh["nCells"])
        assert pos[rid == 1].max() < pos[rid == 2].min()
        lts.lts_regions_destroy(r1)
        lts.lts_regions_destroy(r2)
        close = _two_disks(mesh, 75e3)      # disks nearly touching
        try:
            lts.lts_regions_set_multi(mh, close, [4, 2])
            assert False, "touching regions should be rejected"
        except lts.LtsError as e:
            assert e.code == lts.LTS_EINVAL and "too close" in str(e)
        try:
            lts.lts_regions_set_multi(mh, rid, [4, 0])
            assert False, "M = 0 should be rejected"
        except lts.LtsError as e:
            assert e.code == lts.LTS_EINVAL
    finally:
        lts.lts_mesh_destroy(mh)


CITATION = re.compile(r"Eq\.|Eqs\.|Algorithm|Appendix|Section|Remark|no\s+(?:\*\s+)?counterpart")


def declaration_comments():
    """Each declared function with the comment block nearest above it (a
    comment documents the declarations that follow it up to the next one)."""
    text = HEADER.read_text()
    out, last = {}, ""
    # block comments that open a line (field comments inside structs do not)
    for m in re.finditer(r"^/\*.*?\*/|^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(lts_[a-z0-9_]+)\s*\(",
                         text, re.S | re.M):
        if m.group(0).lstrip().startswith("/*"):
            last = m.group(0)
        else:
            out[m.group(1)] = last
    return out


def test_every_entry_point_cites_its_passage():
    """Every function include/lts.h declares names the passage of the paper
    it implements (equation, algorithm, section, appendix) or says that the
    paper has no counterpart."""
    docs = declaration_comments()
    assert set(docs) == set(declared_functions())
    missing = sorted(n for n, c in docs.items() if not CITATION.search(c))
    assert not missing, missing
