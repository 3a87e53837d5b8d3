"""ctypes binding of liblts.so (include/lts.h), same names as the C ABI.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Loading fails loudly if the in-tree liblts.so is missing; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

PKG = Path(__file__).resolve().parent
LIB_PATH = PKG / "liblts.so"

LTS_OK = 0
LTS_EINVAL = -1
LTS_ENOMEM = -2
LTS_ECUDA = -3
LTS_ENONFINITE = -4
LTS_ETIMEOUT = -5
LTS_ENODEV = -6
LTS_FP32 = 0
LTS_FP64 = 1
LTS_MODE_LTS = 0
LTS_MODE_LTS3 = 0
LTS_MODE_SSPRK3 = 1
LTS_MODE_SSPRK2 = 2
LTS_NKINDS = 4
KIND_NAMES = ("vertex", "ring", "edge", "tile")
PATH_THREE = 0
PATH_FUSED = 1
LTS_ORDER_HILBERT = 0
LTS_ORDER_INDEX = 1
LTS_TUNE_ORDERING = 1
LTS_COARSE_FAR = 0      # the default
LTS_COARSE_STEP4 = 1
LTS_COARSE_SERIAL = 2

NBANDS = 12
BAND_NAMES = ("F_deep", "F3", "F2", "F1", "I1", "I2", "C1", "C2", "C3", "C4", "C5", "C_rest")

_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)


class LtsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"liblts error {code}: {msg}")
        self.code = code


class lts_mesh_desc(C.Structure):
    _fields_ = [
        ("nCells", C.c_int32), ("nEdges", C.c_int32), ("nVertices", C.c_int32),
        ("maxEdges", C.c_int32), ("on_sphere", C.c_int32), ("radius", C.c_double),
        ("period_x", C.c_double), ("period_y", C.c_double),
        ("xCell", _DP), ("yCell", _DP), ("zCell", _DP),
        ("xEdge", _DP), ("yEdge", _DP), ("zEdge", _DP),
        ("xVertex", _DP), ("yVertex", _DP), ("zVertex", _DP),
        ("nEdgesOnCell", _IP), ("edgesOnCell", _IP), ("cellsOnCell", _IP),
        ("verticesOnCell", _IP), ("cellsOnEdge", _IP), ("verticesOnEdge", _IP),
        ("edgesOnVertex", _IP), ("cellsOnVertex", _IP),
        ("areaCell", _DP), ("areaTriangle", _DP), ("kiteAreasOnVertex", _DP),
        ("dcEdge", _DP), ("dvEdge", _DP), ("fVertex", _DP), ("bottom", _DP),
        ("nEdgesOnEdge", _IP), ("edgesOnEdge", _IP), ("weightsOnEdge", _DP),
    ]


class lts_cap(C.Structure):
    _fields_ = [("lon", C.c_double), ("lat", C.c_double), ("radius", C.c_double),
                ("width", C.c_double), ("ratio", C.c_double)]


class lts_density(C.Structure):
    _fields_ = [("ncaps", C.c_int32), ("cap", lts_cap * 4)]


class lts_params(C.Structure):
    _fields_ = [("g", C.c_double), ("dt", C.c_double), ("precision", C.c_int32),
                ("mode", C.c_int32), ("compensated", C.c_int32), ("use_graph", C.c_int32),
                ("block_size", C.c_int32), ("profile", C.c_int32), ("pdl", C.c_int32),
                ("kernel_path", C.c_int32), ("stream", C.c_void_p), ("no_l2_hints", C.c_int32),
                ("layers", C.c_int32), ("ring_occupancy", C.c_int32), ("coarse_schedule", C.c_int32),
                ("elems_per_thread", C.c_int32)]


class lts_tune_entry(C.Structure):
    _fields_ = [("block_size", C.c_int32), ("kernel_path", C.c_int32), ("pdl", C.c_int32),
                ("l2_hints", C.c_int32), ("coarse_schedule", C.c_int32), ("ordering", C.c_int32),
                ("ring_occupancy", C.c_int32), ("elems_per_thread", C.c_int32), ("ms", C.c_double)]


class lts_tune_report(C.Structure):
    _fields_ = [("candidates", C.c_int32), ("ordering", C.c_int32), ("best_ms", C.c_double),
                ("default_ms", C.c_double), ("entry", lts_tune_entry * 32)]


class lts_ensemble_params(C.Structure):
    _fields_ = [("use_graph", C.c_int32), ("pdl", C.c_int32), ("persistent", C.c_int32),
                ("stream", C.c_void_p)]


class lts_diag(C.Structure):
    _fields_ = [("mass", C.c_double), ("energy", C.c_double), ("time", C.c_double),
                ("steps", C.c_int64)]


# (field, dtype, length key) of every array in lts_mesh_desc
_CELL, _EDGE, _VERT = "nCells", "nEdges", "nVertices"
MESH_ARRAYS = [
    ("xCell", np.float64, (_CELL, 1)), ("yCell", np.float64, (_CELL, 1)),
    ("zCell", np.float64, (_CELL, 1)), ("xEdge", np.float64, (_EDGE, 1)),
    ("yEdge", np.float64, (_EDGE, 1)), ("zEdge", np.float64, (_EDGE, 1)),
    ("xVertex", np.float64, (_VERT, 1)), ("yVertex", np.float64, (_VERT, 1)),
    ("zVertex", np.float64, (_VERT, 1)),
    ("nEdgesOnCell", np.int32, (_CELL, 1)), ("edgesOnCell", np.int32, (_CELL, "maxEdges")),
    ("cellsOnCell", np.int32, (_CELL, "maxEdges")), ("verticesOnCell", np.int32, (_CELL, "maxEdges")),
    ("cellsOnEdge", np.int32, (_EDGE, 2)), ("verticesOnEdge", np.int32, (_EDGE, 2)),
    ("edgesOnVertex", np.int32, (_VERT, 3)), ("cellsOnVertex", np.int32, (_VERT, 3)),
    ("areaCell", np.float64, (_CELL, 1)), ("areaTriangle", np.float64, (_VERT, 1)),
    ("kiteAreasOnVertex", np.float64, (_VERT, 3)), ("dcEdge", np.float64, (_EDGE, 1)),
    ("dvEdge", np.float64, (_EDGE, 1)), ("fVertex", np.float64, (_VERT, 1)),
    ("bottom", np.float64, (_CELL, 1)),
]
SCALARS = ["nCells", "nEdges", "nVertices", "maxEdges", "on_sphere", "radius", "period_x",
           "period_y"]

_lib = None


def lib():
    """The loaded liblts.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not LIB_PATH.exists():
            raise RuntimeError(f"{LIB_PATH} is missing: run __graft_entry__.build() first")
        L = C.CDLL(str(LIB_PATH))
        L.lts_last_error.restype = C.c_char_p
        L.lts_build_hex_periodic.argtypes = [C.c_int32, C.c_int32, C.c_double, C.c_double,
                                             C.POINTER(lts_mesh_desc)]
        L.lts_build_scvt.argtypes = [C.c_int64, C.c_uint64, C.POINTER(lts_density), C.c_int32,
                                     C.c_double, C.POINTER(lts_mesh_desc)]
        L.lts_mesh_desc_free.argtypes = [C.POINTER(lts_mesh_desc)]
        L.lts_mesh_desc_free.restype = None
        if hasattr(L, "lts_mesh_create"):
            L.lts_mesh_create.argtypes = [C.POINTER(lts_mesh_desc), C.POINTER(C.c_void_p)]
            L.lts_mesh_destroy.argtypes = [C.c_void_p]
            L.lts_mesh_destroy.restype = None
            L.lts_regions_set.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32,
                                          C.POINTER(C.c_void_p)]
            L.lts_regions_destroy.argtypes = [C.c_void_p]
            L.lts_regions_destroy.restype = None
            L.lts_regions_labels.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
            L.lts_regions_counts.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.lts_regions_tiling.argtypes = [C.c_void_p, C.c_int32]
            L.lts_regions_ordering.argtypes = [C.c_void_p, C.c_int32]
            L.lts_regions_set_multi.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p, C.c_int32,
                                                C.c_int32, C.POINTER(C.c_void_p)]
            L.lts_autotune.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.POINTER(lts_params), C.c_int32, C.c_int32,
                                       C.POINTER(lts_params), C.POINTER(lts_tune_report)]
            L.lts_regions_permutation.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
            L.lts_state_create.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                           C.POINTER(lts_params), C.POINTER(C.c_void_p)]
            L.lts_state_destroy.argtypes = [C.c_void_p]
            L.lts_state_destroy.restype = None
            L.lts_step.argtypes = [C.c_void_p, C.c_int32]
            L.lts_read.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(lts_diag)]
            L.lts_write.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int64]
            L.lts_read_async.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(lts_diag)]
            L.lts_sync.argtypes = [C.c_void_p]
            L.lts_step_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p]
            L.lts_diagnostics_noalloc.argtypes = [C.c_void_p, C.c_void_p]
            L.lts_ensemble_create.argtypes = [C.c_void_p, C.c_int32, C.POINTER(lts_ensemble_params),
                                              C.POINTER(C.c_void_p)]
            L.lts_ensemble_destroy.argtypes = [C.c_void_p]
            L.lts_ensemble_destroy.restype = None
            L.lts_ensemble_step.argtypes = [C.c_void_p, C.c_int32]
            L.lts_ensemble_read_async.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                                  C.POINTER(lts_diag)]
            L.lts_ensemble_sync.argtypes = [C.c_void_p]
            L.lts_ensemble_read.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                            C.POINTER(lts_diag)]
            L.lts_ensemble_write.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p,
                                             C.c_double, C.c_int64]
            L.lts_ensemble_stats.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p]
        _lib = L
    return _lib


def lts_last_error() -> str:
    return lib().lts_last_error().decode()


def _check(rc: int):
    if rc != LTS_OK:
        raise LtsError(rc, lts_last_error())


def _desc_to_dict(d: lts_mesh_desc) -> dict:
    out = {k: getattr(d, k) for k in SCALARS}
    for name, dt, (nkey, width) in MESH_ARRAYS:
        ptr = getattr(d, name)
        if not ptr:
            out[name] = None
            continue
        n = out[nkey] * (out[width] if isinstance(width, str) else width)
        arr = np.ctypeslib.as_array(ptr, shape=(n,)).copy().astype(dt, copy=False)
        if not isinstance(width, int) or width != 1:
            arr = arr.reshape(out[nkey], -1)
        out[name] = arr
    return out


def lts_build_hex_periodic(nx: int, ny: int, dc: float, f0: float) -> dict:
    """Doubly periodic hexagonal mesh as a dict of MPAS arrays (see include/lts.h)."""
    d = lts_mesh_desc()
    _check(lib().lts_build_hex_periodic(nx, ny, dc, f0, C.byref(d)))
    try:
        return _desc_to_dict(d)
    finally:
        lib().lts_mesh_desc_free(C.byref(d))


def lts_build_scvt(n: int, seed: int, caps, lloyd_iters: int, radius: float) -> dict:
    """Spherical SCVT; caps = list of (lon, lat, radius, width, ratio) in radians."""
    den = lts_density()
    den.ncaps = len(caps)
    for k, c in enumerate(caps):
        den.cap[k] = lts_cap(*map(float, c))
    d = lts_mesh_desc()
    _check(lib().lts_build_scvt(int(n), int(seed) & (2**64 - 1), C.byref(den), int(lloyd_iters),
                                float(radius), C.byref(d)))
    try:
        return _desc_to_dict(d)
    finally:
        lib().lts_mesh_desc_free(C.byref(d))


# ---------------------------------------------------------------------------
# device objects


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _dict_to_desc(mesh: dict):
    """lts_mesh_desc pointing into contiguous copies of the dict's arrays
    (returned alongside so they stay alive during the call)."""
    d = lts_mesh_desc()
    keep = []
    for k in SCALARS:
        setattr(d, k, mesh.get(k) or 0)
    for name, dt, _ in MESH_ARRAYS:
        v = mesh.get(name)
        if v is None:
            setattr(d, name, None)
            continue
        arr = _f64(v).ravel() if dt == np.float64 else _i32(v).ravel()
        keep.append(arr)
        ctype = C.c_double if dt == np.float64 else C.c_int32
        setattr(d, name, arr.ctypes.data_as(C.POINTER(ctype)))
    return d, keep


def lts_mesh_create(mesh: dict) -> C.c_void_p:
    d, keep = _dict_to_desc(mesh)
    h = C.c_void_p()
    _check(lib().lts_mesh_create(C.byref(d), C.byref(h)))
    return h


def lts_mesh_destroy(h):
    if h:
        lib().lts_mesh_destroy(h)


def lts_regions_set(mesh_h, fine_mask, order: int, M: int, interface_layers: int = 1):
    fm = np.ascontiguousarray(fine_mask, dtype=np.int8)
    h = C.c_void_p()
    _check(lib().lts_regions_set(mesh_h, fm.ctypes.data, order, M, interface_layers, C.byref(h)))
    return h


def lts_regions_set_multi(mesh_h, region_of_cell, Ms, order: int = 3, interface_layers: int = 1):
    rid = np.ascontiguousarray(region_of_cell, dtype=np.int8)
    Ms = np.ascontiguousarray(Ms, dtype=np.int32)
    h = C.c_void_p()
    _check(lib().lts_regions_set_multi(mesh_h, rid.ctypes.data, len(Ms), Ms.ctypes.data, order,
                                       interface_layers, C.byref(h)))
    return h


def lts_regions_destroy(h):
    if h:
        lib().lts_regions_destroy(h)


def lts_regions_labels(reg_h, nCells: int, nEdges: int):
    cl = np.zeros(nCells, np.int8)
    el = np.zeros(nEdges, np.int8)
    _check(lib().lts_regions_labels(reg_h, cl.ctypes.data, el.ctypes.data))
    return cl, el


def lts_regions_tiling(reg_h, tile_cells: int):
    _check(lib().lts_regions_tiling(reg_h, int(tile_cells)))


def lts_regions_ordering(reg_h, ordering: int):
    _check(lib().lts_regions_ordering(reg_h, int(ordering)))


def lts_regions_counts(reg_h):
    c = np.zeros(NBANDS, np.int64)
    e = np.zeros(NBANDS, np.int64)
    v = np.zeros(NBANDS, np.int64)
    _check(lib().lts_regions_counts(reg_h, c.ctypes.data, e.ctypes.data, v.ctypes.data))
    return c, e, v


def lts_regions_permutation(reg_h, nCells: int, nEdges: int, nVertices: int):
    pc = np.zeros(nCells, np.int32)
    pe = np.zeros(nEdges, np.int32)
    pv = np.zeros(nVertices, np.int32)
    _check(lib().lts_regions_permutation(reg_h, pc.ctypes.data, pe.ctypes.data, pv.ctypes.data))
    return pc, pe, pv


def make_params(g: float, dt: float, precision: int = LTS_FP32, mode: int = LTS_MODE_LTS3,
                compensated: bool = True, use_graph: bool = True, block_size: int = 0,
                profile: int = 0, stream: int | None = None, pdl: bool = True,
                kernel_path: int = 0, l2_hints: bool = True, coarse_schedule: int = 0,
                layers: int = 1, ring_occupancy: int = 0, elems_per_thread: int = 0):
    return lts_params(g, dt, precision, mode, int(compensated), int(use_graph), block_size,
                      int(profile), int(pdl), int(kernel_path), stream, int(not l2_hints),
                      int(layers), int(ring_occupancy), int(coarse_schedule), int(elems_per_thread))


def params_dict(p: lts_params) -> dict:
    return {"block_size": p.block_size, "kernel_path": p.kernel_path, "pdl": bool(p.pdl),
            "l2_hints": not p.no_l2_hints, "coarse_schedule": int(p.coarse_schedule),
            "layers": int(p.layers), "ring_occupancy": int(p.ring_occupancy),
            "elems_per_thread": int(p.elems_per_thread), "use_graph": bool(p.use_graph)}


def lts_autotune(mesh_h, reg_h, h0, u0, base: lts_params, steps: int = 20,
                 tune_ordering: bool = False):
    """Returns (best lts_params, report dict); see include/lts.h."""
    best = lts_params()
    rep = lts_tune_report()
    _check(lib().lts_autotune(mesh_h, reg_h, _f64(h0).ctypes.data, _f64(u0).ctypes.data,
                              C.byref(base), int(steps), LTS_TUNE_ORDERING if tune_ordering else 0,
                              C.byref(best), C.byref(rep)))
    table = [{f: getattr(e, f) for f, _ in lts_tune_entry._fields_}
             for e in rep.entry[:min(rep.candidates, 32)]]
    return best, {"candidates": rep.candidates, "ordering": rep.ordering, "best_ms": rep.best_ms,
                  "default_ms": rep.default_ms, "table": table}


def lts_state_create_p(mesh_h, reg_h, h0, u0, p: lts_params):
    h = C.c_void_p()
    _check(lib().lts_state_create(mesh_h, reg_h, _f64(h0).ctypes.data, _f64(u0).ctypes.data,
                                  C.byref(p), C.byref(h)))
    return h


def lts_state_create(mesh_h, reg_h, h0, u0, g: float, dt: float, precision: int = LTS_FP32,
                     mode: int = LTS_MODE_LTS3, compensated: bool = True, use_graph: bool = True,
                     block_size: int = 0, profile: int = 0, stream: int | None = None,
                     pdl: bool = True, kernel_path: int = 0, l2_hints: bool = True,
                     coarse_schedule: int = 0):
    p = make_params(g, dt, precision, mode, compensated, use_graph, block_size, profile, stream,
                    pdl, kernel_path, l2_hints, coarse_schedule)
    h = C.c_void_p()
    _check(lib().lts_state_create(mesh_h, reg_h, _f64(h0).ctypes.data, _f64(u0).ctypes.data,
                                  C.byref(p), C.byref(h)))
    return h


def lts_state_destroy(h):
    if h:
        lib().lts_state_destroy(h)


def lts_step(state_h, n_coarse: int):
    _check(lib().lts_step(state_h, int(n_coarse)))


def lts_read(state_h, nCells: int, nEdges: int, h_out=None, u_out=None):
    """Returns (h, u, diag dict); writes into h_out/u_out when given (e.g. pinned buffers)."""
    h = np.zeros(nCells) if h_out is None else h_out
    u = np.zeros(nEdges) if u_out is None else u_out
    d = lts_diag()
    rc = lib().lts_read(state_h, h.ctypes.data, u.ctypes.data, C.byref(d))
    _check(rc)
    return h, u, {"mass": d.mass, "energy": d.energy, "time": d.time, "steps": d.steps}


def lts_write(state_h, h, u, time: float = 0.0, steps: int = 0):
    _check(lib().lts_write(state_h, _f64(h).ctypes.data, _f64(u).ctypes.data, float(time),
                           int(steps)))


def _ptr(a):
    if a is None:
        return None
    if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"] or not a.flags["WRITEABLE"]:
        raise ValueError("output arrays must be writeable, C-contiguous float64")
    return a.ctypes.data


def lts_read_async(state_h, h_out=None, u_out=None, diag: bool = False):
    """Enqueues the copy of the state into h_out / u_out (float64 arrays the
    caller keeps alive; pinned for overlap).  Returns the lts_diag that the
    next lts_sync fills (None without diagnostics); the caller keeps it alive
    until then (Model.read_async does)."""
    d = lts_diag() if diag else None
    _check(lib().lts_read_async(state_h, _ptr(h_out), _ptr(u_out), C.byref(d) if d is not None else None))
    return d


def lts_sync(state_h):
    _check(lib().lts_sync(state_h))


def lts_step_stats(state_h):
    n = C.c_int32()
    b = np.zeros(LTS_NKINDS)
    ms = np.zeros(LTS_NKINDS)
    k = np.zeros(LTS_NKINDS, np.int32)
    _check(lib().lts_step_stats(state_h, C.byref(n), b.ctypes.data, ms.ctypes.data, k.ctypes.data))
    return {"launches": int(n.value), "bytes": b.tolist(), "ms": ms.tolist(),
            "launches_per_kind": k.tolist()}


def lts_diagnostics_noalloc(state_h, d_out_ptr: int):
    """Enqueues mass and energy of the current state into caller-owned device
    memory (2 doubles at d_out_ptr) without allocating; see include/lts.h."""
    _check(lib().lts_diagnostics_noalloc(state_h, C.c_void_p(int(d_out_ptr))))


def lts_ensemble_create(state_handles, use_graph: bool = True, pdl: bool = True,
                        persistent: bool = False, stream: int | None = None):
    arr = (C.c_void_p * len(state_handles))(*[C.c_void_p(h.value if isinstance(h, C.c_void_p) else h)
                                               for h in state_handles])
    p = lts_ensemble_params(int(use_graph), int(pdl), int(persistent), stream)
    out = C.c_void_p()
    _check(lib().lts_ensemble_create(arr, len(state_handles), C.byref(p), C.byref(out)))
    return out


def lts_ensemble_destroy(h):
    if h:
        lib().lts_ensemble_destroy(h)


def lts_ensemble_step(ens_h, n_coarse: int):
    _check(lib().lts_ensemble_step(ens_h, int(n_coarse)))


def lts_ensemble_read(ens_h, i: int, nCells: int, nEdges: int, h_out=None, u_out=None):
    h = np.zeros(nCells) if h_out is None else h_out
    u = np.zeros(nEdges) if u_out is None else u_out
    d = lts_diag()
    _check(lib().lts_ensemble_read(ens_h, int(i), h.ctypes.data, u.ctypes.data, C.byref(d)))
    return h, u, {"mass": d.mass, "energy": d.energy, "time": d.time, "steps": d.steps}


def lts_ensemble_read_async(ens_h, i: int, h_out=None, u_out=None, diag: bool = False):
    """Enqueues member i's copy into h_out / u_out (float64 arrays the caller
    keeps alive); returns the lts_diag the next lts_ensemble_sync fills, which
    the caller keeps alive until then (Ensemble.read_async does)."""
    d = lts_diag() if diag else None
    _check(lib().lts_ensemble_read_async(ens_h, int(i), _ptr(h_out), _ptr(u_out),
                                         C.byref(d) if d is not None else None))
    return d


def lts_ensemble_sync(ens_h):
    _check(lib().lts_ensemble_sync(ens_h))


def lts_ensemble_write(ens_h, i: int, h, u, time: float = 0.0, steps: int = 0):
    _check(lib().lts_ensemble_write(ens_h, int(i), _f64(h).ctypes.data, _f64(u).ctypes.data,
                                    float(time), int(steps)))


def lts_ensemble_stats(ens_h):
    n = C.c_int32()
    nseg = C.c_int32()
    cells = C.c_int64()
    b = np.zeros(LTS_NKINDS)
    _check(lib().lts_ensemble_stats(ens_h, C.byref(n), b.ctypes.data, C.byref(cells), C.byref(nseg)))
    return {"launches": int(n.value), "bytes": b.tolist(), "cells": int(cells.value),
            "segments": int(nseg.value)}


class Ensemble:
    """Several Models advanced together (one launch per phase for all)."""

    def __init__(self, models, use_graph: bool = True, pdl: bool = True, persistent: bool = False,
                 stream: int | None = None):
        self.models = list(models)
        self._pending = []
        self.h = None
        self.h = lts_ensemble_create([m.state_h for m in self.models], use_graph, pdl, persistent,
                                     stream)

    def step(self, n: int):
        lts_ensemble_step(self.h, n)

    def read(self, i: int, h_out=None, u_out=None):
        m = self.models[i]
        return lts_ensemble_read(self.h, i, m.nC, m.nE, h_out, u_out)

    def write(self, i: int, h, u, time=0.0, steps=0):
        lts_ensemble_write(self.h, i, h, u, time, steps)

    def read_async(self, i: int, h_out=None, u_out=None, diag: bool = False):
        """Enqueues member i's copy; h_out, u_out (and the returned record)
        are valid after sync()."""
        m = self.models[i]
        if h_out is not None and h_out.size != m.nC:
            raise ValueError("h_out must hold nCells values")
        if u_out is not None and u_out.size != m.nE:
            raise ValueError("u_out must hold nEdges values")
        d = lts_ensemble_read_async(self.h, i, h_out, u_out, diag)
        if d is not None:
            self._pending.append(d)   # the library writes it at the sync: keep it alive
        return d

    def sync(self):
        """Waits for the ensemble and its members; returns the diagnostics of
        the asynchronous reads since the last sync, in order."""
        pending, self._pending = self._pending, []
        lts_ensemble_sync(self.h)
        return [{"mass": d.mass, "energy": d.energy, "time": d.time, "steps": d.steps} for d in pending]

    def stats(self):
        return lts_ensemble_stats(self.h)

    def close(self):
        lts_ensemble_destroy(self.h)
        self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Model:
    """Mesh + regions + state, with the handles released on close()."""

    def __init__(self, mesh: dict, fine_mask, M: int, h0, u0, dt: float, g: float = 9.81,
                 precision: int = LTS_FP32, mode: int = LTS_MODE_LTS3, compensated: bool = True,
                 use_graph: bool = True, block_size: int = 0, profile: int = 0,
                 interface_layers: int = 1, stream: int | None = None, pdl: bool = True,
                 kernel_path: int = 0, tile_cells: int = 0, l2_hints: bool = True,
                 coarse_schedule: int = 0, ordering: int = LTS_ORDER_HILBERT,
                 autotune: int = 0, tune_ordering: bool = False, order: int = 3, layers: int = 1,
                 ring_occupancy: int = 0, elems_per_thread: int = 0):
        """autotune > 0: time that many coarse steps per candidate configuration
        (lts_autotune) and build the state with the fastest; the choice is in
        self.tuned.  layers > 1: h0, u0 (and read/write) are [layers][nCells],
        [layers][nEdges] arrays."""
        self.layers = max(1, int(layers))
        self.nC = int(mesh["nCells"])
        self.nE = int(mesh["nEdges"])
        self.nV = int(mesh["nVertices"])
        self.mesh_h = self.reg_h = self.state_h = None
        self.tuned = None
        self._pending = []
        self.mesh_h = lts_mesh_create(mesh)
        if np.ndim(M) > 0:   # several fine regions: fine_mask holds region ids 1..len(M)
            self.reg_h = lts_regions_set_multi(self.mesh_h, fine_mask, list(M), order, interface_layers)
        else:
            self.reg_h = lts_regions_set(self.mesh_h, fine_mask, order, M, interface_layers)
        if tile_cells:
            lts_regions_tiling(self.reg_h, tile_cells)
        if ordering != LTS_ORDER_HILBERT:
            lts_regions_ordering(self.reg_h, ordering)
        p = make_params(g, dt, precision, mode, compensated, use_graph, block_size, profile, stream,
                        pdl, kernel_path, l2_hints, coarse_schedule, self.layers, ring_occupancy,
                        elems_per_thread)
        h0 = np.ascontiguousarray(h0, np.float64).reshape(-1)
        u0 = np.ascontiguousarray(u0, np.float64).reshape(-1)
        if h0.size != self.layers * self.nC or u0.size != self.layers * self.nE:
            raise ValueError("h0/u0 must hold layers x nCells / layers x nEdges values")
        if autotune:
            p, rep = lts_autotune(self.mesh_h, self.reg_h, h0, u0, p, autotune, tune_ordering)
            self.tuned = dict(params_dict(p), **rep)
        self.state_h = lts_state_create_p(self.mesh_h, self.reg_h, h0, u0, p)

    def step(self, n: int):
        lts_step(self.state_h, n)

    def read(self, h_out=None, u_out=None):
        L = self.layers
        h, u, d = lts_read(self.state_h, L * self.nC, L * self.nE, h_out, u_out)
        self._pending = []          # lts_read also completes earlier asynchronous reads
        if L > 1 and h_out is None:
            h, u = h.reshape(L, self.nC), u.reshape(L, self.nE)
        return h, u, d

    def read_async(self, h_out=None, u_out=None, diag: bool = False):
        """Enqueues the copy of the state as it stands after the work enqueued
        so far into h_out / u_out (float64, layers x nCells / layers x nEdges
        values; pinned memory overlaps the copy with the following steps).
        The arrays (and the returned diagnostics record) are valid after
        sync()."""
        L = self.layers
        if h_out is not None and h_out.size != L * self.nC:
            raise ValueError("h_out must hold layers x nCells values")
        if u_out is not None and u_out.size != L * self.nE:
            raise ValueError("u_out must hold layers x nEdges values")
        d = lts_read_async(self.state_h, h_out, u_out, diag)
        if d is not None:
            self._pending.append(d)
        return d

    def sync(self):
        """Waits for the state's work and copies; returns the diagnostics of
        the asynchronous reads since the last sync, in order."""
        pending, self._pending = self._pending, []
        lts_sync(self.state_h)
        return [{"mass": d.mass, "energy": d.energy, "time": d.time, "steps": d.steps} for d in pending]

    def write(self, h, u, time=0.0, steps=0):
        lts_write(self.state_h, np.ascontiguousarray(h, np.float64).reshape(-1),
                  np.ascontiguousarray(u, np.float64).reshape(-1), time, steps)

    def labels(self):
        return lts_regions_labels(self.reg_h, self.nC, self.nE)

    def counts(self):
        return lts_regions_counts(self.reg_h)

    def stats(self):
        return lts_step_stats(self.state_h)

    def close(self):
        lts_state_destroy(self.state_h)
        lts_regions_destroy(self.reg_h)
        lts_mesh_destroy(self.mesh_h)
        self.state_h = self.reg_h = self.mesh_h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
