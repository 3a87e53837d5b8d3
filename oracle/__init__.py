"""Python front end of the FP64 CPU oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline / reference arm of ``bench.py``; the product package
never imports it.  Each function names the passage of arXiv:2106.07154 that
it follows; the arithmetic itself lives in oracle.c.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "oracle.c"
LIB = HERE / "liboracle.so"

_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i8p = np.ctypeslib.ndpointer(dtype=np.int8, flags="C_CONTIGUOUS")


def build(force: bool = False) -> Path:
    """gcc -O2 with FMA contraction off, so x86 and Arm give the same bits."""
    if force or not LIB.exists() or LIB.stat().st_mtime < max(
            SRC.stat().st_mtime, (HERE / "oracle.h").stat().st_mtime):
        tmp = LIB.with_suffix(".so.tmp")
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
               "-fno-fast-math", str(SRC), "-o", str(tmp), "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(str(LIB))
        L.or_mesh_new.restype = C.c_void_p
        L.or_mesh_new.argtypes = [C.c_int] * 4 + [_i32p] * 6 + [_f64p] * 6 + [C.c_void_p]
        L.or_mesh_free.argtypes = [C.c_void_p]
        L.or_weights.argtypes = [C.c_void_p, _i32p, _i32p, _f64p]
        for name in ("or_divergence", "or_gradient", "or_vorticity", "or_kinetic", "or_tangential"):
            getattr(L, name).argtypes = [C.c_void_p, _f64p, _f64p]
        L.or_thickness_flux.argtypes = [C.c_void_p, _f64p, _f64p, _f64p]
        L.or_pv_vertex.argtypes = [C.c_void_p, _f64p, _f64p, _f64p]
        L.or_pv_flux.argtypes = [C.c_void_p, _f64p, _f64p, _f64p]
        L.or_rhs_swe.argtypes = [C.c_void_p, C.c_double, _f64p, _f64p, _f64p, _f64p]
        L.or_regions.argtypes = [C.c_void_p, _i8p, _i8p, _i8p]
        L.or_regions_layers.argtypes = [C.c_void_p, _i8p, C.c_int, _i8p, _i8p]
        L.or_lts3_predict_coeffs.argtypes = [C.c_int, C.c_int, C.c_int, _f64p]
        L.or_ssprk3.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_int, _f64p, _f64p]
        L.or_rk4.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_int, _f64p, _f64p]
        L.or_lts3.argtypes = [C.c_void_p, C.c_void_p, _i8p, _i8p, C.c_int, C.c_double, C.c_int,
                              C.c_int, _f64p, _f64p]
        L.or_lts2.argtypes = [C.c_void_p, C.c_void_p, _i8p, _i8p, C.c_int, C.c_double, C.c_int,
                              C.c_int, _f64p, _f64p]
        L.or_ssprk2.argtypes = [C.c_void_p, C.c_void_p, C.c_double, C.c_int, _f64p, _f64p]
        L.or_region_ids.argtypes = [C.c_void_p, _i8p, _i8p, _i8p, _i8p, _i8p]
        L.or_lts3_multi.argtypes = [C.c_void_p, C.c_void_p, _i8p, _i8p, _i8p, _i8p, C.c_int,
                                    np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS"),
                                    C.c_double, C.c_int, C.c_int, _f64p, _f64p]
        L.or_lts2_predict_coeffs.argtypes = [C.c_int, C.c_int, C.c_int, _f64p]
        L.or_mass.restype = C.c_double
        L.or_mass.argtypes = [C.c_void_p, _f64p]
        L.or_energy.restype = C.c_double
        L.or_energy.argtypes = [C.c_void_p, C.c_double, _f64p, _f64p]
        L.or_num_threads.restype = C.c_int
        _lib = L
    return _lib


class _System(C.Structure):
    _fields_ = [("kind", C.c_int), ("g", C.c_double), ("lam_c", C.c_void_p), ("lam_e", C.c_void_p)]


def num_threads() -> int:
    return int(lib().or_num_threads())


class Oracle:
    """FP64 oracle bound to one mesh (a dict of MPAS arrays, see workloads)."""

    def __init__(self, mesh: dict):
        L = lib()
        self.nC = int(mesh["nCells"])
        self.nE = int(mesh["nEdges"])
        self.nV = int(mesh["nVertices"])
        self.maxE = int(mesh["maxEdges"])
        i32 = lambda k: np.ascontiguousarray(mesh[k], dtype=np.int32)
        f64 = lambda k: np.ascontiguousarray(mesh[k], dtype=np.float64)
        self._keep = [i32("nEdgesOnCell"), i32("edgesOnCell"), i32("cellsOnEdge"),
                      i32("verticesOnEdge"), i32("edgesOnVertex"), i32("cellsOnVertex"),
                      f64("areaCell"), f64("areaTriangle"), f64("kiteAreasOnVertex"),
                      f64("dcEdge"), f64("dvEdge"), f64("fVertex")]
        b = mesh.get("bottom")
        self._b = None if b is None else np.ascontiguousarray(b, dtype=np.float64)
        self.areaCell = self._keep[6]
        self._h = L.or_mesh_new(self.nC, self.nE, self.nV, self.maxE, *self._keep,
                                None if self._b is None else self._b.ctypes.data)
        if not self._h:
            raise ValueError("oracle rejected the mesh")

    def __del__(self):
        if getattr(self, "_h", None):
            lib().or_mesh_free(self._h)
            self._h = None

    # ---------------------------------------------------------- systems
    def _sys(self, g=9.81, lam_c=None, lam_e=None):
        if lam_c is None:
            s = _System(0, g, None, None)
            s._arrays = ()
        else:
            lc = np.ascontiguousarray(lam_c, dtype=np.float64)
            le = np.ascontiguousarray(lam_e, dtype=np.float64)
            s = _System(1, g, lc.ctypes.data, le.ctypes.data)
            s._arrays = (lc, le)
        return s

    # ---------------------------------------------------------- operators (Appendix B)
    def weights(self):
        """EE(e) and w_{e,e'} of Eq. (weights)."""
        w = 2 * self.maxE
        n = np.zeros(self.nE, np.int32)
        eoe = np.zeros(self.nE * w, np.int32)
        woe = np.zeros(self.nE * w, np.float64)
        lib().or_weights(self._h, n, eoe, woe)
        return n, eoe.reshape(self.nE, w), woe.reshape(self.nE, w)

    def _op(self, name, x, nout):
        out = np.zeros(nout, np.float64)
        getattr(lib(), name)(self._h, np.ascontiguousarray(x, np.float64), out)
        return out

    def divergence(self, F):
        return self._op("or_divergence", F, self.nC)

    def gradient(self, phi):
        return self._op("or_gradient", phi, self.nE)

    def vorticity(self, u):
        return self._op("or_vorticity", u, self.nV)

    def kinetic(self, u):
        return self._op("or_kinetic", u, self.nC)

    def tangential(self, F):
        return self._op("or_tangential", F, self.nE)

    def thickness_flux(self, h, u):
        out = np.zeros(self.nE)
        lib().or_thickness_flux(self._h, np.ascontiguousarray(h, np.float64),
                                np.ascontiguousarray(u, np.float64), out)
        return out

    def pv_vertex(self, h, u):
        out = np.zeros(self.nV)
        lib().or_pv_vertex(self._h, np.ascontiguousarray(h, np.float64),
                           np.ascontiguousarray(u, np.float64), out)
        return out

    def pv_flux(self, F, qe):
        out = np.zeros(self.nE)
        lib().or_pv_flux(self._h, np.ascontiguousarray(F, np.float64),
                         np.ascontiguousarray(qe, np.float64), out)
        return out

    def rhs(self, h, u, g=9.81):
        """Eq. (1): (H_i, U_e) on the whole mesh."""
        H = np.zeros(self.nC)
        U = np.zeros(self.nE)
        lib().or_rhs_swe(self._h, g, np.ascontiguousarray(h, np.float64),
                         np.ascontiguousarray(u, np.float64), H, U)
        return H, U

    def regions(self, fine_mask, layers=1):
        """Labels of Eqs. (3)-(5): cells 0 F\\Fbar,1 F2,2 F1,3 I1,4 I2,5 C; edges 0,1,3,4,5.
        layers > 1: interfaces that many cells thick."""
        cl = np.zeros(self.nC, np.int8)
        el = np.zeros(self.nE, np.int8)
        fm = np.ascontiguousarray(fine_mask, np.int8)
        if layers == 1:
            lib().or_regions(self._h, fm, cl, el)
        elif lib().or_regions_layers(self._h, fm, int(layers), cl, el) != 0:
            raise ValueError("layers must be >= 1")
        return cl, el

    # ---------------------------------------------------------- integrators (Section 2)
    def ssprk3(self, h, u, dt, nsteps, g=9.81, lam_c=None, lam_e=None):
        """Algorithm 2.1 (SSPRK3)."""
        h = np.array(h, np.float64)
        u = np.array(u, np.float64)
        s = self._sys(g, lam_c, lam_e)
        lib().or_ssprk3(self._h, C.addressof(s), dt, nsteps, h, u)
        return h, u

    def ssprk2(self, h, u, dt, nsteps, g=9.81, lam_c=None, lam_e=None):
        """Algorithm 2.1 (SSPRK2)."""
        h = np.array(h, np.float64)
        u = np.array(u, np.float64)
        s = self._sys(g, lam_c, lam_e)
        lib().or_ssprk2(self._h, C.addressof(s), dt, nsteps, h, u)
        return h, u

    def lts2(self, h, u, cell_label, edge_label, M, dt, nsteps, g=9.81, step5_form=0,
             lam_c=None, lam_e=None):
        """Algorithm 2.2, LTS2 branches."""
        h = np.array(h, np.float64)
        u = np.array(u, np.float64)
        s = self._sys(g, lam_c, lam_e)
        rc = lib().or_lts2(self._h, C.addressof(s), np.ascontiguousarray(cell_label, np.int8),
                           np.ascontiguousarray(edge_label, np.int8), int(M), float(dt),
                           int(nsteps), int(step5_form), h, u)
        if rc != 0:
            raise ValueError("or_lts2 failed")
        return h, u

    def region_ids(self, region_of_fine, cell_label, edge_label):
        """Region (1..R) of every fine/interface cell and edge, 0 on the coarse sets."""
        creg = np.zeros(self.nC, np.int8)
        ereg = np.zeros(self.nE, np.int8)
        rc = lib().or_region_ids(self._h, np.ascontiguousarray(region_of_fine, np.int8),
                                 np.ascontiguousarray(cell_label, np.int8),
                                 np.ascontiguousarray(edge_label, np.int8), creg, ereg)
        if rc != 0:
            raise ValueError("the regions' fine and interface sets touch")
        return creg, ereg

    def lts3_multi(self, h, u, region_of_fine, Ms, dt, nsteps, g=9.81, step5_form=0,
                   lam_c=None, lam_e=None):
        """Several disjoint fine regions with their own M sharing the coarse step."""
        rof = np.ascontiguousarray(region_of_fine, np.int8)
        cl, el = self.regions((rof > 0).astype(np.int8))
        creg, ereg = self.region_ids(rof, cl, el)
        h = np.array(h, np.float64)
        u = np.array(u, np.float64)
        s = self._sys(g, lam_c, lam_e)
        Ms = np.ascontiguousarray(Ms, np.int32)
        rc = lib().or_lts3_multi(self._h, C.addressof(s), cl, el, creg, ereg, len(Ms), Ms,
                                 float(dt), int(nsteps), int(step5_form), h, u)
        if rc != 0:
            raise ValueError("or_lts3_multi failed")
        return h, u

    def rk4(self, h, u, dt, nsteps, g=9.81, lam_c=None, lam_e=None):
        """Classical RK4, the reference-solution generator of Section 3.2."""
        h = np.array(h, np.float64)
        u = np.array(u, np.float64)
        s = self._sys(g, lam_c, lam_e)
        lib().or_rk4(self._h, C.addressof(s), dt, nsteps, h, u)
        return h, u

    def lts3(self, h, u, cell_label, edge_label, M, dt, nsteps, g=9.81, step5_form=0,
             lam_c=None, lam_e=None):
        """Algorithm 2.2 (LTS3); step5_form 0 = replay reading, 1 = Step 5 as printed."""
        h = np.array(h, np.float64)
        u = np.array(u, np.float64)
        s = self._sys(g, lam_c, lam_e)
        rc = lib().or_lts3(self._h, C.addressof(s), np.ascontiguousarray(cell_label, np.int8),
                           np.ascontiguousarray(edge_label, np.int8), int(M), float(dt),
                           int(nsteps), int(step5_form), h, u)
        if rc != 0:
            raise ValueError("or_lts3 failed")
        return h, u

    def mass(self, h):
        return float(lib().or_mass(self._h, np.ascontiguousarray(h, np.float64)))

    def energy(self, h, u, g=9.81):
        return float(lib().or_energy(self._h, g, np.ascontiguousarray(h, np.float64),
                                     np.ascontiguousarray(u, np.float64)))


def predict_coeffs(k: int, M: int, stage: int, order: int = 3) -> np.ndarray:
    """Steps 3.1.1/3.2.1/3.3.1: (c_old, c_1st, c_2nd) of the I1 prediction."""
    c = np.zeros(3)
    if order == 2:
        lib().or_lts2_predict_coeffs(k, M, stage, c)
    else:
        lib().or_lts3_predict_coeffs(k, M, stage, c)
    return c
