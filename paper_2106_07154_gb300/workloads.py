"""Seeded synthetic workloads: meshes, initial states, fine-cell masks, time steps.

This module is an input generator shared by the tests, the benchmark and
the oracle checks.  It holds none of the method's arithmetic (no operators,
no time stepping); it only builds inputs with the shapes of the paper's
experiments (Section 3: a zonal flow over an isolated mountain on a sphere
with a refined cap around the mountain; Section 3.2's cone mountain is
replaced by a Gaussian of height 2000 m and radius 20 degrees).

Meshes come from the library's seeded builders and are cached on disk
(``$LTS_MESH_CACHE`` or ``<repo>/.mesh_cache``) keyed by their parameters.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from pathlib import Path

import numpy as np

from . import lts

G = 9.81
OMEGA = 7.292e-5
R_EARTH = 6371.0e3

CACHE = Path(os.environ.get("LTS_MESH_CACHE", Path(__file__).resolve().parent.parent / ".mesh_cache"))


def _cache_path(name: str) -> Path:
    return CACHE / f"{name}.npz"


def _save(mesh: dict, path: Path):
    path.parent.mkdir(parents=True, exist_ok=True)
    arrays = {k: v for k, v in mesh.items() if isinstance(v, np.ndarray)}
    scalars = {k: np.asarray(v) for k, v in mesh.items() if not isinstance(v, np.ndarray) and v is not None}
    tmp = path.with_suffix(".tmp.npz")
    np.savez(tmp, **arrays, **scalars)
    os.replace(tmp, path)


def _load(path: Path) -> dict:
    with np.load(path) as z:
        out = {}
        for k in z.files:
            v = z[k]
            out[k] = v.item() if v.ndim == 0 else v
    for k in lts.SCALARS:
        if k in out and isinstance(out[k], float) and k.startswith("n"):
            out[k] = int(out[k])
    out.setdefault("bottom", None)
    return out


def hex_mesh(nx: int, ny: int, dc: float, f0: float) -> dict:
    return lts.lts_build_hex_periodic(nx, ny, dc, f0)


def scvt_mesh(n: int, seed: int, caps, lloyd_iters: int, radius: float = R_EARTH,
              cache: bool = True) -> dict:
    key = f"scvt_n{n}_s{seed}_it{lloyd_iters}_r{int(radius)}_" + "_".join(
        "-".join(f"{x:.6g}" for x in c) for c in caps)
    path = _cache_path(key)
    if cache and path.exists():
        try:
            return _load(path)
        except Exception:
            pass
    mesh = lts.lts_build_scvt(n, seed, caps, lloyd_iters, radius)
    if cache:
        try:
            _save(mesh, path)
        except OSError:
            pass
    return mesh


# ----------------------------------------------------------------------------
# workloads


@dataclass
class Workload:
    name: str
    mesh: dict
    h0: np.ndarray
    u0: np.ndarray
    fine_mask: np.ndarray
    M: int
    dt: float            # coarse step (LTS3)
    nsteps: int
    g: float = G
    info: dict = field(default_factory=dict)
    order: int = 3             # 3 = LTS3, 2 = LTS2
    interface_layers: int = 1  # interface thickness in cells (Eqs. 3-5 with thicker I1, I2)

    @property
    def nCells(self) -> int:
        return int(self.mesh["nCells"])


def _cfl_dt(mesh, h, u, coarse_cells, cfl, g=G):
    """CFL * min spacing of the given cells / (max|u| + sqrt(g max h))."""
    dc = np.asarray(mesh["dcEdge"])
    eoc = np.asarray(mesh["edgesOnCell"])
    noc = np.asarray(mesh["nEdgesOnCell"])
    mask = np.arange(eoc.shape[1])[None, :] < noc[:, None]
    mind = np.where(mask, dc[np.where(mask, eoc, 0)], np.inf).min(axis=1)
    c = float(np.abs(u).max() + math.sqrt(g * float(h.max())))
    cells = np.nonzero(coarse_cells)[0]
    return cfl * float(mind[cells].min()) / c, mind, c


def hex_bump(nx: int = 32, ny: int = 32, dc: float = 10e3, f0: float = 1e-4, M: int = 2,
             seed: int = 1, radius: float = 60e3, sigma: float = 40e3, nsteps: int = 100,
             cfl: float = 0.5, amplitude: float = 1.0) -> Workload:
    """Doubly periodic hexagons, flat bottom, h = 1000 m + a Gaussian bump of
    `amplitude` m (1 m by default) at a seeded centre, u = 0, fine region =
    cells within `radius` of the bump."""
    mesh = hex_mesh(nx, ny, dc, f0)
    rng = np.random.default_rng(seed)
    Lx, Ly = mesh["period_x"], mesh["period_y"]
    cx, cy = rng.uniform(0, Lx), rng.uniform(0, Ly)
    dx = mesh["xCell"] - cx
    dy = mesh["yCell"] - cy
    dx -= Lx * np.round(dx / Lx)
    dy -= Ly * np.round(dy / Ly)
    r2 = dx * dx + dy * dy
    h0 = 1000.0 + amplitude * np.exp(-r2 / (2.0 * sigma * sigma))
    u0 = np.zeros(mesh["nEdges"])
    mesh["bottom"] = np.zeros(mesh["nCells"])
    fine = (r2 <= radius * radius).astype(np.int8)
    dt, _, _ = _cfl_dt(mesh, h0, u0, np.ones(mesh["nCells"], bool), cfl)
    return Workload("hex_bump", mesh, h0, u0, fine, M, dt, nsteps,
                    info={"center": (cx, cy), "nx": nx, "ny": ny, "dc": dc})


def _lonlat(x, y, z):
    r = np.sqrt(x * x + y * y + z * z)
    return np.arctan2(y, x), np.arcsin(np.clip(z / r, -1, 1))


def _great_circle(lon, lat, lon0, lat0):
    c = np.sin(lat) * math.sin(lat0) + np.cos(lat) * math.cos(lat0) * np.cos(lon - lon0)
    return np.arccos(np.clip(c, -1.0, 1.0))


def zonal_state(mesh: dict, u0: float = 20.0, mean_depth: float = 5960.0,
                mountain_height: float = 2000.0, mountain_radius: float = math.radians(20.0),
                centre=(1.5 * math.pi, math.pi / 6), g: float = G, omega: float = OMEGA):
    """Balanced zonal flow u = u0 cos(lat) over a Gaussian mountain.

    The free surface follows the steady balance of the continuous equations
    (Appendix A) for u = u0 cos(lat):  g eta = g H0 - (R Omega u0 + u0^2/2) sin^2(lat);
    H0 is set so that the area mean of eta is `mean_depth`; h = eta - b."""
    R = float(mesh["radius"])
    lonc, latc = _lonlat(mesh["xCell"], mesh["yCell"], mesh["zCell"])
    coef = (R * omega * u0 + 0.5 * u0 * u0) / g
    H0 = mean_depth + coef / 3.0   # area mean of sin^2(lat) over the sphere is 1/3
    eta = H0 - coef * np.sin(latc) ** 2
    d = _great_circle(lonc, latc, *centre)
    b = mountain_height * np.exp(-(d / mountain_radius) ** 2)
    h = eta - b
    # normal velocity at x_e along n_e (from cellsOnEdge[:,0] to cellsOnEdge[:,1])
    xe = np.stack([mesh["xEdge"], mesh["yEdge"], mesh["zEdge"]], 1)
    xe /= np.linalg.norm(xe, axis=1, keepdims=True)
    xc = np.stack([mesh["xCell"], mesh["yCell"], mesh["zCell"]], 1)
    coe = mesh["cellsOnEdge"]
    t = xc[coe[:, 1]] - xc[coe[:, 0]]
    t -= np.sum(t * xe, axis=1, keepdims=True) * xe
    n = t / np.linalg.norm(t, axis=1, keepdims=True)
    lone, late = _lonlat(xe[:, 0], xe[:, 1], xe[:, 2])
    east = np.stack([-np.sin(lone), np.cos(lone), np.zeros_like(lone)], 1)
    u = u0 * np.cos(late) * np.sum(east * n, axis=1)
    return h, u, b


def sphere_cap(n: int, ratio: float, M: int, seed: int = 1, lloyd_iters: int = 200,
               nsteps: int = 100, cap_radius: float = math.radians(15.0),
               cap_width: float = math.radians(5.0), fine_threshold: float = 0.9,
               cfl: float = 0.5, u0: float = 20.0, mountain: bool = True,
               name: str = "sphere_cap", cache: bool = True,
               centre=(1.5 * math.pi, math.pi / 6), bump=None) -> Workload:
    """Spherical SCVT with a refined cap centred on the mountain (Section 3:
    centre (3 pi/2, pi/6)); fine region = cells whose target spacing is below
    `fine_threshold` times the coarse spacing; dt = CFL limit of the coarse,
    interface and fine-boundary cells.  `bump` = (amplitude m, radius rad)
    adds a Gaussian thickness perturbation at the cap centre."""
    cap = (centre[0], centre[1], cap_radius, cap_width, ratio)
    mesh = scvt_mesh(n, seed, [cap], lloyd_iters, cache=cache)
    h0, uu, b = zonal_state(mesh, u0=u0, mountain_height=2000.0 if mountain else 0.0,
                            centre=centre)
    mesh["bottom"] = b
    lonc, latc = _lonlat(mesh["xCell"], mesh["yCell"], mesh["zCell"])
    d = _great_circle(lonc, latc, *centre)
    if bump is not None:
        h0 = h0 + bump[0] * np.exp(-(d / bump[1]) ** 2)
    s = 1.0 / ratio + (1.0 - 1.0 / ratio) * 0.5 * (1.0 + np.tanh((d - cap_radius) / cap_width))
    fine = (s < fine_threshold).astype(np.int8)
    dt, mind, c = _cfl_dt(mesh, h0, uu, fine == 0, cfl)
    fine_cfl = dt / M * c / float(mind[fine == 1].min()) if fine.any() else 0.0
    return Workload(name, mesh, h0, uu, fine, M, dt, nsteps,
                    info={"ratio": ratio, "seed": seed, "lloyd_iters": lloyd_iters,
                          "fine_cfl": fine_cfl, "coarse_cfl": cfl, "n_fine": int(fine.sum())})


def ensemble(n_members: int = 64, seed: int = 7, min_cells: int = 2562, max_cells: int = 163842,
             lloyd_iters: int = 200, cache: bool = True):
    """Uneven ensemble of spherical SCVT members: sizes log-uniform in
    [min_cells, max_cells], resolution ratio 2, 4 or 8 in a cap at a seeded
    position with M equal to the ratio, a balanced zonal flow with u0 uniform
    in [10, 40] m/s over a flat bottom, and a Gaussian thickness perturbation
    of amplitude uniform in [1, 10] m and radius 10 degrees at the cap centre."""
    return [sphere_cap(**kw) for kw in ensemble_recipes(n_members, seed, min_cells, max_cells,
                                                        lloyd_iters, cache)]


def ensemble_recipes(n_members: int = 64, seed: int = 7, min_cells: int = 2562,
                     max_cells: int = 163842, lloyd_iters: int = 200, cache: bool = True):
    """The sphere_cap arguments of every member of `ensemble` (no mesh built)."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_members):
        n = int(round(math.exp(rng.uniform(math.log(min_cells), math.log(max_cells)))))
        ratio = float(rng.choice([2.0, 4.0, 8.0]))
        centre = (float(rng.uniform(0.0, 2.0 * math.pi)), float(math.asin(rng.uniform(-0.9, 0.9))))
        u0 = float(rng.uniform(10.0, 40.0))
        amp = float(rng.uniform(1.0, 10.0))
        out.append(dict(n=n, ratio=ratio, M=int(ratio), seed=seed * 1000 + k,
                        lloyd_iters=lloyd_iters, u0=u0, mountain=False, centre=centre,
                        bump=(amp, math.radians(10.0)), name=f"ens{k}", cache=cache))
    return out


def ridges(mesh: dict, n_ridges: int = 32, seed: int = 5, h_max: float = 3000.0):
    """Sum of anisotropic Gaussian ridges on the sphere: seeded centres
    (uniform on the sphere), orientations, along-ridge lengths 2..15 degrees
    (across-ridge width a quarter of that) and heights up to h_max."""
    rng = np.random.default_rng(seed)
    X = np.stack([mesh["xCell"], mesh["yCell"], mesh["zCell"]], 1)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    b = np.zeros(len(X))
    for _ in range(n_ridges):
        c = rng.standard_normal(3)
        c /= np.linalg.norm(c)
        # a tangent frame at c, turned by a seeded orientation
        a = np.cross(c, [0.0, 0.0, 1.0] if abs(c[2]) < 0.9 else [1.0, 0.0, 0.0])
        a /= np.linalg.norm(a)
        t = np.cross(c, a)
        phi = rng.uniform(0, math.pi)
        e1 = math.cos(phi) * a + math.sin(phi) * t
        e2 = np.cross(c, e1)
        length = math.radians(rng.uniform(2.0, 15.0))
        width = 0.25 * length
        height = rng.uniform(0.2, 1.0) * h_max
        s1 = X @ e1
        s2 = X @ e2
        near = X @ c > 0.0                      # the hemisphere around the centre
        b += np.where(near, height * np.exp(-(s1 / length) ** 2 - (s2 / width) ** 2), 0.0)
    return b


def spectral_noise(mesh: dict, rms: float = 5.0, lmax: int = 64, slope: float = -3.0, seed: int = 6,
                   modes_per_degree: int = 8):
    """A random field on the sphere with power per degree l proportional to
    l**slope for l = 1..lmax, scaled to `rms` (area-weighted) with zero
    mean: for each l, `modes_per_degree` plane waves of wavenumber l/R in
    seeded directions, restricted to the sphere (a tractable stand-in for a
    spherical-harmonic synthesis)."""
    rng = np.random.default_rng(seed)
    X = np.stack([mesh["xCell"], mesh["yCell"], mesh["zCell"]], 1)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    f = np.zeros(len(X))
    for l in range(1, lmax + 1):
        amp = math.sqrt(l ** slope / modes_per_degree)
        for _ in range(modes_per_degree):
            k = rng.standard_normal(3)
            k *= (l + 0.5) / np.linalg.norm(k)
            f += amp * np.cos(X @ k + rng.uniform(0, 2 * math.pi))
    A = np.asarray(mesh["areaCell"])
    f -= np.sum(A * f) / np.sum(A)
    f *= rms / math.sqrt(np.sum(A * f * f) / np.sum(A))
    return f


def two_caps(n: int = 2621442, seed: int = 5, lloyd_iters: int = 200, cfl: float = 0.5,
             u0: float = 20.0, cache: bool = True, name: str = "scvt_2621442_2caps") -> Workload:
    """The large single instance: a spherical SCVT with two separate refined
    caps (8:1 with M = 8 at the Section-3 mountain position, 4:1 with M = 4
    on the other side), 32 seeded ridges up to 3000 m, a balanced zonal flow
    and 5 m of h noise of spectral slope -3.  fine_mask holds the region id
    (1 or 2) of each fine cell; M is the pair (8, 4)."""
    cap_r, cap_w = math.radians(15.0), math.radians(5.0)
    caps = [(1.5 * math.pi, math.pi / 6, cap_r, cap_w, 8.0), (0.5 * math.pi, -math.pi / 4, cap_r, cap_w, 4.0)]
    mesh = scvt_mesh(n, seed, caps, lloyd_iters, cache=cache)
    h0, uu, _ = zonal_state(mesh, u0=u0, mountain_height=0.0)
    b = ridges(mesh, seed=seed)
    mesh["bottom"] = b
    h0 = h0 - b + spectral_noise(mesh, seed=seed + 1)
    lon, lat = _lonlat(mesh["xCell"], mesh["yCell"], mesh["zCell"])
    rid = np.zeros(mesh["nCells"], np.int8)
    for r, (lo, la, rad, wid, ratio) in enumerate(caps, start=1):
        d = _great_circle(lon, lat, lo, la)
        s = 1.0 / ratio + (1.0 - 1.0 / ratio) * 0.5 * (1.0 + np.tanh((d - rad) / wid))
        rid[s < 0.9] = r
    dt, _, _ = _cfl_dt(mesh, h0, uu, rid == 0, cfl)
    return Workload(name, mesh, h0, uu, rid, (8, 4), dt, 2000,
                    info={"ratios": (8.0, 4.0), "n_fine": int((rid > 0).sum()), "seed": seed})


def workload(name: str, **kw) -> Workload:
    """The named synthetic workloads, seeded stand-ins for the meshes of the
    paper's Section 3 (which are not available):
      hex_1024            32x32 doubly periodic hexagons, dc = 10 km, f-plane, flat
                          bottom, 1 m Gaussian bump (sigma 40 km) at a seeded centre,
                          fine region a 60 km circle, M = 2
      scvt_40962          spherical SCVT (200 Lloyd iterations), 4:1 cap of radius 15
                          degrees (tanh width 5) at (3 pi/2, pi/6), balanced zonal flow
                          u0 = 20 m/s, 2000 m Gaussian mountain, M = 4
      scvt_655362         the same recipe at 655,362 cells with an 8:1 cap, M = 8
      scvt_2562           small test sphere (4:1 cap, 60 Lloyd iterations)
      scvt_2621442_2caps  two caps (8:1 with M = 8, 4:1 with M = 4), 32 seeded
                          ridges, 5 m of spectral-slope -3 noise
      ensemble64          64 uneven spheres (see ensemble)"""
    if name == "hex_1024":          # 32x32 periodic hexagons, M = 2, 100 coarse steps
        return hex_bump(**kw)
    if name == "scvt_40962":        # 4:1 cap, M = 4, 500 coarse steps
        args = dict(n=40962, ratio=4.0, M=4, nsteps=500, name=name)
        args.update(kw)
        return sphere_cap(**args)
    if name == "scvt_655362":       # 8:1 cap, M = 8
        args = dict(n=655362, ratio=8.0, M=8, nsteps=100, name=name)
        args.update(kw)
        return sphere_cap(**args)
    if name == "scvt_2562":         # small test sphere
        args = dict(n=2562, ratio=4.0, M=4, nsteps=20, lloyd_iters=60, name=name)
        args.update(kw)
        return sphere_cap(**args)
    if name == "scvt_2621442_2caps":   # two caps (8:1, M = 8 and 4:1, M = 4), ridges, noise
        return two_caps(**kw)
    if name == "scvt_10242":        # medium test sphere
        args = dict(n=10242, ratio=4.0, M=4, nsteps=20, lloyd_iters=100, name=name)
        args.update(kw)
        return sphere_cap(**args)
    raise KeyError(name)
