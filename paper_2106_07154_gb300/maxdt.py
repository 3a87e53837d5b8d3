"""Largest stable time steps of LTS on a given mesh and state: the protocol
of the paper's speed-up runs (Section 3.3).  First the largest fine step
with M = 1 (LTS reduces to the underlying SSP-RK scheme), then, for M =
2, 3, ..., the largest coarse step M * dt_fine that stays stable; the
largest such M is the payoff of LTS for that mesh and interface width.

A run counts as stable when it reaches the simulated time T without a
non-finite value or a thickness <= 0 (the library reports those as
LTS_ENONFINITE) and with the total energy within `energy_tol` (relative)
of its initial value; an unstable SSP-RK run grows exponentially, so
either test ends it.  Host logic over the C ABI only.
"""
from __future__ import annotations

import argparse
import json
import math
import time

from . import lts


def _stable(make_model, dt: float, T: float, energy_tol: float) -> bool:
    n = max(1, int(math.ceil(T / dt)))
    try:
        with make_model(dt) as m:
            _, _, d0 = m.read()
            done = 0
            while done < n:        # in chunks, so a blow-up ends the run early
                k = min(50, n - done)
                m.step(k)
                done += k
                _, _, d = m.read()
                if not math.isfinite(d["energy"]):
                    return False
                if abs(d["energy"] - d0["energy"]) > energy_tol * abs(d0["energy"]):
                    return False
        return True
    except lts.LtsError as e:
        if e.code == lts.LTS_ENONFINITE:
            return False
        raise


def largest_stable_dt(make_model, dt_lo: float, dt_hi: float, T: float, rel_tol: float = 0.02,
                      energy_tol: float = 1e-2) -> float:
    """Bisection for the largest dt in [dt_lo, dt_hi] whose run over T is
    stable; make_model(dt) returns an lts.Model.  dt_lo must be stable."""
    if not _stable(make_model, dt_lo, T, energy_tol):
        raise ValueError("dt_lo is not stable")
    if _stable(make_model, dt_hi, T, energy_tol):
        return dt_hi
    lo, hi = dt_lo, dt_hi
    while hi - lo > rel_tol * lo:
        mid = 0.5 * (lo + hi)
        if _stable(make_model, mid, T, energy_tol):
            lo = mid
        else:
            hi = mid
    return lo


def max_dt_protocol(mesh: dict, fine_mask, h0, u0, g: float, dt_guess: float, T: float,
                    M_max: int = 32, precision: int = lts.LTS_FP32, layers: int = 1,
                    order: int = 3, rel_tol: float = 0.02, energy_tol: float = 1e-2):
    """The speed-up protocol: (1) the largest fine step dt_f with M = 1;
    (2) for M = 2..M_max, whether the coarse step M * dt_f is stable (the
    fine step stays dt_f).  Returns {"dt_fine", "M_max_stable", "dt_coarse",
    "tried": [(M, stable)]}."""
    def maker(M):
        return lambda dt: lts.Model(mesh, fine_mask, M, h0, u0, dt, g, precision=precision,
                                    interface_layers=layers, order=order)

    dt_f = largest_stable_dt(maker(1), dt_guess / 4.0, dt_guess * 4.0, T, rel_tol, energy_tol)
    best, tried = 1, []
    for M in range(2, M_max + 1):
        ok = _stable(maker(M), M * dt_f, T, energy_tol)
        tried.append((M, ok))
        if not ok:
            break
        best = M
    return {"dt_fine": dt_f, "M_max_stable": best, "dt_coarse": best * dt_f, "tried": tried}


def main(argv=None) -> int:
    """python -m paper_2106_07154_gb300.maxdt [--workload NAME] [--layers 1 2 3]:
    the protocol on a named synthetic workload for each interface thickness,
    one JSON line each."""
    from . import workloads as W

    ap = argparse.ArgumentParser(description=main.__doc__)
    ap.add_argument("--workload", default="scvt_40962")
    ap.add_argument("--layers", type=int, nargs="+", default=[1, 2, 3],
                    help="interface thicknesses (cells) to run the protocol for")
    ap.add_argument("--coarse-steps", type=float, default=100.0,
                    help="simulated time T in units of the workload's coarse step")
    ap.add_argument("--M-max", type=int, default=32)
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    args = ap.parse_args(argv)
    w = W.workload(args.workload)
    T = args.coarse_steps * w.dt
    prec = lts.LTS_FP32 if args.precision == "fp32" else lts.LTS_FP64
    for L in args.layers:
        t0 = time.perf_counter()
        res = max_dt_protocol(w.mesh, w.fine_mask, w.h0, w.u0, w.g, w.dt / w.M, T, M_max=args.M_max,
                              precision=prec, layers=L)
        res.update({"workload": w.name, "interface_layers": L, "T_s": T,
                    "workload_dt_fine_s": w.dt / w.M, "seconds": time.perf_counter() - t0})
        print(json.dumps(res), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
