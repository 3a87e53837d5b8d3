"""Benchmark of the LTS3 coarse step (Algorithm 2.2) on one or more GB300s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl lts|reference]

A "step" is one LTS3 coarse step of the whole hot path (Steps 1-5 with M fine
substeps) over the synthetic 655,362-cell spherical SCVT with an 8:1 refined
cap (M = 8), FP32 state with compensation words.  The JSON line reports
coarse-step cell-updates/s (nCells x coarse steps / time), timed with CUDA
events on the state's stream over exactly K steps after W warm-up steps,
max over ranks.  Under torchrun every rank advances its own replica (the path
has no exchange step on one GPU), so the aggregate is weak scaling.

--workload ensemble64 times the batched ensemble instead: 64 uneven
spherical SCVT members (2,562 to 163,842 cells, ratios and M in {2, 4, 8})
advanced together, one launch per phase for all members; under torchrun the
members are partitioned over the ranks (strong scaling, no collective on
the data path).

--impl reference times the FP64 CPU oracle (the reference arm of this
build) on the host cores on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import dataclasses
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

METRIC = "LTS coarse-step cell-updates/s"
UNIT = "cell-updates/s"
PEAKS = ROOT / "MEASURED_PEAKS.json"
HBM_FALLBACK_GBS = 6800.0
TRAFFIC_SUMMARY = ROOT / "profiles" / "ring_kernel_scvt655362_fp32c.md"
LAUNCH_SUMMARY = ROOT / "profiles" / "lts3_step_launches_scvt655362_fp32c.md"
KERNEL_SRC = ROOT / "paper_2106_07154_gb300" / "csrc" / "kernels.cu"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="lts", choices=["lts", "reference"])
    ap.add_argument("--workload", default="scvt_655362")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--e2e-steps", type=int, default=100)
    ap.add_argument("--no-extras", action="store_true", help="skip e2e/roofline/baselines")
    ap.add_argument("--no-graph", action="store_true", help="direct launches instead of the graph")
    ap.add_argument("--no-pdl", action="store_true", help="no programmatic dependent launch")
    ap.add_argument("--layers", type=int, default=1,
                    help="independent layers per cell (the paper's 100-layer ocean workload)")
    ap.add_argument("--order", type=int, default=3, choices=[2, 3],
                    help="3 = LTS3 (default), 2 = LTS2 (Algorithm 2.2's second-order branches)")
    ap.add_argument("--interface-layers", type=int, default=1,
                    help="interface thickness in cells (the paper's thick-interface runs)")
    ap.add_argument("--dt-scale", type=float, default=1.0,
                    help="multiplies the workload's coarse step (LTS2 is not stable at the "
                         "LTS3 step on pure gravity waves)")
    ap.add_argument("--elems-per-thread", type=int, default=0, choices=[0, 1, 2],
                    help="elements per thread of the vertex and edge launches (0 = library default)")
    ap.add_argument("--autotune", type=int, default=0,
                    help="time the run with the configuration the library's autotuner picks "
                         "(coarse steps per candidate; 0 = library defaults)")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# --------------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------- helpers

def kernel_hash() -> str:
    """The first 16 hex digits of the sha256 of kernels.cu's code: comments
    and blank lines removed, so that a comment edit keeps the committed ncu
    figures while any change to the code retires them."""
    src = KERNEL_SRC.read_text()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    code = "\n".join(ln.rstrip() for ln in src.splitlines() if ln.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def hbm_peak():
    try:
        p = json.loads(PEAKS.read_text())
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_FALLBACK_GBS, "fallback"


def dram_traffic_per_launch():
    """DRAM bytes per launch of the ring kernel from the committed ncu
    summary, or None when the kernel source changed since the capture."""
    try:
        text = TRAFFIC_SUMMARY.read_text()
        m = re.search(r"```json\s*(\{.*?\})\s*```", text, re.S)
        data = json.loads(m.group(1))
        if data.get("kernels_cu_code_sha256_16") != kernel_hash():
            return None
        return float(data["ring_dram_bytes_per_launch"])
    except Exception:
        return None


def device_time_shares():
    """Per-kind shares of device time from the committed ncu launch list, or
    None when the kernel source changed since the capture."""
    try:
        text = LAUNCH_SUMMARY.read_text()
        m = re.search(r"```json\s*(\{.*?\})\s*```", text, re.S)
        data = json.loads(m.group(1))
        if data.get("kernels_cu_code_sha256_16") != kernel_hash():
            return None
        return data["shares"]
    except Exception:
        return None


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    return "unknown"


def mmax(w):
    """The largest M of the workload (several fine regions carry one M each)."""
    return int(max(w.M)) if np.ndim(w.M) else int(w.M)


def oracle_lts(o, w, h, u, n, labels=None):
    """n oracle coarse steps of the workload (several regions: or_lts3_multi;
    order 2: LTS2; thicker interfaces through the labels)."""
    if np.ndim(w.M):
        return o.lts3_multi(h, u, w.fine_mask, list(w.M), w.dt, n, g=w.g)
    cl, el = labels if labels is not None else oracle_labels(o, w)
    if w.order == 2:
        return o.lts2(h, u, cl, el, w.M, w.dt, n, g=w.g)
    return o.lts3(h, u, cl, el, w.M, w.dt, n, g=w.g)


def load_workload(args):
    """The named workload with the command line's scheme order, interface
    thickness and time-step scale."""
    from paper_2106_07154_gb300 import workloads as W

    w = W.workload(args.workload)
    if args.order == 3 and args.interface_layers == 1 and args.dt_scale == 1.0:
        return w
    if np.ndim(w.M) and (args.order != 3 or args.interface_layers != 1):
        raise SystemExit("the workload with several fine regions runs LTS3 with one-cell interfaces")
    return dataclasses.replace(w, order=args.order, interface_layers=args.interface_layers,
                               dt=w.dt * args.dt_scale)


def is_variant(w):
    return w.order != 3 or w.interface_layers != 1


def oracle_labels(o, w):
    return None if np.ndim(w.M) else o.regions(w.fine_mask, w.interface_layers)


def predicted_speedup(counts, M):
    """Work-count prediction of the LTS3 speed-up over global SSP-RK3 at the
    fine step (the paper's optimal-ratio estimate of Section 3.3, extended by
    the interface corrections): cell right-hand-side evaluations per coarse
    step, 3 M N for global SSP-RK3 against
    3 N_C + (2 + 3M) N_I + N_Fbar + 3M N_F for LTS3.  Band counts in library
    band order: F deep, F3, F2, F1 (fine), I1, I2 (interface), C1.. (coarse);
    Fbar = F2 and F1, the fine cells Step 1 also evaluates."""
    c = np.asarray(counts, np.float64)
    nF, nFbar, nI, nC = c[0:4].sum(), c[2:4].sum(), c[4:6].sum(), c[6:].sum()
    n = c.sum()
    lts_work = 3 * nC + (2 + 3 * M) * nI + nFbar + 3 * M * nF
    return {"predicted": float(3 * M * n / lts_work), "cells": {"fine": int(nF), "interface": int(nI),
                                                                "coarse": int(nC)}}


def set_omp_threads(n: int) -> bool:
    """Sets the OpenMP thread count of the calling thread (the oracle's
    parallel loops then use n threads); False if libgomp is not loaded."""
    import ctypes

    try:
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(int(n))
        return True
    except (OSError, AttributeError):
        return False


def oracle_single_thread(w, budget_s=20.0):
    """The oracle on one host thread: LTS3 coarse steps of the full mesh until
    `budget_s` is spent (at least one); cell-updates/s, steps, seconds."""
    import oracle

    o = oracle.Oracle(w.mesh)
    labels = oracle_labels(o, w)
    cores = oracle.num_threads()
    if not set_omp_threads(1):
        return None
    try:
        h, u = w.h0, w.u0
        steps, t = 0, 0.0
        while steps == 0 or t < budget_s:
            t0 = time.perf_counter()
            h, u = oracle_lts(o, w, h, u, 1, labels)
            t += time.perf_counter() - t0
            steps += 1
            if steps >= 3:
                break
    finally:
        set_omp_threads(cores)
    return w.nCells * steps / t, steps, t


def oracle_sample(w, nsteps_cap=3, budget_s=20.0, h0=None, u0=None):
    """Times the FP64 oracle's LTS3 coarse step on the full workload (from
    h0, u0 when given, else the workload's initial state); returns
    (cell-updates/s, steps, seconds, threads, result)."""
    import oracle

    o = oracle.Oracle(w.mesh)
    labels = oracle_labels(o, w)
    h, u = (w.h0, w.u0) if h0 is None else (h0, u0)
    steps, t_total = 0, 0.0
    while steps < nsteps_cap and t_total < budget_s:
        t0 = time.perf_counter()
        h, u = oracle_lts(o, w, h, u, 1, labels)
        t_total += time.perf_counter() - t0
        steps += 1
    return w.nCells * steps / t_total, steps, t_total, oracle.num_threads(), (h, u)


# --------------------------------------------------------------------- arms

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2106_07154_gb300 import workloads as W

    if args.workload == "ensemble64":
        return run_reference_ensemble(args)
    w = load_workload(args)
    import oracle

    o = oracle.Oracle(w.mesh)
    labels = oracle_labels(o, w)
    h, u = w.h0, w.u0
    # one oracle coarse step takes about a second on the 655k-cell mesh:
    # the requested warm-up steps run (stopped after 60 s, which the line
    # then reports), and the timed steps stop after 90 s, so the whole arm
    # ends within a few minutes
    warm, tw = 0, time.perf_counter()
    while warm < args.warmup and time.perf_counter() - tw < 60.0:
        h, u = oracle_lts(o, w, h, u, 1, labels)
        warm += 1
    t0 = time.perf_counter()
    steps = 0
    while steps < args.steps:
        h, u = oracle_lts(o, w, h, u, 1, labels)
        steps += 1
        if time.perf_counter() - t0 > 90.0:
            break
    el_s = time.perf_counter() - t0
    value = w.nCells * steps / el_s
    cores = oracle.num_threads()
    sample = (f"{steps} {scheme(w)} coarse steps (M={w.M}) of the full {w.nCells}-cell mesh by the FP64 "
              f"C oracle (full-mesh right-hand sides) after {warm} warm-up step(s)"
              f"{'' if warm == args.warmup else f' (of {args.warmup} requested; warm-up stopped at 60 s)'}"
              f"; timed steps capped at 90 s")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": warm, "ms_per_step": 1e3 * el_s / steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": workload_config(w, "fp64-oracle"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_reference_ensemble(args):
    """The oracle on the ensemble's members in order, one coarse step each,
    until 90 s of oracle time (the members' meshes are built untimed)."""
    import oracle
    from paper_2106_07154_gb300 import workloads as W

    recipes = W.ensemble_recipes()
    cells, t_or, done = 0, 0.0, 0
    for r in recipes:
        w = W.sphere_cap(**r)
        o = oracle.Oracle(w.mesh)
        cl, el = o.regions(w.fine_mask)
        t0 = time.perf_counter()
        o.lts3(w.h0, w.u0, cl, el, w.M, w.dt, 1, g=w.g)
        t_or += time.perf_counter() - t0
        cells += w.nCells
        done += 1
        if t_or > 90.0:
            break
    value = cells / t_or
    cfg = ensemble_config(recipes, recipes, 1)
    cfg["nCells_total"] = sum(r["n"] for r in recipes)
    sample = f"one LTS3 coarse step of the first {done} members ({cells} cells) by the FP64 C oracle"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 1,
            "steps": 1, "warmup": 0, "ms_per_step": 1e3 * t_or * cfg["nCells_total"] / cells,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample, "cpu": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def scheme(w):
    s = f"LTS{w.order}"
    if w.interface_layers != 1:
        s += f" with {w.interface_layers}-cell interfaces"
    return s


def workload_config(w, precision):
    if np.ndim(w.M):
        caps = " and ".join(f"{int(r)}:1 (M={m})" for r, m in zip(w.info["ratios"], w.M))
        what = f"two refined caps {caps}, 32 ridges, 5 m spectral noise, {scheme(w)}"
    elif "ratio" in w.info:
        what = f"{int(w.info['ratio'])}:1 cap, {scheme(w)} M={w.M}"
    else:
        what = f"fine circle, {scheme(w)} M={w.M}"
    mesh = "spherical SCVT, 200 Lloyd iterations" if w.mesh.get("on_sphere") else "doubly periodic hexagons"
    return {"workload": f"{w.name}: {mesh}, {w.nCells} cells, {what}",
            "nCells": w.nCells, "nEdges": int(w.mesh["nEdges"]),
            "M": list(w.M) if np.ndim(w.M) else w.M,
            "dt_coarse_s": w.dt, "precision": precision,
            "l2": "inputs larger than L2 (each coarse step streams the whole mesh)",
            "parallelism": "replicas"}


def run_lts(args):
    import torch

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend=backend)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for --impl lts")
    torch.cuda.set_device(local)
    from paper_2106_07154_gb300 import lts

    # rank 0 builds (and caches) the mesh first, the others load it
    if world > 1 and rank != 0:
        torch.distributed.barrier()
    w = load_workload(args)
    if world > 1 and rank == 0:
        torch.distributed.barrier()
    prec = lts.LTS_FP32 if args.precision == "fp32" else lts.LTS_FP64
    stream = torch.cuda.Stream()
    tune = args.autotune if (args.autotune and not args.no_graph and not args.no_pdl) else 0
    L = max(1, args.layers)
    h0, u0 = w.h0, w.u0
    if L > 1:   # seeded, slightly different layers
        rng = np.random.default_rng(11)
        h0 = w.h0[None, :] * (1.0 + 1e-4 * rng.standard_normal((L, w.nCells)))
        u0 = np.tile(w.u0, (L, 1)) * (1.0 + 0.01 * np.arange(L))[:, None]
    model = lts.Model(w.mesh, w.fine_mask, w.M, h0, u0, w.dt, w.g, precision=prec,
                      compensated=True, use_graph=not args.no_graph, stream=stream.cuda_stream,
                      pdl=not args.no_pdl, autotune=tune, tune_ordering=bool(tune), layers=L,
                      order=w.order, interface_layers=w.interface_layers,
                      elems_per_thread=args.elems_per_thread)
    stats = model.stats()
    model.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    start.record(stream)
    model.step(args.steps)
    stop.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = start.elapsed_time(stop)
    if world > 1:
        torch.distributed.barrier()
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    h_gpu, u_gpu, diag = model.read()
    value = world * w.nCells * L * args.steps / (ms * 1e-3)
    launch_cfg = ("direct launches" if args.no_graph else "one CUDA graph per coarse step") + \
        ("" if args.no_pdl else ", programmatic dependent launch")
    if model.tuned:
        launch_cfg += ", configuration chosen by the library's autotuner"
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == lts.LTS_FP32 else "f64", "data": "synthetic",
            "config": workload_config(w, args.precision + ("+compensation" if prec == 0 else "")),
            "gpu_launches": stats["launches"] * args.steps, "clocks": clk, "launch": launch_cfg,
            "sim_seconds_per_wall_second": w.dt * args.steps / (ms * 1e-3)}
    if model.tuned:
        line["config"]["tuned"] = model.tuned
    if L > 1:
        line["config"]["layers"] = L
        line["config"]["workload"] += f", {L} independent layers per cell (cell-layer updates)"
    if L > 1 or np.ndim(w.M) or is_variant(w):
        # per-kernel profiling runs single-region single-layer LTS3 states only:
        # the whole step against the roofline instead
        peak, peak_src = hbm_peak()
        bytes_step = float(sum(stats["bytes"]))
        achieved = bytes_step / (ms / args.steps * 1e-3) / 1e9
        line["roofline"] = {"bound": "hbm", "kernel": "whole step (all kinds)", "achieved": achieved,
                            "peak": peak, "unit": "GB/s", "frac": achieved / peak, "traffic": None,
                            "algorithmic_bytes_per_step": bytes_step,
                            "bytes_per_cell_layer_step": bytes_step / (w.nCells * L)}
    if (np.ndim(w.M) or is_variant(w)) and L == 1 and not args.no_extras and rank == 0:
        # several fine regions, LTS2, thick interfaces: the oracle baseline
        # and the error of one step
        cells_per_s, n_or, t_or, cores, (rh, ru) = oracle_sample(w, nsteps_cap=1)
        one = lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=prec,
                        compensated=True, stream=stream.cuda_stream, order=w.order,
                        interface_layers=w.interface_layers)
        one.step(1)
        h1, u1, _ = one.read()
        one.close()
        line["cpu_baseline"] = {"value": cells_per_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                                "sample": f"{n_or} coarse step(s) of the full mesh by the FP64 C oracle "
                                          f"({scheme(w)}, {t_or:.1f} s)", "cpu": cpu_model()}
        line["error_vs_oracle_1step"] = {
            "h_rel_maxnorm": float(np.max(np.abs(h1 - rh)) / np.max(np.abs(rh))),
            "u_rel_maxnorm": float(np.max(np.abs(u1 - ru)) / np.max(np.abs(ru)))}
    if L > 1 and not args.no_extras and rank == 0:
        # multi-layer state: the oracle's coarse step on three of its layers
        # (first, middle, last) and the GPU's error on them after one step
        sample = sorted({0, L // 2, L - 1})
        one = lts.Model(w.mesh, w.fine_mask, w.M, h0, u0, w.dt, w.g, precision=prec, compensated=True,
                        stream=stream.cuda_stream, layers=L, order=w.order,
                        interface_layers=w.interface_layers)
        one.step(1)
        h1, u1, _ = one.read()
        one.close()
        t_or, eh, eu, cores = 0.0, 0.0, 0.0, 1
        for k in sample:
            _, _, t, cores, (rh, ru) = oracle_sample(w, nsteps_cap=1, h0=h0[k], u0=u0[k])
            t_or += t
            eh = max(eh, float(np.max(np.abs(h1[k] - rh)) / np.max(np.abs(rh))))
            eu = max(eu, float(np.max(np.abs(u1[k] - ru)) / np.max(np.abs(ru))))
        line["cpu_baseline"] = {"value": w.nCells * len(sample) / t_or, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "cpu": cpu_model(),
                                "sample": f"one coarse step of layers {sample} of the full mesh by the FP64 C "
                                          f"oracle ({scheme(w)}, {t_or:.1f} s; cell-layer updates)"}
        line["error_vs_oracle_1step"] = {"layers": sample, "h_rel_maxnorm": eh, "u_rel_maxnorm": eu}
    if not args.no_extras and rank == 0 and L == 1 and not np.ndim(w.M) and not is_variant(w):
        args._ms = ms
        line.update(extras(args, w, model, stats, stream, h_gpu, u_gpu, diag))
    model.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def in_graph_estimate(args, bytes_kind, launches_kind, dom, peak):
    """The dominant kernel inside the production graph, where programmatic
    dependent launch overlaps consecutive kernels: its share of device time
    (committed ncu launch list) times the graph's step time, per launch."""
    shares = device_time_shares()
    if not shares or args._ms is None:
        return None
    from paper_2106_07154_gb300 import lts

    share = shares.get(lts.KIND_NAMES[dom])
    if not share:
        return None
    t_launch = args._ms / args.steps * share / launches_kind[dom]
    gbs = bytes_kind[dom] / launches_kind[dom] / (t_launch * 1e-3) / 1e9
    return {"GB_per_s": float(gbs), "frac": float(gbs / peak), "share": share,
            "method": "graph step time x the kind's ncu share of device time / its launches per step"}


def extras(args, w, model, stats, stream, h_gpu, u_gpu, diag):
    import torch
    from paper_2106_07154_gb300 import lts

    out = {}
    prec = lts.LTS_FP32 if args.precision == "fp32" else lts.LTS_FP64
    nC, nE = w.nCells, int(w.mesh["nEdges"])
    # ---- end to end through the C ABI with pinned host buffers
    hb = torch.empty(nC, dtype=torch.float64, pin_memory=True).numpy()
    ub = torch.empty(nE, dtype=torch.float64, pin_memory=True).numpy()
    hb[:] = w.h0
    ub[:] = w.u0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        model.write(hb, ub)
        model.step(1)
        model.read(hb, ub)
    e2e_s = time.perf_counter() - t0
    round_trip = {"value": nC * args.e2e_steps / e2e_s, "unit": UNIT,
                  "h2d_bytes_per_step": 8 * (nC + nE),
                  "d2h_bytes_per_step": 8 * (nC + nE) + 16 + 4,
                  "steps": args.e2e_steps,
                  "note": "lts_write (H2D of h,u) + lts_step(1) + lts_read (D2H of h,u, FP64 "
                          "mass/energy) per step, each step resuming from the state read back; "
                          "pinned host buffers, wall clock"}
    # ---- streamed: every step uploads a state, advances it one coarse step
    #      and reads it back with its diagnostics (lts_write, lts_step,
    #      lts_read_async), one lts_sync per `depth` steps, so the copies of
    #      neighbouring steps overlap the steps
    depth = 16
    hin = [torch.empty(nC, dtype=torch.float64, pin_memory=True).numpy() for _ in range(depth)]
    uin = [torch.empty(nE, dtype=torch.float64, pin_memory=True).numpy() for _ in range(depth)]
    hout = [torch.empty(nC, dtype=torch.float64, pin_memory=True).numpy() for _ in range(depth)]
    uout = [torch.empty(nE, dtype=torch.float64, pin_memory=True).numpy() for _ in range(depth)]
    for j in range(depth):
        hin[j][:] = w.h0
        uin[j][:] = w.u0
    nstream = depth * max(1, args.e2e_steps // depth)
    for j in range(depth):      # one untimed group
        model.write(hin[j], uin[j])
        model.step(1)
        model.read_async(hout[j], uout[j], diag=True)
    model.sync()
    t0 = time.perf_counter()
    for k in range(nstream):
        j = k % depth
        model.write(hin[j], uin[j])
        model.step(1)
        model.read_async(hout[j], uout[j], diag=True)
        if j == depth - 1:
            model.sync()
    e2e_s = time.perf_counter() - t0
    out["e2e"] = {"value": nC * nstream / e2e_s, "unit": UNIT,
                  "h2d_bytes_per_step": 8 * (nC + nE),
                  "d2h_bytes_per_step": 8 * (nC + nE) + 16 + 4,
                  "steps": nstream,
                  "note": f"streamed through the C ABI: per step lts_write (H2D of h,u from pinned "
                          f"memory), lts_step(1), lts_read_async (D2H of h,u and FP64 mass/energy); "
                          f"one lts_sync per {depth} steps, so copies overlap neighbouring steps; "
                          f"wall clock",
                  "round_trip": round_trip}
    # ---- per-kernel timing: the same coarse-step graph with an event-record
    #      node before and after every kernel node, on the state's stream
    tuned = model.tuned or {}
    knobs = {k: tuned[k] for k in ("block_size", "kernel_path", "l2_hints", "coarse_schedule",
                                   "ring_occupancy", "elems_per_thread") if k in tuned}
    knobs.setdefault("elems_per_thread", args.elems_per_thread)
    if "ordering" in tuned:
        knobs["ordering"] = tuned["ordering"]
    prof = lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=prec,
                     compensated=True, profile=2, stream=stream.cuda_stream, **knobs)
    nprof = 20
    prof.step(2)
    ms_sum = np.zeros(lts.LTS_NKINDS)
    for _ in range(nprof):
        prof.step(1)
        ms_sum += np.array(prof.stats()["ms"])
    prof.close()
    ms_kind = ms_sum / nprof
    # the same launches issued directly on the stream with an event pair
    # around each (no graph, no programmatic overlap)
    prof1 = lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=prec,
                      compensated=True, profile=1, stream=stream.cuda_stream, **knobs)
    prof1.step(2)
    ms1 = np.zeros(lts.LTS_NKINDS)
    for _ in range(nprof):
        prof1.step(1)
        ms1 += np.array(prof1.stats()["ms"])
    prof1.close()
    ms1 /= nprof
    bytes_kind = np.array(stats["bytes"])
    launches_kind = np.array(stats["launches_per_kind"])
    has = launches_kind > 0
    gbs = np.where(has, bytes_kind / np.maximum(ms_kind, 1e-12) / 1e6, 0.0)
    dom = int(np.argmax(np.where(has, ms_kind, -1.0)))
    peak, peak_src = hbm_peak()
    traffic = dram_traffic_per_launch() if dom == 1 else None
    out["roofline"] = {
        "bound": "hbm", "kernel": lts.KIND_NAMES[dom],
        "achieved": float(gbs[dom]), "peak": peak, "unit": "GB/s", "frac": float(gbs[dom] / peak),
        "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)" if peak_src == "measured" else "fallback 6.8 TB/s",
        "traffic": traffic,
        "algorithmic_bytes_per_launch": float(bytes_kind[dom] / launches_kind[dom]),
        "avg_launch_ms": float(ms_kind[dom] / launches_kind[dom]),
        "per_kind": {lts.KIND_NAMES[k]: {"ms_per_step": float(ms_kind[k]),
                                          "bytes_per_step": float(bytes_kind[k]),
                                          "launches_per_step": int(launches_kind[k]),
                                          "GB_per_s": float(gbs[k])}
                     for k in range(lts.LTS_NKINDS) if has[k]},
        "timing": "per-kernel CUDA events: an event-record node before and after every kernel "
                  "node of the coarse-step graph (20 steps after the timed region)",
        "in_graph_estimate": in_graph_estimate(args, bytes_kind, launches_kind, dom, peak),
        "per_kind_direct_launch_events": {
            lts.KIND_NAMES[k]: {"ms_per_step": float(ms1[k]),
                                "GB_per_s": float(bytes_kind[k] / (ms1[k] * 1e-3) / 1e9) if ms1[k] > 0 else None}
            for k in range(lts.LTS_NKINDS) if has[k]},
    }
    # ---- the library's autotuner on this workload (report only)
    if not model.tuned:
        base = lts.make_params(w.g, w.dt, prec, lts.LTS_MODE_LTS3, True, True)
        mh = lts.lts_mesh_create(w.mesh)
        rh = (lts.lts_regions_set_multi(mh, w.fine_mask, list(w.M)) if np.ndim(w.M)
              else lts.lts_regions_set(mh, w.fine_mask, 3, w.M))
        best, rep = lts.lts_autotune(mh, rh, w.h0, w.u0, base, 20, tune_ordering=True)
        lts.lts_regions_destroy(rh)
        lts.lts_mesh_destroy(mh)
        out["autotune"] = dict(lts.params_dict(best), **rep)
    # ---- the GPU's own FP64 global SSP-RK3 at the fine step (same simulated time)
    Mx = mmax(w)
    ref = lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt / Mx, w.g, precision=lts.LTS_FP64,
                    mode=lts.LTS_MODE_SSPRK3, stream=stream.cuda_stream)
    ref.step(Mx)
    torch.cuda.synchronize()
    ncmp = max(2, min(50, args.steps // 20))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    ref.step(ncmp * Mx)
    e1.record(stream)
    torch.cuda.synchronize()
    ref_ms = e0.elapsed_time(e1) / ncmp
    ref.close()
    out["fp64_ssprk3_fine_dt"] = {"ms_per_coarse_interval": ref_ms,
                                  "sim_seconds_per_wall_second": w.dt / (ref_ms * 1e-3),
                                  "note": f"FP64 SSPRK3 on the whole mesh at dt/M = {w.dt / Mx:.3f} s"}
    # ---- the LTS speed-up at equal precision: global FP32 SSP-RK3 at dt/M
    #      against this run's coarse step, beside the work-count prediction
    ref32 = lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt / Mx, w.g, precision=prec,
                      compensated=True, mode=lts.LTS_MODE_SSPRK3, stream=stream.cuda_stream)
    ref32.step(Mx)
    torch.cuda.synchronize()
    e0.record(stream)
    ref32.step(ncmp * Mx)
    e1.record(stream)
    torch.cuda.synchronize()
    ref32_ms = e0.elapsed_time(e1) / ncmp
    counts, _, _ = lts.lts_regions_counts(model.reg_h)
    out["lts_speedup"] = dict(predicted_speedup(counts, Mx),
                              measured=ref32_ms / (args._ms / args.steps),
                              ssprk3_fine_dt_ms_per_coarse_interval=ref32_ms,
                              note="global SSPRK3 (same precision) at dt/M over dt, divided by one LTS3 "
                                   "coarse step; predicted = RHS cell-evaluations of the two")
    ref32.close()
    # ---- CPU baseline (oracle on the host cores) and the error of this run's
    #      first coarse step against it
    cells_per_s, n_or, t_or, cores, (rh, ru) = oracle_sample(w, nsteps_cap=1)
    one = lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=prec,
                    compensated=True, stream=stream.cuda_stream)
    one.step(1)
    h1, u1, _ = one.read()
    one.close()
    out["cpu_baseline"] = {"value": cells_per_s, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"{n_or} LTS3 coarse step(s) of the full mesh by the FP64 C "
                                     f"oracle ({t_or:.1f} s)", "cpu": cpu_model()}
    st1 = oracle_single_thread(w)
    if st1 is not None:
        out["cpu_baseline"]["single_thread"] = {
            "value": st1[0], "unit": UNIT, "cores": 1,
            "sample": f"{st1[1]} LTS3 coarse step(s) of the full mesh by the FP64 C oracle on one "
                      f"thread ({st1[2]:.1f} s)"}
    # ---- the workload's own run length (hex_1024: 100 coarse steps,
    #      scvt_40962: 500): FP32 and FP64 against the oracle after that many
    #      steps, and the drift of mass and energy, where the oracle needs at
    #      most a minute for them on the host cores
    if t_or / n_or * w.nsteps <= 60.0:
        import oracle

        o = oracle.Oracle(w.mesh)
        labels = oracle_labels(o, w)
        t0 = time.perf_counter()
        rhn, run_ = oracle_lts(o, w, w.h0, w.u0, w.nsteps, labels)
        t_full = time.perf_counter() - t0
        res = {"coarse_steps": w.nsteps,
               "oracle": {"seconds": t_full, "value": nC * w.nsteps / t_full, "unit": UNIT,
                          "cores": cores,
                          "mass_drift": (o.mass(rhn) - o.mass(w.h0)) / o.mass(w.h0),
                          "energy_drift": (o.energy(rhn, run_, w.g) - o.energy(w.h0, w.u0, w.g))
                          / o.energy(w.h0, w.u0, w.g)}}
        for name, p_ in (("fp32", lts.LTS_FP32), ("fp64", lts.LTS_FP64)):
            with lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=p_,
                           compensated=True, stream=stream.cuda_stream) as m_:
                _, _, d0 = m_.read()
                m_.step(w.nsteps)
                hn, un_, dn = m_.read()
            res[name] = {"h_rel_maxnorm": float(np.max(np.abs(hn - rhn)) / np.max(np.abs(rhn))),
                         "u_rel_maxnorm": float(np.max(np.abs(un_ - run_)) / np.max(np.abs(run_))),
                         "mass_drift": (dn["mass"] - d0["mass"]) / d0["mass"],
                         "energy_drift": (dn["energy"] - d0["energy"]) / d0["energy"]}
        out["run_vs_oracle"] = res
    out["error_vs_oracle_1step"] = {
        "h_rel_maxnorm": float(np.max(np.abs(h1 - rh)) / np.max(np.abs(rh))),
        "u_rel_maxnorm": float(np.max(np.abs(u1 - ru)) / np.max(np.abs(ru)))}
    out["mass"] = diag["mass"]
    # ---- FP64 LTS3 (oracle-matching precision) on the same workload
    m64 = lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=lts.LTS_FP64,
                    stream=stream.cuda_stream)
    m64.step(1)
    h64, u64, _ = m64.read()
    m64.step(3)
    torch.cuda.synchronize()
    n64 = max(5, min(200, args.steps // 10))
    e0.record(stream)
    m64.step(n64)
    e1.record(stream)
    torch.cuda.synchronize()
    ms64 = e0.elapsed_time(e1) / n64
    m64.close()
    out["fp64_lts3"] = {"ms_per_step": ms64, "value": nC / (ms64 * 1e-3), "unit": UNIT,
                        "error_vs_oracle_1step": {
                            "h_rel_maxnorm": float(np.max(np.abs(h64 - rh)) / np.max(np.abs(rh))),
                            "u_rel_maxnorm": float(np.max(np.abs(u64 - ru)) / np.max(np.abs(ru)))}}
    # ---- accuracy at equal simulated time: 10 coarse steps of LTS3-FP32 and of
    #      FP64 SSPRK3 at dt/M, both against FP64 SSPRK3 at dt/(4M)
    nco = 10

    def run(prec_, mode_, dt_, n_):
        with lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, dt_, w.g, precision=prec_, mode=mode_,
                       stream=stream.cuda_stream) as m_:
            m_.step(n_)
            hh, uu, _ = m_.read()
        return hh, uu

    hr, ur = run(lts.LTS_FP64, lts.LTS_MODE_SSPRK3, w.dt / (4 * Mx), nco * 4 * Mx)
    hl, ul = run(lts.LTS_FP32, lts.LTS_MODE_LTS3, w.dt, nco)
    hs, us = run(lts.LTS_FP64, lts.LTS_MODE_SSPRK3, w.dt / Mx, nco * Mx)

    def err(a, b):
        return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))

    out["accuracy_10_coarse_steps"] = {
        "reference": f"FP64 SSPRK3 at dt/(4M) = {w.dt / (4 * Mx):.3f} s over {nco} coarse steps",
        "lts3_fp32": {"h": err(hl, hr), "u": err(ul, ur),
                      "sim_seconds_per_wall_second": w.dt * args.steps / (args._ms * 1e-3)},
        "ssprk3_fp64_fine_dt": {"h": err(hs, hr), "u": err(us, ur),
                                "sim_seconds_per_wall_second": w.dt / (ref_ms * 1e-3)},
        "h_initial_vs_reference": err(w.h0, hr)}
    return out


# ------------------------------------------------------------------ ensemble

def ensemble_config(recipes, mine, world):
    return {"workload": f"ensemble64: {len(recipes)} spherical SCVT members, "
                        f"{min(r['n'] for r in recipes)}..{max(r['n'] for r in recipes)} cells, "
                        "ratio = M in {2,4,8}, 200 Lloyd iterations, one launch per phase",
            "members": len(recipes), "members_rank0": len(mine),
            "nCells_total": None, "precision": "fp32+compensation",
            "l2": "inputs larger than L2 (each coarse step streams every member's mesh)",
            "parallelism": f"members partitioned over {world} rank(s)" if world > 1 else "1 GPU"}


def run_ensemble(args):
    import torch
    from paper_2106_07154_gb300 import lts, shard
    from paper_2106_07154_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group(backend="nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU for --impl lts")
    torch.cuda.set_device(local)
    recipes = W.ensemble_recipes()
    weights = [r["n"] * r["M"] for r in recipes]
    parts = shard.greedy_partition(weights, world)
    mine = parts[rank]
    ws = [W.sphere_cap(**recipes[i]) for i in mine]
    cells_all = None
    stream = torch.cuda.Stream()
    models = [lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=lts.LTS_FP32,
                        compensated=True) for w in ws]
    ens = lts.Ensemble(models, stream=stream.cuda_stream)
    st = ens.stats()
    my_cells = st["cells"]
    if world > 1:
        t = torch.tensor([my_cells], dtype=torch.int64, device="cuda")
        torch.distributed.all_reduce(t)
        cells_all = int(t.item())
    else:
        cells_all = my_cells
    ens.step(args.warmup)
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device())
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0.record(stream)
    ens.step(args.steps)
    e1.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    if world > 1:
        torch.distributed.barrier()
        t = torch.tensor([ms], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    cfg = ensemble_config(recipes, mine, world)
    cfg["nCells_total"] = cells_all
    peak, peak_src = hbm_peak()
    bytes_step = float(sum(st["bytes"]))
    line = {"metric": METRIC, "value": cells_all * args.steps / (ms * 1e-3), "unit": UNIT,
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": cfg,
            "gpu_launches": st["launches"] * args.steps, "clocks": clk,
            "launch": "one CUDA graph per ensemble coarse step, one segment-table launch per phase "
                      "for all members (one block per 256-element piece), programmatic dependent launch",
            "segments_per_step": st["segments"]}
    if rank == 0 and not args.no_extras:
        achieved = bytes_step / (ms / args.steps * 1e-3) / 1e9
        line["roofline"] = {"bound": "hbm", "kernel": "whole ensemble step (all kinds)",
                            "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": None,
                            "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                            "algorithmic_bytes_per_step": bytes_step}
        # the same members as separate states, one after another on one stream
        sep = [lts.Model(w.mesh, w.fine_mask, w.M, w.h0, w.u0, w.dt, w.g, precision=lts.LTS_FP32,
                         compensated=True, stream=stream.cuda_stream) for w in ws]
        nsep = max(3, min(50, args.steps // 10))
        for m in sep:
            m.step(2)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(nsep):
            for m in sep:
                m.step(1)
        e1.record(stream)
        torch.cuda.synchronize()
        sep_ms = e0.elapsed_time(e1) / nsep
        for m in sep:
            m.close()
        line["separate_states"] = {"ms_per_step": sep_ms,
                                   "value": my_cells / (sep_ms * 1e-3),
                                   "note": "each member its own state and graph, stepped one "
                                           "after another on the same stream"}
        # end to end: every member written from and read back to pinned host memory
        n_e2e = 5
        bufs = []
        for w in ws:
            hb = torch.empty(w.nCells, dtype=torch.float64, pin_memory=True).numpy()
            ub = torch.empty(int(w.mesh["nEdges"]), dtype=torch.float64, pin_memory=True).numpy()
            hb[:] = w.h0
            ub[:] = w.u0
            bufs.append((hb, ub))
        h2d = sum(8 * (b[0].size + b[1].size) for b in bufs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            for i, (hb, ub) in enumerate(bufs):
                ens.write(i, hb, ub)
            ens.step(1)
            for i, (hb, ub) in enumerate(bufs):
                ens.read(i, hb, ub)
        e2e_s = time.perf_counter() - t0
        round_trip = {"value": my_cells * n_e2e / e2e_s, "unit": UNIT, "steps": n_e2e,
                      "note": "per step: lts_ensemble_write of every member, one ensemble step, "
                              "lts_ensemble_read of every member (pinned host buffers, wall clock)"}
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            for i, (hb, ub) in enumerate(bufs):
                ens.write(i, hb, ub)
            ens.step(1)
            for i, (hb, ub) in enumerate(bufs):
                ens.read_async(i, hb, ub, diag=True)
            ens.sync()
        e2e_s = time.perf_counter() - t0
        line["e2e"] = {"value": my_cells * n_e2e / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": h2d + 36 * len(bufs), "steps": n_e2e,
                       "note": "per step: lts_ensemble_write of every member, one ensemble step, "
                               "lts_ensemble_read_async of every member with its FP64 diagnostics, "
                               "one lts_ensemble_sync (pinned host buffers, wall clock)",
                       "round_trip": round_trip}
        # CPU baseline: the oracle's coarse step over every member (passes
        # repeated until about 8 s of oracle time; tables built outside the
        # timed region), and on one thread over the members in size order
        # until about 10 s
        import oracle

        small = sorted(range(len(ws)), key=lambda i: ws[i].nCells)[:2]
        prepared = []
        for w in ws:
            o = oracle.Oracle(w.mesh)
            cl, el = o.regions(w.fine_mask)
            prepared.append((o, cl, el))

        def oracle_steps(order, budget_s):
            t, cells, n = 0.0, 0, 0
            for i in order:
                o, cl, el = prepared[i]
                w = ws[i]
                t0 = time.perf_counter()
                o.lts3(w.h0, w.u0, cl, el, w.M, w.dt, 1, g=w.g)
                t += time.perf_counter() - t0
                cells += w.nCells
                n += 1
                if t >= budget_s:
                    break
            return cells, t, n

        cells, t_or, passes = 0, 0.0, 0
        while t_or < 8.0 and passes < 5:
            c, t, _ = oracle_steps(range(len(ws)), float("inf"))
            cells, t_or, passes = cells + c, t_or + t, passes + 1
        line["cpu_baseline"] = {"value": cells / t_or, "unit": UNIT, "cores": oracle.num_threads(),
                                "kind": "oracle", "cpu": cpu_model(),
                                "sample": f"{passes} LTS3 coarse step(s) of each of the {len(ws)} members "
                                          f"({cells} cell-updates) by the FP64 C oracle ({t_or:.1f} s)"}
        cores = oracle.num_threads()
        if set_omp_threads(1):
            by_size = sorted(range(len(ws)), key=lambda i: ws[i].nCells)
            c1, t1, n1 = oracle_steps(by_size, 10.0)
            set_omp_threads(cores)
            line["cpu_baseline"]["single_thread"] = {
                "value": c1 / t1, "unit": UNIT, "cores": 1,
                "sample": f"one coarse step of the {n1} smallest members ({c1} cells) on one thread ({t1:.1f} s)"}
        del prepared
        # the two smallest members as an ensemble of their own: 20 coarse steps
        # in FP32 against the oracle, and the drift of mass and energy
        nref = 20
        sub = [lts.Model(ws[i].mesh, ws[i].fine_mask, ws[i].M, ws[i].h0, ws[i].u0, ws[i].dt, ws[i].g,
                         precision=lts.LTS_FP32, compensated=True) for i in small]
        d0s = [m.read()[2] for m in sub]
        sens = lts.Ensemble(sub, stream=stream.cuda_stream)
        sens.step(nref)
        chk = []
        for j, i in enumerate(small):
            w = ws[i]
            hg, ug, dn = sens.read(j)
            o = oracle.Oracle(w.mesh)
            cl, el = o.regions(w.fine_mask)
            rh, ru = o.lts3(w.h0, w.u0, cl, el, w.M, w.dt, nref, g=w.g)
            chk.append({"cells": w.nCells, "M": w.M, "coarse_steps": nref,
                        "h_rel_maxnorm": float(np.max(np.abs(hg - rh)) / np.max(np.abs(rh))),
                        "u_rel_maxnorm": float(np.max(np.abs(ug - ru)) / np.max(np.abs(ru))),
                        "mass_drift": (dn["mass"] - d0s[j]["mass"]) / d0s[j]["mass"],
                        "energy_drift": (dn["energy"] - d0s[j]["energy"]) / d0s[j]["energy"]})
        sens.close()
        for m in sub:
            m.close()
        line["members_vs_oracle"] = chk
    ens.close()
    for m in models:
        m.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "ensemble64":
        return run_ensemble(args)
    return run_lts(args)


if __name__ == "__main__":
    sys.exit(main())
