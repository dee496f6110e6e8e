#!/usr/bin/env python
"""Benchmark: forward + adjoint gradient of the coupled LKS / rigid-body march on GB300.

One step = one full gradient (lks_forward over all N_t time steps, lks_adjoint, lks_sensitivity)
of the 512x256 D2Q9 rotating-body workload (128x128 design grid, 5000 steps, N_itr = 5, FP32
fields with FP64 force/torque/EOM, checkpoints every 100 steps) on synthetic seeded inputs.
value = analysis-cell updates per second of the forward + adjoint pass, summed over all ranks
(each rank runs an independent replica: the method has no data-parallel exchange).

Prints one JSON line (rank 0). --impl reference times the FP64 CPU oracle on a bounded sample of
the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "forward+adjoint LKS cell-updates/s vs HBM roofline; gradient rel. err vs FP64"
UNIT = "cell-updates/s"
CONFIG_INDEX = 2


def replica_totals(total_ms: float, launches: int, dist=None, device=None):
    """Whole-job figures of N independent replicas: the slowest rank's time (max over ranks) and
    the launches of all ranks (sum). Without a process group, the local figures."""
    import torch
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    nl = torch.tensor([float(launches)], dtype=torch.float64, device=device)
    if dist:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(nl, op=dist.ReduceOp.SUM)
    return float(t.item()), int(nl.item())


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Algorithmic bytes per launch of each kernel family. N = analysis cells, box_cells = body-box
# cells, ND = design points, esz = bytes per field value, K = N_itr (the persistent families
# "couple" and "adj_body" run all K iterations of a step in one launch).
def _alg_bytes(family: str, P, box_cells: int, esz: int, persistent: bool = True) -> float:
    N, ND = P.n_cells, P.n_design
    d, K = P.dim, P.n_itr
    if family == "stencil_fwd":
        return 2 * (d + 1) * esz * N  # read p, u; write p*, u*
    if family == "stencil_adj":
        return (3 * d + 2) * esz * N  # read the adjoint (d+1 planes) and u(t-1) (d planes); write d+1 planes
    if family == "couple":
        per_iter = d * esz * box_cells + 4 * ND  # read u* in the box (+ kappa^ref)
        if persistent:  # K iterations, then u(t) and the stored u* written once
            return K * per_iter + 2 * d * esz * box_cells
        return per_iter
    if family == "recompute":
        return 3 * d * esz * box_cells + 4 * ND  # read u*, write u and the stored u*
    cell = (5 * d + 1) * esz * box_cells      # read stored u*, acc r/w, scratch write (2d+1 planes)
    design = (2 * d + 1) * esz * box_cells + 20 * ND  # read scratch once, dJ/dkappa^ref r/w + kappa^ref
    if family == "adj_cell":
        return cell
    if family == "adj_design":
        return design
    if family == "adj_body":
        return K * (cell + design)
    if family == "alks_stencil":
        # the paper's adjoint equilibrium and gather. 2D, one tiled pass: read p~, u~, s~
        # (1 + d + d(d+1)/2 planes) and u (d), write the star moments. 3D, two passes: read the
        # moments and u, write Z (d); read p~, Z (1 + d), write the star moments
        ns = 1 + d + d * (d + 1) // 2
        if d == 2:
            return (ns + d + ns) * esz * N
        return ((ns + 2 * d) + (1 + d + ns)) * esz * N
    return 0.0


def _traffic(workload: str, family: str):
    """DRAM bytes per launch of a kernel family measured by ncu (profiles/dram_traffic.json), or None."""
    try:
        with open(os.path.join(ROOT, "profiles", "dram_traffic.json")) as f:
            return json.load(f)[workload][family]["bytes_per_launch"]
    except Exception:
        return None


def _box_cells(P) -> int:
    """Body-box cells of a 2D problem whose body may rotate (circumscribed box, as the library sizes it)."""
    import math
    s = 1 if P.weight_kind == 1 else 2
    half = [(P.ndx - 1) / 2.0, (P.ndy - 1) / 2.0]
    r = math.sqrt(half[0] ** 2 + half[1] ** 2)
    hb = math.ceil(r - 1e-12)
    B = 2 * hb + 2 * s + 2 + 2
    return B * B


def _handle_box_cells(solver, P) -> int:
    """Body-box cells of the handle's workspace (lks_support_sets reports the box it uses)."""
    from paper_2601_18272_gb300 import lks
    _, B, _ = lks.lks_support_sets(solver.handle, _initial_dofs(P))
    return int(np.prod(B))


def _initial_dofs(P):
    from workloads import initial_state
    return initial_state(P)[2]


def _fluid_problem(dim: int, n: tuple, name: str, n_steps: int = 20, every: int = 10):
    """A large grid with a 2^dim design block carrying gamma = 0 (no body): the full-grid stencil
    kernels alone, for their HBM roofline."""
    from workloads import BC_INFLOW_OUTFLOW, BC_PERIODIC, CKPT_UNIFORM, W_COS4, Problem
    nz = n[2] if dim == 3 else 1
    c = (n[0] / 4 + 0.3, n[1] / 2 + 0.4, nz / 2 + 0.2 if dim == 3 else 0.0)
    P = Problem(dim=dim, nx=n[0], ny=n[1], nz=nz, ndx=2, ndy=2, ndz=2 if dim == 3 else 1, body_centre=c,
                rot_axis=2, dof_mask=0, mass=1.0, inertia=1.0, nu=0.032, u_in=0.05, dp=0.0,
                bc=(BC_INFLOW_OUTFLOW, BC_PERIODIC, BC_PERIODIC), kappa_max=1.0, q=0.1, weight_kind=W_COS4,
                n_steps=n_steps, n_itr=5, obj_weights=(1.0,) + (0.0,) * 7, field_precision=32,
                ckpt_policy=CKPT_UNIFORM, ckpt_every=every, name=name)
    return P, np.zeros(P.n_design)


def _family_times(solver, run):
    """Per-family kernel time (ms) and launch count of one call of run() with every launch
    bracketed by CUDA events on the launching stream."""
    import torch
    from paper_2601_18272_gb300 import lks
    lks.lks_set_kernel_timing(solver.handle, True)
    run()
    torch.cuda.synchronize()
    fams = {f: lks.lks_kernel_time(solver.handle, f)
            for f in ("stencil_fwd", "couple", "recompute", "adj_cell", "adj_design", "adj_body", "stencil_adj",
                      "alks_body", "alks_stencil")}
    fams = {f: v for f, v in fams.items() if v[1] > 0}
    lks.lks_set_kernel_timing(solver.handle, False)
    return fams


def stencil_roofline(dev, peak: float, dim: int, n: tuple, name: str, n_steps: int = 20, every: int = 10) -> dict:
    """HBM roofline of the predictor and its transpose on a grid far larger than L2."""
    import torch
    from paper_2601_18272_gb300.lks import Solver
    P, g = _fluid_problem(dim, n, name, n_steps, every)
    S = Solver(P)
    gamma = torch.tensor(g, dtype=torch.float64, device=dev)
    grad = torch.empty_like(gamma)

    def run():
        S.forward(gamma)
        S.adjoint(1.0)
        S.sensitivity(grad)

    def run_paper():
        S.forward(gamma)
        S.adjoint_alks(1.0)
        S.sensitivity(grad)

    run()
    run_paper()
    torch.cuda.synchronize()
    fams = _family_times(S, run)
    fams.update({k: v for k, v in _family_times(S, run_paper).items() if k == "alks_stencil"})
    S.close()
    out = {"workload": name, "grid": list(n), "cells": P.n_cells, "dtype": "f32"}
    for fam in ("stencil_fwd", "stencil_adj", "alks_stencil"):
        ms, cnt = fams[fam]
        per = ms / 1000.0 / cnt
        alg = _alg_bytes(fam, P, 0, 4)
        out[fam] = {"achieved": alg / per / 1e9, "peak": peak, "unit": "GB/s", "frac": alg / per / 1e9 / peak,
                    "alg_bytes_per_launch": alg, "avg_launch_us": per * 1e6, "launches": cnt,
                    "cell_updates_per_s": P.n_cells / per}
    return out


def _timed(stream, flush, fn) -> float:
    """CUDA-event milliseconds of fn() on the stream, after an L2 flush."""
    import torch
    torch.cuda.synchronize()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1)


def _fwd_roofline(P, ms: float, peak: float) -> dict:
    """Forward-only throughput and its HBM fraction from the full-grid stencil bytes per cell-update
    (24 B in 2D, 32 B in 3D, FP32): what the march must move if nothing stays in L2."""
    bpc = 2 * (P.dim + 1) * 4
    value = P.n_cells * P.n_steps / (ms / 1000.0)
    return {"value": value, "unit": UNIT, "ms": ms, "bytes_per_cell_update": bpc,
            "hbm_frac": value * bpc / 1e9 / peak}


def gradient_throughput(dev, flush, peak: float, index: int, n_steps: int = 0, plain_steps: int = 0,
                        warm: bool = True) -> dict:
    """Whole-gradient and forward-only throughput of a workload (optionally truncated to n_steps): one
    timed gradient (after one warm-up gradient if warm), one timed forward, the kernel families of a
    gradient; with plain_steps, the plain FP64 store-all form on the first plain_steps steps and this
    form's gradient error against it there."""
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    from workloads import CKPT_STORE_ALL, config
    P, g = config(index)
    if n_steps:
        P = P.replace(n_steps=n_steps)
    gamma = torch.tensor(g, dtype=torch.float64, device=dev)
    grad = torch.empty_like(gamma)
    stream = torch.cuda.current_stream(dev)

    def run(S, out):
        S.forward(gamma)
        S.adjoint(1.0)
        S.sensitivity(out)

    S = Solver(P)
    if warm:
        run(S, grad)
    ms = _timed(stream, flush, lambda: run(S, grad))
    ms_fwd = _timed(stream, flush, lambda: S.forward(gamma))
    out = {"workload": P.name, "value": P.n_cells * P.n_steps / (ms / 1000.0), "unit": UNIT, "ms_per_gradient": ms,
           "n_steps": P.n_steps, "dtype": "f32",
           "checkpoints": _ckpt_desc(P, lks.lks_checkpoint_slots(S.handle)),
           "workspace_gb": lks.lks_workspace_bytes(S.handle) / 1e9,
           "persistent_coupling": lks.lks_persistent_coupling(S.handle, -1),
           "forward": _fwd_roofline(P, ms_fwd, peak)}
    if warm:
        fams = _family_times(S, lambda: run(S, grad))
        out["kernel_ms_per_gradient"] = {k: round(v[0], 3) for k, v in fams.items()}
    S.close()
    if plain_steps:
        Pp = P.replace(n_steps=plain_steps)
        S = Solver(Pp)
        g32 = torch.empty_like(gamma)
        run(S, g32)
        if not warm:
            fams = _family_times(S, lambda: run(S, g32))
            out["kernel_ms_first_steps"] = {"n_steps": plain_steps, **{k: round(v[0], 3) for k, v in fams.items()}}
        S.close()
        S = Solver(Pp, precision=64, ckpt_policy=CKPT_STORE_ALL)
        g64 = torch.empty_like(gamma)
        run(S, g64)
        ms64 = _timed(stream, flush, lambda: run(S, g64))
        out["plain_fp64_store_all"] = {"n_steps": plain_steps, "value": P.n_cells * plain_steps / (ms64 / 1000.0),
                                       "unit": UNIT, "ms_per_gradient": ms64,
                                       "workspace_gb": lks.lks_workspace_bytes(S.handle) / 1e9}
        out["dJdgamma_rel_l2_vs_fp64_first_steps"] = float(torch.linalg.norm(g32 - g64) / torch.linalg.norm(g64))
        S.close()
    return out


def _ckpt_desc(P, slots: int) -> str:
    fmt = {0: "fp32", 1: "bf16", 2: "fp16"}.get(P.ckpt_format, "?")
    if P.ckpt_policy == 2:
        budget = f" (as many as {P.hbm_budget_bytes / 1e9:.0f} GB hold)" if P.ckpt_every == 0 else ""
        return f"binomial, {slots} snapshots{budget}, {fmt}"
    if P.ckpt_policy == 0:
        return "every state stored"
    return f"uniform every {P.ckpt_every}, {fmt}"


def paper_adjoint_study(dev, flush) -> dict:
    """The paper's adjoint (ALKS, lks_adjoint_alks) beside the exact discrete adjoint. On the 512x256
    gradient workload: its time per gradient and its deviation from the exact gradient. On the 80x40
    translation workload and the two sensitivity checks of Appendix B (FP64): its deviation from the
    exact gradient and both against central differences along seeded random directions."""
    import numpy as np
    import torch
    from paper_2601_18272_gb300.lks import Solver
    from workloads import config, verification
    stream = torch.cuda.current_stream(dev)
    out = {}
    P, g = config(2)
    gamma = torch.tensor(g, dtype=torch.float64, device=dev)
    gex, gpa = torch.empty_like(gamma), torch.empty_like(gamma)
    S = Solver(P)

    def paper():
        S.forward(gamma)
        S.adjoint_alks(1.0)
        S.sensitivity(gpa)

    S.forward(gamma)
    S.adjoint(1.0)
    S.sensitivity(gex)
    paper()
    torch.cuda.synchronize()
    flush.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    paper()
    e1.record(stream)
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    fams = _family_times(S, paper)
    S.close()
    a, b = gex.cpu().numpy(), gpa.cpu().numpy()
    out[P.name] = {"ms_per_gradient": ms, "value": P.n_cells * P.n_steps / (ms / 1000.0), "unit": UNIT,
                   "kernel_ms_per_gradient": {k: round(v[0], 3) for k, v in fams.items()},
                   "launches_per_gradient": {k: v[1] for k, v in fams.items()},
                   "rel_l2_vs_exact": float(np.linalg.norm(b - a) / np.linalg.norm(a)),
                   "cosine_vs_exact": float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b)))}
    rng = np.random.default_rng(20260118)
    for (P, g), ndir in ((config(1), 3), (verification("translation"), 2), (verification("rotation"), 2)):
        S = Solver(P)
        gam = torch.tensor(g, dtype=torch.float64, device=dev)
        gex, gpa = torch.empty_like(gam), torch.empty_like(gam)
        S.forward(gam)
        S.adjoint(1.0)
        S.sensitivity(gex)
        S.adjoint_alks(1.0)
        S.sensitivity(gpa)
        torch.cuda.synchronize()
        a, b = gex.cpu().numpy(), gpa.cpu().numpy()
        h = 1e-5
        dirs = []
        for _ in range(ndir):
            v = rng.standard_normal(P.n_design)
            jp = S.forward(torch.tensor(g + h * v, dtype=torch.float64, device=dev))
            jm = S.forward(torch.tensor(g - h * v, dtype=torch.float64, device=dev))
            fd = (jp - jm) / (2 * h)
            dirs.append({"fd": fd, "exact": float(a @ v), "paper": float(b @ v)})
        S.close()
        out[P.name] = {"n_steps": P.n_steps, "rel_l2_vs_exact": float(np.linalg.norm(b - a) / np.linalg.norm(a)),
                       "cosine_vs_exact": float(a @ b / (np.linalg.norm(a) * np.linalg.norm(b))),
                       "exact_vs_fd_max_rel": max(abs(d["exact"] - d["fd"]) / abs(d["fd"]) for d in dirs),
                       "paper_vs_fd_max_rel": max(abs(d["paper"] - d["fd"]) / abs(d["fd"]) for d in dirs),
                       "directions": dirs}
    return out


def ckpt_precision_study(dev, n_steps: int = 0) -> dict:
    """Gradient error of FP32 / BF16 / FP16 checkpoints (FP32 fields, checkpoints every 100) on the
    1024x512 / 256x256 x-y-theta workload, at its full 20000 steps unless n_steps is given, against
    the FP64 form (FP64 fields and checkpoints every 100, which reproduces the FP64 store-all
    gradient to rounding and fits in memory at this length)."""
    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    from workloads import CKPT_BF16, CKPT_FP16, CKPT_FP32, CKPT_UNIFORM, config
    P, g = config(3)
    if n_steps:
        P = P.replace(n_steps=n_steps)
    gamma = torch.tensor(g, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)

    def grad(S):
        out = torch.empty_like(gamma)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        J = S.forward(gamma)
        S.adjoint(1.0)
        S.sensitivity(out)
        e1.record(stream)
        e1.synchronize()
        return J, out, e0.elapsed_time(e1)

    ref = Solver(P, precision=64, ckpt_policy=CKPT_UNIFORM, ckpt_every=100)
    J64, g64, ms64 = grad(ref)
    ref.close()
    out = {"workload": P.name, "n_steps": P.n_steps, "reference": "FP64 fields, FP64 checkpoints every 100",
           "reference_ms_per_gradient": ms64}
    for name, fmt in (("fp32", CKPT_FP32), ("bf16", CKPT_BF16), ("fp16", CKPT_FP16)):
        S = Solver(P, precision=32, ckpt_policy=CKPT_UNIFORM, ckpt_every=100, ckpt_format=fmt)
        J, d, ms = grad(S)  # one gradient each (graphs captured in its first segment)
        out[name] = {"dJdgamma_rel_l2": float(torch.linalg.norm(d - g64) / torch.linalg.norm(g64)),
                     "J_rel": abs(J - J64) / abs(J64), "ms_per_gradient": ms,
                     "workspace_gb": lks.lks_workspace_bytes(S.handle) / 1e9}
        S.close()
    return out


def run_reference(args, ws, rank):
    """The FP64 oracle on the host cores, each step a bounded sample of the same workload."""
    if rank != 0:
        return 0
    from oracle import oracle as O
    from workloads import config, initial_state
    P, g = config(CONFIG_INDEX)
    sample = args.ref_sample_steps
    p0, u0, s0 = initial_state(P)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        O.gradient(P, g, p0, u0, s0, n_steps=sample)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = P.n_cells * sample * len(times) / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * total / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": P.name, "grid": [P.nx, P.ny], "design": [P.ndx, P.ndy], "n_steps": P.n_steps,
                       "n_itr": P.n_itr, "sample_steps_per_bench_step": sample},
            "cpu_baseline": {"kind": "oracle", "value": value, "unit": UNIT, "cores": 1,
                             "sample": f"{sample} forward+adjoint time steps of the {P.name} workload per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def cpu_baseline(sample_steps: int):
    """The oracle (single-threaded FP64) on a bounded sample of the benchmark workload, and its OpenMP
    timing build (the same arithmetic over all host cores) on the same sample."""
    from oracle import oracle as O
    from workloads import config, initial_state
    P, g = config(CONFIG_INDEX)
    p0, u0, s0 = initial_state(P)
    t0 = time.perf_counter()
    O.gradient(P, g, p0, u0, s0, n_steps=sample_steps)
    dt = time.perf_counter() - t0
    out = {"value": P.n_cells * sample_steps / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"forward+adjoint of the first {sample_steps} of {P.n_steps} time steps of {P.name}, "
                     f"single-threaded FP64 ({dt:.1f} s)"}
    try:
        if O.set_variant("openmp"):
            t0 = time.perf_counter()
            O.gradient(P, g, p0, u0, s0, n_steps=sample_steps)
            dto = time.perf_counter() - t0
            out["openmp"] = {"value": P.n_cells * sample_steps / dto, "unit": UNIT, "cores": O.threads(),
                             "nproc": os.cpu_count(), "sample": "the same sample; per-node loops over all cores, "
                             "design-point scatter and reductions serial (results bitwise the single-threaded "
                             f"oracle's) ({dto:.1f} s)"}
        else:
            out["openmp"] = {"unavailable": "the host compiler built no OpenMP variant"}
    finally:
        O.set_variant("serial")
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--ref-sample-steps", type=int, default=8)
    ap.add_argument("--cpu-sample-steps", type=int, default=24)
    ap.add_argument("--skip-extras", action="store_true", help="only the timed region and e2e")
    ap.add_argument("--time-steps", type=int, default=0,
                    help="truncate N_t (profiling runs only: keeps the per-step kernel mix, shrinks the launch list)")
    ap.add_argument("--config", type=int, default=0,
                    help="profiling runs with --case gradient or alks: the workload index (default: the benchmark's)")
    ap.add_argument("--case", choices=["fluid2d", "fluid3d", "alks", "gradient"], default=None,
                    help="profiling runs only: the stencil roofline of a fluid grid (--grid NXxNY[xNZ]) alone")
    ap.add_argument("--grid", default=None)
    ap.add_argument("--case-steps", type=int, default=4)
    args = ap.parse_args()
    ws, rank, local = _dist()
    if args.impl == "reference":
        return run_reference(args, ws, rank)
    if args.case in ("alks", "gradient"):  # profiling runs only: gradients (exact or the paper's adjoint)
        import torch
        from paper_2601_18272_gb300.lks import Solver
        from workloads import config
        torch.cuda.set_device(local)
        P, g = config(args.config or CONFIG_INDEX)
        if args.time_steps:
            P = P.replace(n_steps=args.time_steps, ckpt_every=min(P.ckpt_every, max(1, args.time_steps // 2)))
        S = Solver(P)
        gamma = torch.tensor(g, dtype=torch.float64, device=torch.device("cuda", local))
        grad = torch.empty_like(gamma)
        for _ in range(args.warmup + args.steps):
            J = S.forward(gamma)
            (S.adjoint_alks if args.case == "alks" else S.adjoint)(1.0)
            S.sensitivity(grad)
        torch.cuda.synchronize()
        S.close()
        print(json.dumps({"case": args.case, "workload": P.name, "n_steps": P.n_steps, "J": J}), flush=True)
        return 0
    if args.case:
        import torch
        torch.cuda.set_device(local)
        dim = 2 if args.case == "fluid2d" else 3
        n = tuple(int(v) for v in (args.grid or ("4096x4096" if dim == 2 else "256x256x256")).split("x"))
        name = f"{args.case}_{'x'.join(map(str, n))}"
        out = stencil_roofline(torch.device("cuda", local), _peaks()[0], dim, n, name, args.case_steps,
                               max(1, args.case_steps // 2))
        print(json.dumps(out), flush=True)
        return 0

    import torch
    from paper_2601_18272_gb300 import lks
    from paper_2601_18272_gb300.lks import Solver
    from workloads import CKPT_STORE_ALL, config

    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    P, g = config(CONFIG_INDEX)
    if args.time_steps:
        P = P.replace(n_steps=args.time_steps, ckpt_every=min(P.ckpt_every, max(1, args.time_steps // 2)))
    solver = Solver(P)
    gamma = torch.tensor(g, dtype=torch.float64, device=dev)
    grad = torch.empty_like(gamma)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 129 MB L2
    stream = torch.cuda.current_stream(dev)

    def step():
        solver.forward(gamma)
        solver.adjoint(1.0)
        solver.sensitivity(grad)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local)
    sampler.start()
    l0 = solver.launches()
    ms = []
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms, all_launches = replica_totals(sum(ms), solver.launches() - l0, dist, dev)
    cell_steps = P.n_cells * P.n_steps
    value = ws * args.steps * cell_steps / (total_ms / 1000.0)

    # end to end: host gamma (pinned) -> device, forward, adjoint, sensitivity, gradient -> host
    g_host = torch.tensor(g, dtype=torch.float64).pin_memory()
    d_host = torch.empty(P.n_design, dtype=torch.float64).pin_memory()
    gptr, dptr = g_host.numpy(), d_host.numpy()
    solver.gradient_host(gptr)  # warm
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        J = lks.lks_gradient_host(solver.handle, gptr, dptr, stream.cuda_stream)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e_s, _ = replica_totals(e2e_s, 0, dist, dev)
    e2e_value = ws * args.steps * cell_steps / e2e_s

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": P.name, "grid": [P.nx, P.ny], "design": [P.ndx, P.ndy], "velocity_set": "D2Q9",
                       "n_steps": P.n_steps, "n_itr": P.n_itr, "motion": "rotation about the body centre",
                       "fields": "fp32 (force/torque/EOM fp64)", "checkpoints": f"uniform every {P.ckpt_every}, fp32",
                       "l2": "flushed (256 MB write) between timed steps", "replicas": ws},
            "clocks": clocks,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * P.n_design,
                    "d2h_bytes_per_step": 8 * P.n_design + 8, "J": J},
            "gpu_launches": all_launches}

    if rank == 0 and not args.skip_extras:
        # dominant kernel: one more gradient with every launch bracketed by CUDA events
        fams = _family_times(solver, step)
        dom = max(fams, key=lambda k: fams[k][0])
        dom_ms, dom_n = fams[dom]
        peak, peak_kind = _peaks()
        per_launch_s = dom_ms / 1000.0 / dom_n
        persistent = lks.lks_persistent_coupling(solver.handle, -1)
        alg = _alg_bytes(dom, P, _box_cells(P), 4, persistent)
        achieved = alg / per_launch_s / 1e9
        line["roofline"] = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                            "frac": achieved / peak, "traffic": _traffic(P.name, dom), "peak_source": peak_kind,
                            "alg_bytes_per_launch": alg, "avg_launch_us": per_launch_s * 1e6,
                            "persistent_coupling": persistent,
                            "kernel_ms_per_gradient": {k: round(v[0], 3) for k, v in fams.items()},
                            "launches_per_gradient": {k: v[1] for k, v in fams.items()}}
        # forward-only throughput of this workload (the march alone, lks_forward)
        ms_fwd = _timed(stream, flush, lambda: solver.forward(gamma))
        line["roofline"]["forward_only"] = {P.name: _fwd_roofline(P, ms_fwd, peak)}
        # the gradient in autograd form: LKSObjective.apply(gamma, solver).backward() (the backward
        # reads the incoming gradient on the host: one synchronisation, as lks_forward already has)
        from paper_2601_18272_gb300.autograd import objective
        gam_ag = gamma.clone().requires_grad_(True)
        def ag():
            gam_ag.grad = None
            objective(gam_ag, solver).backward()
        ag()
        ag_ms = [_timed(stream, flush, ag) for _ in range(3)]
        line["e2e"]["autograd"] = {"ms_per_gradient": float(np.median(ag_ms)),
                                   "value": cell_steps / (float(np.median(ag_ms)) / 1000.0), "unit": UNIT,
                                   "form": "LKSObjective.apply(gamma, solver).backward()",
                                   "max_abs_diff_vs_raw_calls": float((gam_ag.grad - grad).abs().max())}
        # accuracy of this FP32 checkpointed gradient against the FP64 store-all GPU form, and the
        # throughput of that plain FP64 form
        plain = Solver(P, precision=64, ckpt_policy=CKPT_STORE_ALL)
        g64 = torch.empty_like(gamma)
        plain.forward(gamma)
        plain.adjoint(1.0)
        plain.sensitivity(g64)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        J64 = plain.forward(gamma)
        plain.adjoint(1.0)
        plain.sensitivity(g64)
        e1.record(stream)
        e1.synchronize()
        plain_ms = e0.elapsed_time(e1)
        step()
        torch.cuda.synchronize()
        rel = float(torch.linalg.norm(grad - g64) / torch.linalg.norm(g64))
        line["gradient_rel_err_vs_fp64"] = {"dJdgamma_rel_l2": rel, "J_rel": abs(J - J64) / abs(J64),
                                            "reference": "FP64 store-all GPU form"}
        line["plain_fp64_store_all"] = {"value": cell_steps / (plain_ms / 1000.0), "unit": UNIT,
                                        "ms_per_step": plain_ms, "workspace_gb": lks.lks_workspace_bytes(plain.handle) / 1e9}
        line["workspace_gb"] = lks.lks_workspace_bytes(solver.handle) / 1e9
        plain.close()
        # the full-grid kernels on grids far larger than L2, and the 3D workloads
        line["stencil_roofline_2d"] = stencil_roofline(dev, peak, 2, (8192, 4096), "fluid2d_8192x4096")
        line["stencil_roofline_3d"] = stencil_roofline(dev, peak, 3, (512, 256, 256), "fluid3d_512x256x256")
        line["body3d"] = gradient_throughput(dev, flush, peak, 4)
        # the largest workload at its full 10000 steps: one timed gradient (graphs captured in its
        # first segment) and one timed forward; the plain FP64 store-all form does not fit at this
        # length (1.3 TB), so it is compared on the first 50 steps
        line["turbine3d_6dof"] = gradient_throughput(dev, flush, peak, 5, plain_steps=50, warm=False)
        line["ckpt_precision"] = ckpt_precision_study(dev)
        line["paper_adjoint"] = paper_adjoint_study(dev, flush)
        line["cpu_baseline"] = cpu_baseline(args.cpu_sample_steps)
        # short copies that keep the large-grid fractions and the other workloads' throughput with
        # the roofline record
        sr2, sr3 = line["stencil_roofline_2d"], line["stencil_roofline_3d"]
        line["roofline"]["stencil_frac"] = {"2d_fwd": sr2["stencil_fwd"]["frac"], "2d_adj": sr2["stencil_adj"]["frac"],
                                            "3d_fwd": sr3["stencil_fwd"]["frac"], "3d_adj": sr3["stencil_adj"]["frac"],
                                            "grids": ["8192x4096", "512x256x256"]}
        for key in ("body3d", "turbine3d_6dof"):
            w = line[key]
            line["roofline"]["forward_only"][w["workload"]] = w["forward"]
            line["roofline"].setdefault("gradient", {})[w["workload"]] = {
                "n_steps": w["n_steps"], "ms": w["ms_per_gradient"], "value": w["value"]}
        cp = line["ckpt_precision"]
        line["roofline"]["ckpt_precision"] = {"n_steps": cp["n_steps"],
                                              **{k: cp[k]["dJdgamma_rel_l2"] for k in ("fp32", "bf16", "fp16")}}
    solver.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
