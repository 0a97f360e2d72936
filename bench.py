#!/usr/bin/env python
"""Benchmark of the C-AMS hot path on one GB300 (replicas on N GPUs).

One step = one pass of the whole hot path over one synthetic permeability
field: static transmissibilities (cams_set_permeability), then one implicit
time step (cams_solve): linear-system population, full basis construction,
R A P and its factorisation, ILU(0) factorisation and the C-AMS inner loop,
inside the Newton loop, to the workload's tolerance.

Metric: fine-cell C-AMS iterations per second (N_f x C-AMS iterations / wall
time), with the Newton-step wall time reported beside it.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl cams|reference]
"""
import os

# the CPU oracle (reference arm and cpu_baseline) runs single-threaded, as
# the paper's implementation did
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import argparse
import json
import math
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import WORKLOADS, ensemble_members, make_inputs, line_columns  # noqa: E402

METRIC = ("Newton-step wall time & fine-cell·iters/s to 1e-8 residual; "
          "learned/FP32 vs FP64 C-AMS")
UNIT = "fine-cell·iters/s"
DEFAULT_WORKLOAD = "3d-200x200x100-mixed"
ENSEMBLE = "ensemble-64"
LEARNED_GATE = 0.5      # gate of the learned-surrogate leg: strict enough to keep the C-AMS count
LEARNED_TIGHT_TOL = 1e-9   # the learned leg again at this tolerance (pressure within 1e-6)
REFERENCE_TOL = 1e-11      # tolerance of the converged FP64 reference pressure

# Algorithmic bytes per fine cell of each kernel class (FP64): every operand
# array read once and every result written once (neighbour re-reads served
# on chip); the sentinel re-marks of the wavefront schedule are bookkeeping
# and not counted.
BYTES_PER_CELL = {
    "assemble": 16 + 104,      # density: p -> rho; assembly: p, rho, rho_n, T x3 -> A x4, C, f, eps
    "residual": 56,            # A x4, f, p -> r
    "restrict": 72,            # P x8, r
    "prolong": 80,             # P x8, p read + write
    "ilu_resid": 64,           # A x4, f, p, 1/d -> D^{-1}(f - A p)
    "ilu_fwd": 40,             # D^{-1} r, scaled lower couplings x3 -> w
    "ilu_bwd": 40,             # w, scaled upper couplings x3 -> z
    "ilu_apply": 24,           # z, p read + write
    "galerkin": 96,            # P x8, couplings x3, C
    "ilu_factor": 88,          # A x4 -> 1/d, scaled couplings x6
    "basis_op": 64,
}
# Latency model of a wavefront sweep: its last cell is (nx + ny + nz - 3)
# dependent steps after its first, so no schedule finishes before that many
# steps of one tile's step loop.  T_STEP_US: a tile's time per step alone
# (no neighbour to wait for), measured on this GPU with a lone 8 x 4-row
# tile of 65,536 x-positions (one group of 4 steps: 0.30 us in FP32,
# 0.78 us in FP64).
T_STEP_US = {0: 0.78 / 4, 1: 0.30 / 4}
SWEEP_CLASSES = ("ilu_fwd", "ilu_bwd")

# DRAM bytes per launch measured by ncu (dram__bytes_read.sum + write.sum) for
# a kernel class on a workload, for the kernels as they stand; see profiles/.
MEASURED_TRAFFIC = {
    # profiles/launch_list_3d-200x200x100-mixed.md (the kernels as of the FP32 residual copy)
    ("3d-200x200x100-mixed", "ilu_fwd"): 73.9e6,
    ("3d-200x200x100-mixed", "ilu_bwd"): 70.1e6,
    ("3d-200x200x100-mixed", "ilu_resid"): 121.9e6,
    ("3d-200x200x100-mixed", "ilu_apply"): 32.8e6,
}

# the same classes with the FP32 preconditioner (4-byte operands; r and p stay FP64)
BYTES_PER_CELL_MIXED = dict(BYTES_PER_CELL, **{
    "residual": 60,            # A x4, f, p -> r (FP64) and its FP32 copy
    "restrict": 36,            # P x8, r (FP32)
    "prolong": 36,             # P x8 -> delta (FP32)
    "ilu_resid": 32,           # A x4, delta, 1/d, r (FP32) -> D^{-1}(r - A delta)
    "ilu_fwd": 20,             # FP32 forward sweep
    "ilu_bwd": 20,             # FP32 backward sweep
    "ilu_apply": 12,           # delta += z (FP32)
    "update": 20,              # p (FP64) += delta (FP32)
    "galerkin": 64,            # P x8 (FP32), couplings x3, C
    "ilu_factor": 108,         # A (FP64) -> A (FP32); pivots and scaled couplings in FP32
})


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cams", choices=["cams", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD,
                    choices=sorted(WORKLOADS) + [ENSEMBLE])
    ap.add_argument("--workers", type=int, default=0,
                    help="host threads of the ensemble (0: min(16, CPU count))")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-baseline", action="store_true", help="skip the cpu_baseline leg")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the leg with the learned basis surrogate")
    ap.add_argument("--no-fp64", action="store_true",
                    help="mixed-precision workloads: skip the FP64 comparison run")
    ap.add_argument("--jacobian", action="store_true",
                    help="the full-Jacobian Newton step (flux density differentiated)")
    ap.add_argument("--cf", action="store_true",
                    help="correction functions before every multiscale stage")
    ap.add_argument("--oracle-newton-step", action="store_true",
                    help="with --impl reference: time the oracle on the whole workload for "
                         "its first Newton step, stage by stage (minutes to an hour)")
    ap.add_argument("--restriction", type=int, choices=[0, 1, 2], default=None,
                    help="override the workload's restriction: 0 MSFE, 1 MSFV, "
                         "2 MSFE then a closing MSFV correction")
    return ap.parse_args()


VARIANT = {}      # solver options beyond the workload's (--jacobian, --cf)


def variant_suffix():
    return ((" full-Jacobian Newton" if VARIANT.get("jacobian") else "")
            + (" correction functions" if VARIANT.get("cf") else ""))


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


# --------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *a):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                self.out, _ = self.proc.communicate()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in (self.out or "").splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1])); mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)),
                "reasons": sorted(reasons), "samples": len(sm)}


def class_rooflines(prof, n_cells, precision, peak):
    """Achieved algorithmic GB/s and the fraction of the HBM peak of every
    kernel class with a byte count, from the live per-class profile
    {class: (launch groups, total ms, kernels)}: bytes per cell x cells per
    launch group / average group time."""
    table = BYTES_PER_CELL_MIXED if precision else BYTES_PER_CELL
    out = {}
    for k, (n_l, ms_tot, _) in prof.items():
        if k not in table or n_l <= 0 or ms_tot <= 0.0:
            continue
        avg_ms = ms_tot / n_l
        gbs = table[k] * n_cells / (avg_ms / 1e3) / 1e9
        out[k] = {"launches": int(n_l), "avg_ms": avg_ms, "gbs": gbs, "frac": gbs / peak}
    return out


def sweep_latency_bound(prof, w):
    """The ILU(0) sweeps against their critical path: (nx + ny + nz - 3)
    steps at a lone tile's step time (a bound no schedule of the exact
    lexicographic recurrence beats at that step time)."""
    steps = w.nx + w.ny + w.nz - 3
    bound_us = steps * T_STEP_US[1 if w.precision else 0]
    out = {"model": "(nx+ny+nz-3) dependent steps x t_step of a lone tile",
           "t_step_us": T_STEP_US[1 if w.precision else 0], "steps": steps,
           "bound_us": bound_us}
    for k in SWEEP_CLASSES:
        if k in prof and prof[k][0]:
            avg_us = 1e3 * prof[k][1] / prof[k][0]
            out[k] = {"avg_launch_us": avg_us, "frac": bound_us / avg_us}
    return out


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


# ------------------------------------------------------------ cams arm --

def aggregate_replicas(t_ms, units, world, device=None):
    """Replicas only: every rank solves its own field with no data exchange.
    The job's time is the slowest rank's and its work is the sum over ranks
    (the one collective here is for the measurement, not the data path)."""
    if world <= 1:
        return float(t_ms), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(t_ms)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())



def _handles(cams, w, inp, memspace, dev_arrays=None):
    grid = cams.cams_grid(w.nx, w.ny, w.nz, inp["dx"], inp["dy"], inp["dz"])
    fluid = cams.cams_fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi)
    opt = cams.make_options(w.coarse, basis=w.basis, restriction=w.restriction, n_pre=w.n_pre,
                            n_post=w.n_post, lin_rtol=w.lin_rtol, nl_tol=w.nl_tol,
                            adapt_theta=w.adapt_theta, max_newton=w.max_newton,
                            max_cams=w.max_cams, memspace=memspace, precision=w.precision,
                            **VARIANT)
    k = dev_arrays if dev_arrays is not None else (inp["kx"], inp["ky"], inp["kz"])
    return cams.cams_setup(grid, fluid, opt, *k)


def converged_reference(args, w, local_rank):
    """The step solved by the FP64 engine to a 1e-11 relative ||eps|| (untimed):
    the pressure every leg's error is measured against."""
    import torch
    from paper_1705_05783_gb300 import cams
    torch.cuda.set_device(local_rank)
    wr = w.with_(precision=0, nl_tol=REFERENCE_TOL)
    inp = make_inputs(wr, args.seed)
    h = _handles(cams, wr, inp, cams.CAMS_HOST)
    try:
        bc, keep = cams.make_bc(inp["dirichlet"], wr.p_west, wr.p_east,
                                inp["src_cell"] if len(inp["src_cell"]) else None,
                                inp["src_rate"] if len(inp["src_rate"]) else None,
                                inp["fix_cell"] if len(inp["fix_cell"]) else None,
                                inp["fix_value"] if len(inp["fix_value"]) else None)
        p = inp["p0"].copy()
        cams.cams_solve(h, inp["p0"], inp["dt"], bc, p)
    finally:
        cams.cams_destroy(h)
    return p


def rel_linf(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def run_cams(args, w, rank, world, local_rank, e2e_leg=True, surrogate=None):
    """surrogate: (parameters, gate tolerance) to build the interiors with the
    learned surrogate, or None for the exact local solves."""
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_1705_05783_gb300 import cams

    inp = make_inputs(w, args.seed)
    N = w.n_cells
    # inputs resident in HBM for the device-timed value
    dk = [torch.from_numpy(inp[k]).to(dev) for k in ("kx", "ky", "kz")]
    p0 = torch.from_numpy(inp["p0"]).to(dev)
    p = torch.empty_like(p0)
    src = None
    if len(inp["src_cell"]):
        src = (torch.from_numpy(inp["src_cell"].astype(np.int32)).to(dev),
               torch.from_numpy(inp["src_rate"]).to(dev))
    fix = None
    if len(inp["fix_cell"]):
        fix = (torch.from_numpy(inp["fix_cell"].astype(np.int32)).to(dev),
               torch.from_numpy(inp["fix_value"]).to(dev))
    bc, keep = cams.make_bc(inp["dirichlet"], w.p_west, w.p_east,
                            src[0] if src else None, src[1] if src else None,
                            fix[0] if fix else None, fix[1] if fix else None)
    stream = torch.cuda.current_stream(dev)
    h = _handles(cams, w, inp, cams.CAMS_DEVICE, dk)
    if surrogate is not None:
        cams.cams_set_surrogate(h, surrogate[0], surrogate[1])
    cams.cams_set_stream(h, stream.cuda_stream)

    def step():
        cams.cams_set_permeability(h, *dk)
        p.copy_(p0)
        return cams.cams_solve(h, p0, inp["dt"], bc, p)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # L2 is 129 MB; every step streams > 1 GB of fields (4M cells x 8 B x
    # ~40 arrays), so the inputs of one iteration never stay L2-resident.
    # The timed steps run as the library ships: the C-AMS iteration replayed
    # as a captured CUDA graph, no per-class events.
    l0 = cams.launches(h)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    stats = []
    with ClockSampler(local_rank) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            st = step()
            stats.append((st.newton_its, st.cams_its, st.t_assemble, st.t_precond, st.t_iterate))
        ev1.record(stream)
        torch.cuda.synchronize()
    launches = cams.launches(h) - l0
    # the per-kernel-class breakdown in a separate pass of the same steps:
    # CUDA events on the handle's stream bracket every class (direct launches)
    prof_steps = max(1, min(args.steps, 3))
    cams.cams_profile(h, True)
    for _ in range(prof_steps):
        step()
    torch.cuda.synchronize()
    prof = cams.profile_table(h)
    cams.cams_profile(h, False)
    prof = {k: (v[0] * args.steps / prof_steps, v[1] * args.steps / prof_steps, v[2])
            for k, v in prof.items()}
    newton = sum(s[0] for s in stats)
    its = sum(s[1] for s in stats)
    t_ms, units = aggregate_replicas(ev0.elapsed_time(ev1), N * its, world, dev)
    value = units / (t_ms / 1e3)

    # dominant kernel class by time, with its live per-launch duration
    dom = max((k for k in prof if prof[k][0] > 0 and k in BYTES_PER_CELL), key=lambda k: prof[k][1])
    n_l, ms_tot, _ = prof[dom]
    avg_ms = ms_tot / n_l
    peak, peak_kind = measured_peaks()
    bytes_per_launch = (BYTES_PER_CELL_MIXED if w.precision else BYTES_PER_CELL)[dom] * N
    achieved = bytes_per_launch / (avg_ms / 1e3) / 1e9

    p_final = p.cpu().numpy()
    surr = None
    if surrogate is not None:
        sizes = cams.cams_get_int(h, cams.CAMS_Q_SIZES, np.zeros(8, np.int32))
        surr = {"interiors_supplied": int(sizes[7]), "gate_tol": float(surrogate[1])}
    if not e2e_leg:
        cams.cams_destroy(h)
        return {"value": value, "unit": UNIT, "ms_per_step": t_ms / args.steps, "surrogate": surr,
                "dtype": "f32+f64" if w.precision else "f64",
                "newton_its_per_step": newton / args.steps, "cams_its_per_step": its / args.steps,
                "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items() if v[0]},
                "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                             "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                             "bytes_per_launch": bytes_per_launch, "avg_launch_ms": avg_ms},
                "_p": p_final}

    # end to end through the C-ABI with HOST buffers (copies inside the timed region)
    h_host = _handles(cams, w, inp, cams.CAMS_HOST)
    if surrogate is not None:
        cams.cams_set_surrogate(h_host, surrogate[0], surrogate[1])
    bch, keeph = cams.make_bc(inp["dirichlet"], w.p_west, w.p_east,
                              inp["src_cell"] if len(inp["src_cell"]) else None,
                              inp["src_rate"] if len(inp["src_rate"]) else None,
                              inp["fix_cell"] if len(inp["fix_cell"]) else None,
                              inp["fix_value"] if len(inp["fix_value"]) else None)
    ph = np.empty(N)
    for _ in range(1):
        cams.cams_set_permeability(h_host, inp["kx"], inp["ky"], inp["kz"])
        ph[:] = inp["p0"]
        cams.cams_solve(h_host, inp["p0"], inp["dt"], bch, ph)
    t0 = time.perf_counter()
    e_its = 0
    for _ in range(args.steps):
        cams.cams_set_permeability(h_host, inp["kx"], inp["ky"], inp["kz"])
        ph[:] = inp["p0"]
        st = cams.cams_solve(h_host, inp["p0"], inp["dt"], bch, ph)
        e_its += st.cams_its
    e_s = time.perf_counter() - t0
    cams.cams_destroy(h_host)
    cams.cams_destroy(h)
    e2e = {"value": N * e_its * world / e_s, "unit": UNIT,
           "h2d_bytes_per_step": int(8 * N * 5 + 12 * len(inp["src_cell"])),
           "d2h_bytes_per_step": int(8 * N)}

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64" if w.precision else "f64",
        "data": "synthetic",
        "config": {"workload": f"{w.name} {'mixed FP32/FP64' if w.precision else 'FP64'} C-AMS basis B{w.basis} "
                               f"{('MSFE', 'MSFV', 'MSFE+closing MSFV')[w.restriction]} n_post={w.n_post} "
                               f"coarse {w.coarse[0]}x{w.coarse[1]}x{w.coarse[2]} tol {w.nl_tol:g}"
                               + variant_suffix(),
                   "cells": N, "time_step": "first (full basis build) from p=0",
                   "l2": "inputs > L2 (4M-cell fields, >1 GB touched per step)",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "newton_step_ms": t_ms / max(newton, 1),
        "newton_its_per_step": newton / args.steps, "cams_its_per_step": its / args.steps,
        "stage_ms_per_step": {"assemble": sum(s[2] for s in stats) / args.steps,
                              "precond_update": sum(s[3] for s in stats) / args.steps,
                              "iterate": sum(s[4] for s in stats) / args.steps},
        "kernel_ms_per_step": {k: v[1] / args.steps for k, v in prof.items() if v[0]},
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_source": peak_kind,
                     "traffic": MEASURED_TRAFFIC.get((w.name, dom)),
                     "bytes_per_launch": bytes_per_launch,
                     "avg_launch_ms": avg_ms,
                     "timing": "CUDA events per kernel class on the handle's stream, in a "
                               "separate pass of the same steps after the timed region"},
        "kernel_roofline": class_rooflines(prof, N, w.precision, peak),
        "latency_bound": sweep_latency_bound(prof, w),
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "_p": p_final,
    }
    return out


# ------------------------------------------------------------ ensemble --

def run_ensemble(args, rank, world, local_rank):
    """64 independent realisations (sigma in [1, 4], 32^3 .. 128x128x64,
    mixed precision), one implicit step each: all members concurrently
    through cams_ensemble_solve, against the same members one at a time."""
    import torch
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    from paper_1705_05783_gb300 import cams

    members = ensemble_members(64, seed=args.seed)
    workers = args.workers or min(16, os.cpu_count() or 1)
    hs, bcs, keep, dks, p0s, ps, dts, cells = [], [], [], [], [], [], [], []
    for w in members:
        inp = make_inputs(w)
        dk = [torch.from_numpy(inp[k]).to(dev) for k in ("kx", "ky", "kz")]
        hs.append(_handles(cams, w, inp, cams.CAMS_DEVICE, dk))
        bc, kp = cams.make_bc(inp["dirichlet"], w.p_west, w.p_east)
        bcs.append(bc); keep.append(kp); dks.append(dk)
        p0 = torch.from_numpy(inp["p0"]).to(dev)
        p0s.append(p0); ps.append(torch.empty_like(p0)); dts.append(inp["dt"])
        cells.append(w.n_cells)

    def reset():
        for h, dk, p, p0 in zip(hs, dks, ps, p0s):
            cams.cams_set_permeability(h, *dk)
            p.copy_(p0)
        torch.cuda.synchronize()

    def ensemble():
        reset()
        status, st = cams.cams_ensemble_solve(hs, p0s, dts, bcs, ps, workers)
        if any(s != cams.CAMS_OK for s in status):
            raise RuntimeError(f"ensemble member failed: {status}")
        return st

    def sequential():
        reset()
        return [cams.cams_solve(h, p0, dt, bc, p) for h, p0, dt, bc, p in zip(hs, p0s, dts, bcs, ps)]

    def timed(fn):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        l0 = cams.launches(hs[0])
        per, units = [], 0.0
        with ClockSampler(local_rank) as clk:
            t0 = time.perf_counter()
            for _ in range(args.steps):
                st = fn()
                per += [s.t_total for s in st]
                units += sum(n * s.cams_its for n, s in zip(cells, st))
            torch.cuda.synchronize()
            t_ms = (time.perf_counter() - t0) * 1e3
        t_ms, units = aggregate_replicas(t_ms, units, world, dev)
        return {"value": units / (t_ms / 1e3), "ms_per_step": t_ms / args.steps,
                "per_solve_ms": {"p50": float(np.percentile(per, 50)),
                                 "p99": float(np.percentile(per, 99))},
                "gpu_launches": int(cams.launches(hs[0]) - l0), "clocks": clk.summary(),
                "cams_its_per_step": sum(s.cams_its for s in st)}

    out = {}
    results = {}
    for name, fn in (("sequential", sequential), ("ensemble", ensemble)):
        out[name] = timed(fn)
        results[name] = [p.cpu().numpy() for p in ps]
    same = all(np.array_equal(a, b) for a, b in zip(results["sequential"], results["ensemble"]))
    # the schedule autotuner, in the regime the ensemble runs in: whole
    # ensemble steps timed under each candidate schedule (members run
    # concurrently; a schedule timed on one member alone is not a guide)
    from paper_1705_05783_gb300 import autotune
    t0 = time.perf_counter()
    choice, cand_s = autotune.tune_ensemble(hs, ensemble, repeats=2)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0
    out["tuned"] = timed(ensemble)
    tuned_same = all(np.array_equal(p.cpu().numpy(), b) for p, b in zip(ps, results["ensemble"]))
    for h in hs:
        cams.cams_destroy(h)
    ens, seq, tun = out["ensemble"], out["sequential"], out["tuned"]
    return {"metric": "ensemble fine-cell·iters/s, one implicit step of 64 realisations",
            "value": tun["value"], "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": tun["ms_per_step"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{ENSEMBLE}: 64 seeded realisations, sigma U(1,4), grids "
                       "32^3 .. 128x128x64, coarse 8^3, (B4) MSFE, 5 ILU post, tol 1e-8, mixed "
                       "precision", "members": len(hs), "cells": int(sum(cells)),
                       "workers": workers,
                       "l2": "members' fields total > 10 GB; every step streams from HBM"},
            "per_solve_ms": tun["per_solve_ms"], "gpu_launches": tun["gpu_launches"],
            "clocks": tun["clocks"], "cams_its_per_step": tun["cams_its_per_step"],
            "untuned": ens, "sequential": seq,
            "speedup_vs_sequential": seq["ms_per_step"] / tun["ms_per_step"],
            "autotune": {"seconds": tune_s, "choice": list(choice) if choice else None,
                         "candidate_s": {f"{a},{b}": v for (a, b), v in cand_s.items()},
                         "schedule": "(ilu_cta: 0 = one 8x4-row tile per warp, 1 = 2x2 tiles "
                                     "per CTA; coarse_cluster: 0 = one CTA, 1 = cluster)",
                         "results_unchanged": bool(tuned_same)},
            "bitwise_equal_to_sequential": bool(same)}


# ---------------------------------------------------- oracle (CPU) legs --

def _oracle_problem(w, inp, nx, ny, nz):
    """The oracle's Problem and Options for the (nx, ny, nz) corner box of
    workload w's seeded field (the whole field when the sizes are w's)."""
    import oracle
    kx = inp["kx"].reshape(w.nz, w.ny, w.nx)[:nz, :ny, :nx].ravel().copy()
    ky = inp["ky"].reshape(w.nz, w.ny, w.nx)[:nz, :ny, :nx].ravel().copy()
    kz = inp["kz"].reshape(w.nz, w.ny, w.nx)[:nz, :ny, :nx].ravel().copy()
    g = oracle.Grid(nx, ny, nz, inp["dx"], inp["dy"], inp["dz"])
    if w.bc == "lines":
        # the two prescribed columns at the box's own corners
        fc, fv = line_columns(w.with_(nx=nx, ny=ny, nz=nz))
        bc = oracle.BC(False, w.p_west, w.p_east, fix_cell=fc, fix_value=fv)
    elif w.bc == "wells" and (nx, ny, nz) == (w.nx, w.ny, w.nz):
        bc = oracle.BC(inp["dirichlet"], w.p_west, w.p_east, inp["src_cell"], inp["src_rate"],
                       inp["fix_cell"], inp["fix_value"])
    else:
        bc = oracle.BC(True, w.p_west, w.p_east)
    pb = oracle.Problem.build(g, oracle.Fluid(w.law, w.c_or_eta, w.rho0, w.mu, w.phi),
                              bc, kx, ky, kz)
    opt = oracle.Options(coarse=w.coarse, basis=w.basis, restriction=w.restriction,
                         n_pre=w.n_pre, n_post=w.n_post, lin_rtol=w.lin_rtol, nl_tol=w.nl_tol,
                         adapt_theta=w.adapt_theta, max_newton=w.max_newton, max_cams=w.max_cams,
                         full_jacobian=bool(VARIANT.get("jacobian")), cf=bool(VARIANT.get("cf")))
    return pb, opt


def oracle_sample(w, seed, sub=(60, 60, 40), inp=None):
    """A bounded sample of workload w for the CPU oracle: the (sub) corner
    box of the same seeded field, same coarsening, fluid, time step and
    solver options, one implicit step."""
    import oracle
    if inp is None:
        inp = make_inputs(w, seed)
    # each side a whole number of coarse blocks, within the grid
    nx, ny, nz = (min(n, max(2 * b, (s // b) * b))
                  for n, b, s in zip((w.nx, w.ny, w.nz), w.coarse, sub))
    pb, opt = _oracle_problem(w, inp, nx, ny, nz)
    t0 = time.perf_counter()
    _, st = oracle.run(pb, opt, np.zeros(pb.grid.N), inp["dt"], 1)
    dt = time.perf_counter() - t0
    return pb.grid.N * st[0].cams_its / dt, dt, st[0], f"{nx}x{ny}x{nz} corner box of the {w.name} field"


def oracle_newton_step(w, seed):
    """The oracle on the whole workload for its first Newton step, stage by
    stage (Table 1: assembly, ILU(0) factors, basis, R A P and its factor,
    then C-AMS iterations to the inner stopping test of Sec. 4.1.1); the
    wall time of each stage on one host core."""
    import oracle
    from oracle.coarse import coarse_factor
    inp = make_inputs(w, seed)
    t_all = time.perf_counter()
    pb, opt = _oracle_problem(w, inp, w.nx, w.ny, w.nz)
    wb = oracle.build_wirebasket(pb.grid, opt.coarse)
    state = oracle.BasisState(wb)
    stages = {}

    def timed(name, fn, *a):
        t0 = time.perf_counter()
        out = fn(*a)
        stages[name] = stages.get(name, 0.0) + time.perf_counter() - t0
        return out

    p_n = pb.with_fixed(inp["p0"])
    dt = inp["dts"][0]
    lin = timed("assemble", oracle.assemble, pb, p_n, p_n, dt, opt.full_jacobian)
    LU = timed("ilu_factor", oracle.ilu0, lin.A)
    Ab = timed("basis", oracle.basis_operator, pb, opt.basis, lin.rho, lin.c, p_n, dt)
    rebuilt = timed("basis", state.update, Ab, opt.adapt_theta)
    P = timed("basis", state.matrix)
    R = timed("coarse_factor", oracle.restriction,
              0 if opt.restriction == 2 else opt.restriction, P, wb)
    lu = timed("coarse_factor", lambda: coarse_factor(oracle.coarse_operator(R, lin.A, P)))
    p = p_n.copy()
    r0 = float(np.linalg.norm(lin.f - lin.A @ p))
    its = 0
    t0 = time.perf_counter()
    while its < opt.max_cams:
        p = oracle.cams_iteration(lin.A, lin.f, p, P, R, lu, LU, opt.n_pre, opt.n_post)
        its += 1
        if float(np.linalg.norm(lin.f - lin.A @ p)) < opt.lin_rtol * r0:
            break
    stages["cams_iterations"] = time.perf_counter() - t0
    wall = time.perf_counter() - t_all
    N = pb.grid.N
    return {"workload": w.name, "cells": N, "newton_steps": 1, "cams_its": its,
            "entities_built": int(rebuilt), "wall_s": wall,
            "stage_s": {k: round(v, 3) for k, v in stages.items()},
            "setup_s": round(wall - sum(stages.values()), 3),
            "value": N * its / wall, "unit": UNIT,
            "value_iterations_only": N * its / stages["cams_iterations"],
            "cores": cpu_cores_used(), **host_cpu()}


def cpu_cores_used():
    return 1


def host_cpu():
    """The host's core count and CPU model (the oracle's timing host)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu part", "hardware") and ":" in line:
                    model = line.split(":", 1)[1].strip()
                    if key == "model name":
                        break
    except OSError:
        pass
    import platform
    return {"host_cores": os.cpu_count(), "cpu_model": model or platform.processor() or None,
            "machine": platform.machine()}


def run_reference(args, w, rank, world):
    if rank != 0:
        return None
    vals = []
    inp = make_inputs(w, args.seed)
    for _ in range(args.warmup):
        oracle_sample(w, args.seed, inp=inp)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        v, dt, st, sample = oracle_sample(w, args.seed, inp=inp)
        vals.append(v)
    wall = time.perf_counter() - t0
    value = float(np.mean(vals))
    return {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": w.name + variant_suffix(), "sample": sample,
                       "restriction": ("MSFE", "MSFV", "MSFE+closing MSFV")[w.restriction]},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores_used(),
                             "kind": "oracle", "sample": sample, **host_cpu()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    args = parse()
    if args.jacobian:
        VARIANT["jacobian"] = 1
    if args.cf:
        VARIANT["cf"] = True
    rank, world, local_rank = dist_env()
    if args.workload == ENSEMBLE:
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the ensemble leg has no "
                              "oracle arm; run the oracle on single workloads"}), flush=True)
            return
        if world > 1:
            import torch
            torch.cuda.set_device(local_rank)
            torch.distributed.init_process_group("nccl")
        out = run_ensemble(args, rank, world, local_rank)
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    w = WORKLOADS[args.workload]
    if args.restriction is not None:
        w = w.with_(restriction=args.restriction)
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    if args.impl == "reference" and args.oracle_newton_step:
        out = {"impl": "reference", "oracle_newton_step": oracle_newton_step(w, args.seed)} \
            if rank == 0 else None
    elif args.impl == "reference":
        out = run_reference(args, w, rank, world)
    else:
        out = run_cams(args, w, rank, world, local_rank)
        if w.precision and not args.no_fp64:
            # the same step with every stage in FP64, measured the same way
            ref = run_cams(args, w.with_(precision=0), rank, world, local_rank, e2e_leg=False)
            p64 = ref.pop("_p")
            out["fp64"] = ref
            err = float(np.abs(out["_p"] - p64).max() / max(np.abs(p64).max(), 1e-300))
            out["error_vs_fp64"] = {"rel_linf": err, "note": "final pressure of the mixed step "
                                    "against the FP64 step (the FP64 engine is held to the "
                                    "FP64 oracle by the parity tests)"}
        if w.precision and not args.no_learned:
            # the same step with the learned surrogate supplying the interiors it
            # passes, at the metric's tolerance and at LEARNED_TIGHT_TOL; every
            # leg's pressure against a converged FP64 reference
            from paper_1705_05783_gb300 import surrogate as sg
            if os.path.exists(sg.PARAMS_FILE):
                pref = converged_reference(args, w, local_rank)
                conv = {"mixed": rel_linf(out["_p"], pref)}
                if "fp64" in out:
                    conv["fp64"] = rel_linf(p64, pref)
                for key, wl in (("learned", w), ("learned_tight", w.with_(nl_tol=LEARNED_TIGHT_TOL))):
                    lrn = run_cams(args, wl, rank, world, local_rank, e2e_leg=False,
                                   surrogate=(sg.load_params(), LEARNED_GATE))
                    pl = lrn.pop("_p")
                    ref_p = p64 if "fp64" in out else out["_p"]
                    lrn["nl_tol"] = wl.nl_tol
                    lrn["error_vs_fp64" if "fp64" in out else "difference_vs_exact_basis"] = rel_linf(pl, ref_p)
                    lrn["error_vs_converged"] = rel_linf(pl, pref)
                    conv[key] = lrn["error_vs_converged"]
                    out[key] = lrn
                out["error_vs_converged_fp64"] = {
                    **conv, "reference": f"FP64 engine at a {REFERENCE_TOL:g} relative ||eps|| "
                                         "(the parity tests hold the FP64 engine to the oracle)"}
        out.pop("_p", None)
        if rank == 0 and world == 1 and not args.no_baseline:
            v, dt, st, sample = oracle_sample(w, args.seed)
            out["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cpu_cores_used(),
                                   "kind": "oracle", "sample": f"{sample}, one implicit step "
                                   f"({st.newton_its} Newton, {st.cams_its} C-AMS its) in {dt:.1f} s",
                                   **host_cpu()}
    if world > 1:
        import torch
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    if rank == 0 and out is not None:
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
