#!/usr/bin/env python
"""ChFSI benchmark on GB300: seconds per ChFSI iteration on the periodic FCC
Gaussian-well workload (16^3 cells, p = 6, 884,736 unknowns, N = 1000 wanted
pairs + 100 buffer, Chebyshev degree 40; wavefunction block and cell tile
chosen by the library autotuner, the paper-sized block of 200 among the candidates).

One step = one ChFSI iteration on device-resident data: Chebyshev filter
(Eq. chebFilter), CholGS (Algorithm CholGS) and Rayleigh-Ritz (Sec. 3.5) of
arXiv:1903.10959, each through the library's C ABI.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec bf16x3|mixed|fp64|tf32]
                  [--impl ours|reference] [--workload chfsi|c3|batch|serving]

The default precision stores the block in binary32 and forms the cell
products from three bf16 terms per operand (six kind::f16 MMAs, FP32
accumulation); CholGS / Rayleigh-Ritz use 3xTF32 off-diagonal and binary64
diagonal blocks, Cholesky and eigensolve in binary64.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload (extrapolated to one iteration by exact operation
counts).  With N > 1 (torchrun) every rank runs an independent replica of the
workload (the path has no data-path collective; "replicas only").
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "ChFSI s/iter (filter + CholGS + RR), fcc-periodic 16^3 cells p=6"
UNIT = "s/iter"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="bf16x3", choices=["bf16x3", "f16x2", "mixed", "fp64", "tf32"],
                    help="bf16x3: BF16x3 cell products (the fastest mixed path); mixed: 3xTF32")
    ap.add_argument("--e2e-steps", type=int, default=3,
                    help="end-to-end steps (median wall time reported)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--gather", default="rings", choices=["async", "registers", "rings", "rings4", "whole"],
                    help="BF16x3 cell kernel gather (bulk async copies or register loads)")
    ap.add_argument("--lanes", type=int, default=0,
                    help="filter lanes: column groups filtered concurrently on their own streams "
                         "(0 = the library's default)")
    ap.add_argument("--tall-kernel", default="auto", choices=["auto", "narrow", "wide"],
                    help="tile kernel of the mixed rotations X U: 128 x 128 or 256-row tiles")
    ap.add_argument("--fp64-op", default="default", choices=["default", "cells", "matrix-free"],
                    help="binary64 cell operator")
    ap.add_argument("--no-side-arms", action="store_true",
                    help="skip the binary64 / polished arm and the 20^3-cell p=7 arm")
    ap.add_argument("--small", action="store_true", help="small case for profiling runs")
    ap.add_argument("--n-want", type=int, default=0,
                    help="small case: wanted states (default 200; the block adds a 10%% buffer)")
    ap.add_argument("--block", type=int, default=0,
                    help="wavefunction block of the filter (0: chosen by the autotuner)")
    ap.add_argument("--tile", type=int, default=64, choices=[64, 128],
                    help="cell-kernel column tile when --block is given")
    ap.add_argument("--workload", default="chfsi", choices=["chfsi", "c3", "batch", "serving", "kpoint"],
                    help="chfsi: the 16^3-cell p=6 FCC system; c3: 20^3 cells p=7 with "
                         "projectors, N=3000 (block 1100); batch: 64 small Dirichlet systems "
                         "filtered together; serving: request stream through the "
                         "continuous-batching server")
    ap.add_argument("--requests", type=int, default=12, help="serving: number of requests")
    ap.add_argument("--slots", type=int, default=4, help="serving: concurrently admitted requests")
    ap.add_argument("--dof-max", type=float, default=2.0e6, help="serving: largest request (unknowns)")
    ap.add_argument("--fp64-requests", type=int, default=4,
                    help="serving: requests (smallest first) of the FP64 comparison")
    ap.add_argument("--rates", default="0.5,0.8,1.0",
                    help="serving: arrival rates as fractions of the measured mixed capacity")
    return ap.parse_args()


def workload(small=False, kind="chfsi", n_want=0):
    from paper_1903_10959_gb300 import workloads as W
    if kind == "c3":
        if small:   # the same site density and degree on a 10^3-cell box (profiling runs)
            return W.cubic_sites_nonlocal(ncell=10, L=20.0, n_side=5, n_want=600, block=660)
        return W.cubic_sites_nonlocal(block=1100)
    if small:
        return W.fcc_periodic(ncell=8, p=6, L=15.0, n_fcc=2, n_want=n_want or 200, degree=40, iters=4,
                              block=200)
    return W.fcc_periodic()


def workload_config(s, l2_note):
    nl = " + %d sites x 4 projectors" % len(s.nl_centres) if len(s.nl_centres) else ""
    return {
        "workload": "%s %d^3 cells p=%d L=%g, %d unknowns, %d Gaussian wells%s, "
                    "N=%d (+%d buffer), wavefunction block %d, Chebyshev degree %d"
                    % (s.name.rsplit("-", 2)[0], s.ncell, s.p, s.L, s.ndofs, len(s.depths), nl,
                       s.n_want, s.n_buffer, s.block, s.degree),
        "unknowns": s.ndofs, "n_sub": s.n_sub, "block": s.block, "degree": s.degree, "p": s.p,
        "cells": s.ncell ** 3, "l2": l2_note,
    }


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu):
        self.gpu = gpu
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ------------------------------------------------------------------ replicas
def job_seconds_per_iter(t_local, steps, dist=None, device="cpu"):
    """Whole-job time and s/iter of N independent replicas: the slowest rank's
    time (max over ranks, then a barrier) over the steps all ranks ran."""
    import torch
    world = 1
    t = float(t_local)
    if dist is not None and dist.is_initialized():
        world = dist.get_world_size()
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
        dist.barrier()
    return t, t / (steps * world)


# ------------------------------------------------------------------ profiled traffic
def profiled_traffic(kernel, s, n):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of
    `kernel` for this workload and block, from the committed ncu summary
    profiles/<kernel>_traffic.txt (lines "<cells> <p> <block> <bytes>"); None
    when that configuration has not been profiled."""
    path = os.path.join(ROOT, "profiles", kernel + "_traffic.txt")
    if not os.path.exists(path):
        return None
    for line in open(path):
        f = line.split()
        if len(f) == 4 and not line.startswith("#"):
            try:
                if (int(f[0]), int(f[1]), int(f[2])) == (s.ncell ** 3, s.p, min(s.block, n)):
                    return float(f[3])
            except ValueError:
                continue
    return None


# ------------------------------------------------------------------ oracle timing
def oracle_sample_seconds(s, rows_sample=20000, cells_sample=24):
    """Extrapolated seconds of one oracle ChFSI iteration on the workload.

    Sample: the oracle's cell loop (H_e X_e gather/scatter, Eq. discreteHam) on
    `cells_sample` cells x one filter block, the recurrence update, and the
    dense CholGS / RR products on `rows_sample` rows; each timed piece is scaled
    by its exact operation count to the full iteration."""
    from oracle import hamiltonian as oham
    prob = oham.wells_problem(s.ncell, s.p, s.L, True, s.centres, s.depths, s.widths)
    n, B, m = s.n_sub, s.block, s.degree
    M = prob.ndofs
    rng = np.random.default_rng(0)
    X = rng.uniform(-1, 1, (M, B))
    cells = list(range(cells_sample))
    for e in cells:
        prob.cell_hamiltonian(e)            # build outside the timed region
    dm = prob.mesh.dofmap()
    out = np.zeros_like(X)
    t0 = time.perf_counter()
    for e in cells:
        d = dm[e]
        out[d] += prob.cell_hamiltonian(e) @ X[d]
    t_cells = time.perf_counter() - t0
    t_apply = t_cells / cells_sample * prob.mesh.ncells          # one H X on B columns
    Xs = X[:rows_sample]
    t0 = time.perf_counter()
    Y = 0.5 * (Xs - 0.3 * Xs) - 0.2 * Xs                           # recurrence update
    t_upd = (time.perf_counter() - t0) * M / rows_sample
    nb = -(-n // B)
    t_filter = m * nb * (t_apply + t_upd)
    Xr = rng.uniform(-1, 1, (rows_sample, n))
    t0 = time.perf_counter()
    S = Xr.T @ Xr
    t_gram = (time.perf_counter() - t0) * M / rows_sample
    S = S + n * np.eye(n)
    import scipy.linalg as sla
    t0 = time.perf_counter()
    L = np.linalg.cholesky(S)
    Linv = sla.solve_triangular(L, np.eye(n), lower=True)
    t_fact = time.perf_counter() - t0
    t0 = time.perf_counter()
    _ = Xr @ Linv.T
    t_rot = (time.perf_counter() - t0) * M / rows_sample
    t0 = time.perf_counter()
    _ = np.linalg.eigh(0.5 * (S + S.T))
    t_eig = time.perf_counter() - t0
    del Y
    t_cholgs = t_gram + t_fact + t_rot
    t_rr = nb * t_apply + t_gram + t_eig + t_rot
    total = t_filter + t_cholgs + t_rr
    sample = ("oracle cell loop on %d of %d cells x %d columns, recurrence and dense products on "
              "%d of %d rows, %dx%d Cholesky/eigh in full; scaled by exact operation counts to "
              "one iteration" % (cells_sample, prob.mesh.ncells, B, rows_sample, M, n, n))
    return total, sample, {"filter": t_filter, "cholgs": t_cholgs, "rr": t_rr}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


# ------------------------------------------------------------------ reference arm
def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores.  Each step is one
    bounded sample of the workload (the same sample as the GPU arm's
    cpu_baseline: all columns in one block), extrapolated to one ChFSI
    iteration by exact operation counts; the value is the mean over the
    timed samples."""
    import dataclasses
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    s = workload(args.small)
    s = dataclasses.replace(s, block=s.n_sub)
    times = []
    sample = ""
    for i in range(args.warmup + args.steps):
        t, sample, _ = oracle_sample_seconds(s)
        if i >= args.warmup:
            times.append(t)
    v = float(np.mean(times))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": v * 1e3,
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "extrapolated": True,
        "step_note": "each step is one bounded oracle sample extrapolated to one ChFSI iteration",
        "config": workload_config(s, "host memory"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                         "sample": sample, "extrapolated": True},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ rooflines
# Binary64 rate of GB300 from its unit counts: 152 SMs x 2 FP64 FMA per clock
# x 2 flops x 2.07 GHz = 1.259 TFLOP/s (the nominal 1.25).
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
# MMA passes the cell kernel issues per algorithmic multiply-add, by precision.
MMA_PASSES = {"bf16x3": 6, "f16x2": 3, "mixed": 3, "tf32": 1}
# Cell-matrix bytes per element each precision's cell kernel reads.
CELL_MATRIX_BYTES = {"bf16x3": 6, "f16x2": 4, "mixed": 8, "tf32": 4, "fp64": 8}
CELL_KERNEL = {"bf16x3": "tc_cell_bf16_kernel", "f16x2": "tc_cell_bf16_rings_kernel<2, 0, 2>",
               "mixed": "tc_cell_r_kernel",
               "tf32": "tc_cell_r_kernel", "fp64": "cell_fp64_kernel"}
# The BF16x3 cell kernel each gather mode launches.
BF16_KERNEL = {"registers": "tc_cell_bf16_kernel", "async": "tc_cell_bf16_async_kernel",
               "rings": "tc_cell_bf16_rings_kernel", "rings4": "tc_cell_bf16_rings_kernel",
               "whole": "tc_cell_bf16_whole_kernel"}


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        pk = json.load(open(path))
        pk["source"] = "of measured"
        return pk
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "source": "of fallback"}


def dtype_peak(prec, peaks):
    """Dense peak of the MMA's own operand type, sustained (the cell kernel is
    timed inside a seconds-long step): BF16 measured; TF32 = measured BF16 x
    the nominal 1.1 / 2.25 ratio; binary64 from unit counts and clock."""
    bf = peaks.get("bf16_tflops_sustained", 1700.0)
    if prec == "bf16x3":
        return bf, "BF16 dense, measured sustained (MEASURED_PEAKS.json), %s" % peaks["source"]
    if prec == "f16x2":
        return bf, ("FP16 dense = measured BF16 sustained x 1 (the nominal FP16 and BF16 dense rates "
                    "are equal), %s" % peaks["source"])
    if prec in ("mixed", "tf32"):
        return bf * 1.1 / 2.25, ("TF32 dense = measured BF16 sustained x 1.1/2.25 nominal ratio, %s"
                                 % peaks["source"])
    return FP64_PEAK_TFLOPS, "binary64: 152 SMs x 2 FMA/clk x 2 x 2.07 GHz (unit counts and clock)"


def mf_flops_per_cell(p):
    """Flops of one sum-factorised cell apply per vector (n1 = p + 1, q = p + 2)."""
    n1, q = p + 1, p + 2
    return 14 * n1 ** 4 + 3 * n1 ** 3 + 4 * (q * n1 ** 3 + q * q * n1 * n1 + q ** 3 * n1) + q ** 3 + n1 ** 3


def rooflines(prec, s, n, M, peaks, col_steps, steps_blocks, nblocks, cell_ms, cell_n, asm_ms, asm_n,
              fp64_op="cells", gather="rings"):
    """Cell-kernel, assembly and filter-step rooflines from the per-launch event times.

    Cell kernel: algorithmic work = N_c 2 n_e^2 flops per vector and
    application (the dense cell products of Sec. 3.3.1), against the dense
    peak of the MMA's operand type; the MMA passes the split-precision scheme
    executes per algorithmic flop are reported beside it, not folded into the
    peak.  Algorithmic bytes per launch = the cell matrices (N_c n_e^2 s_H) +
    the block read (M nb s_X) + the dense cell blocks written (N_c n_e nb s_X).
    Assembly: the cell blocks read and Y_out written by every launch, Y_in
    read by the m filter steps and Y_prev by the m - 1 after the first (the
    application of H~ in Rayleigh-Ritz reads neither), the unknown -> cell-row
    table ((M + 1 + N_c n_e) 4 B), and the projector term where the assembly
    reads it.
    Filter step: cell kernel + assembly against the fused-recurrence minimum
    (3 s_X per unknown and vector + the cell matrices at s_H)."""
    ne = (s.p + 1) ** 3
    ncells = s.ncell ** 3
    sx = 8 if prec == "fp64" else 4
    s_h = CELL_MATRIX_BYTES[prec]
    alg_flops = col_steps * ncells * 2 * ne * ne
    peak, note = dtype_peak(prec, peaks)
    achieved = alg_flops / (cell_ms / 1e3) / 1e12
    kern = BF16_KERNEL.get(gather, CELL_KERNEL[prec]) if prec == "bf16x3" else CELL_KERNEL[prec]
    roof = {"bound": "alu" if prec == "fp64" else "tensor", "achieved": achieved, "peak": peak,
            "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": profiled_traffic(kern, s, n) if prec != "fp64" else None,
            "kernel": kern, "launches": int(cell_n), "avg_launch_ms": cell_ms / max(cell_n, 1),
            "flops_per_launch": alg_flops / max(cell_n, 1),
            "peak_note": note + "; achieved = algorithmic flops (N_c 2 n_e^2 per vector) / event time"}
    if prec == "fp64":
        if fp64_op == "matrix-free":
            # the sum-factorised apply executes fewer flops than the dense count:
            # report its own flops against the binary64 rate, and the dense-count
            # rate beside it
            mf = col_steps * ncells * mf_flops_per_cell(s.p)
            roof.update({"achieved": mf / (cell_ms / 1e3) / 1e12, "kernel": "mf_cell_fp64_kernel",
                         "flops_per_launch": mf / max(cell_n, 1),
                         "dense_count_tflops": achieved,
                         "peak_note": note + "; achieved = executed sum-factorised flops "
                                             "(14 n1^4 + 3 n1^3 + 4 (q n1^3 + q^2 n1^2 + q^3 n1) + q^3 "
                                             "+ n1^3 per cell and vector) / event time"})
            roof["frac"] = roof["achieved"] / peak
        return roof, None, None
    cell_bytes = (steps_blocks * nblocks * ncells * ne * ne * s_h
                  + col_steps * M * sx + col_steps * ncells * ne * sx)
    passes = MMA_PASSES[prec]
    roof["bytes_per_launch"] = cell_bytes / max(cell_n, 1)
    roof["hbm_gbs"] = cell_bytes / (cell_ms / 1e3) / 1e9
    roof["executed_mma"] = {"passes_per_flop": passes, "tflops": passes * achieved,
                            "frac_of_peak": passes * achieved / peak,
                            "note": "MMA work the split-precision scheme issues (not the method's work)"}
    # every assembly launch reads the cell blocks and writes Y_out; the filter's
    # degree steps also read Y_in (the shift) and, after the first, Y_prev; the
    # application of H~ in Rayleigh-Ritz (one launch per block and iteration)
    # reads neither
    it_cols = col_steps / (s.degree + 1)
    asm_bytes = (col_steps * (ncells * ne + M) * sx + it_cols * (2 * s.degree - 1) * M * sx
                 + steps_blocks * nblocks * (M + 1 + ncells * ne) * 4)
    if len(s.nl_centres) and not (prec == "bf16x3" and gather in ("rings", "rings4")):
        asm_bytes += col_steps * M * sx          # the projector term, read by the assembly unless
                                                 # the ring kernel took it as extra K-chunks
    asm_roof = {"bound": "hbm", "achieved": asm_bytes / (asm_ms / 1e3) / 1e9,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "kernel": "tc_assemble_kernel",
                "launches": int(asm_n), "avg_launch_ms": asm_ms / max(asm_n, 1),
                "bytes_per_launch": asm_bytes / max(asm_n, 1),
                "traffic": profiled_traffic("tc_assemble_kernel", s, n),
                "peak_note": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), %s" % peaks["source"]}
    asm_roof["frac"] = asm_roof["achieved"] / peaks["hbm_gbs"]
    step_bytes = col_steps * 3 * sx * M + steps_blocks * nblocks * ncells * ne * ne * s_h
    step_roof = {"bound": "hbm", "achieved": step_bytes / ((cell_ms + asm_ms) / 1e3) / 1e9,
                 "peak": peaks["hbm_gbs"], "unit": "GB/s", "kernels": kern + " + tc_assemble_kernel",
                 "note": "filter degree step against the fused-recurrence minimum "
                         "(3 s_X per unknown and vector + the cell matrices at %d B)" % s_h}
    step_roof["frac"] = step_roof["achieved"] / peaks["hbm_gbs"]
    return roof, asm_roof, step_roof


# ------------------------------------------------------------------ side arms
def ev_seconds(stream, fn):
    """Device seconds of fn() on the stream (CUDA events, synchronised)."""
    import torch
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / 1e3


def fp64_polish_arm(ctx, s, X, b, D_mixed, stream, mixed_s_per_iter):
    """Binary64 ChFSI iteration on the same workload and GPU, which is also
    the binary64 polish of the mixed block (chfsi_solve_polish's step 3):
    the benchmark's binary32 block (after its mixed iterations) is copied to
    binary64, one binary64 iteration of degree 1 grows the scratch, then one
    timed binary64 iteration {filter of the workload's degree, CholGS, RR}.
    Reports the binary64 s/iter, the polished solve's s/iter over the
    workload's iteration count, and the generalized residuals of the wanted
    pairs before and after the polish."""
    import torch
    n, k = s.n_sub, s.n_want
    X64 = X.double()
    res_mixed = ctx.residuals(X64[:, :k], D_mixed[:k], prec="fp64")[1]
    D = D_mixed

    def iteration(deg, D):
        ctx.filter(X64, deg, float(D[-1]), b, float(D[0]), prec="fp64")
        ctx.cholgs(X64, prec="fp64")
        return ctx.rayleigh_ritz(X64, prec="fp64")

    D = iteration(1, D)                     # grows the binary64 scratch
    out = {}
    t0 = time.perf_counter()
    t = ev_seconds(stream, lambda: out.update(D=iteration(s.degree, D)))
    wall = time.perf_counter() - t0
    D = out["D"]
    res_pol = ctx.residuals(X64[:, :k], D[:k], prec="fp64")[1]
    res_pol32 = ctx.residuals(X64[:, :k].float().double(), D[:k], prec="fp64")[1]
    del X64
    torch.cuda.empty_cache()
    return {
        "fp64_s_per_iter": t, "fp64_wall_s": wall,
        "fp64_vs_mixed_ratio": t / mixed_s_per_iter,
        "polished_s_per_iter": (s.iters * mixed_s_per_iter + t) / s.iters,
        "polished_note": "%d mixed iterations + 1 binary64 polish iteration of degree %d, per "
                         "iteration of the workload" % (s.iters, s.degree),
        "max_gres_mixed": float(np.max(res_mixed)), "max_gres_polished": float(np.max(res_pol)),
        "max_gres_polished_stored_binary32": float(np.max(res_pol32)),
        "max_abs_eval_change_mixed_to_polished": float(np.abs(D[:k] - D_mixed[:k]).max()),
        "n_checked": k,
    }


def c3_arm(stream, steps=1, gather="rings", prec="bf16x3"):
    """The largest single-GPU workload (20^3 cells, p = 7, 1,000 projector
    sites, N = 3,000 + 300, block 1,100, degree 50): one warm-up and `steps`
    timed mixed (BF16x3) ChFSI iterations, with the cell-kernel roofline."""
    import torch
    from paper_1903_10959_gb300 import Context
    from paper_1903_10959_gb300 import workloads as W
    s = W.cubic_sites_nonlocal(block=1100)
    t0 = time.perf_counter()
    ctx = Context(s.ncell, s.L, s.p, periodic=True, stream=stream)
    ctx.set_potential_gaussians(s.centres, s.depths, s.widths)
    ctx.set_projectors(s.nl_centres, s.nl_h, s.nl_sigma, s.nl_rcut)
    ctx.build()
    ctx.set_blocking(s.block, 1)
    ctx.set_cell_gather(gather)
    n, M = s.n_sub, ctx.ndofs
    b = ctx.bounds(20, s.seed)
    X = torch.empty((M, n), dtype=torch.float32, device="cuda")
    ctx.fill_uniform(X, s.seed, prec=prec)
    ctx.cholgs(X, prec=prec)
    state = {"D": ctx.rayleigh_ritz(X, prec=prec)}
    setup_s = time.perf_counter() - t0
    phase = np.zeros(3)

    def step():
        D = state["D"]
        ctx.filter(X, s.degree, float(D[-1]), b, float(D[0]), prec=prec)
        phase[0] += ctx.last_timings()[0]
        ctx.cholgs(X, prec=prec)
        phase[1] += ctx.last_timings()[1]
        state["D"] = ctx.rayleigh_ritz(X, prec=prec)
        phase[2] += ctx.last_timings()[2]

    step()
    phase[:] = 0
    ctx.set_kernel_timing(True)
    ctx.kernel_timings()

    def timed():
        for _ in range(steps):
            step()
    t = ev_seconds(stream, timed) / steps
    kt = [float(v) for v in ctx.kernel_timings()]
    ctx.set_kernel_timing(False)
    nblocks = -(-n // s.block)
    steps_blocks = steps * (s.degree + 1)
    roof, asm_roof, _ = rooflines(prec, s, n, M, load_peaks(), steps_blocks * n, steps_blocks,
                                  nblocks, kt[0], kt[2], kt[1], kt[3], gather=gather)
    ctx.destroy()
    del X
    torch.cuda.empty_cache()
    return {"workload": "nonlocal-periodic 20^3 cells p=7 L=40, %d unknowns, 1000 wells + 1000 "
                        "sites x 4 projectors, N=%d (+%d buffer), block %d, degree %d"
                        % (M, s.n_want, s.n_buffer, s.block, s.degree),
            "s_per_iter": t, "steps": steps, "warmup": 1, "setup_s": setup_s,
            "phases_ms_per_step": {"filter": phase[0] / steps, "cholgs": phase[1] / steps,
                                   "rr": phase[2] / steps},
            "projector_kernels_ms_per_step": kt[4] / steps,
            "roofline": roof, "roofline_assembly": asm_roof, "precision": prec}


# ------------------------------------------------------------------ our arm
def run_ours(args):
    import torch
    from paper_1903_10959_gb300 import Context, _lib

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    import dataclasses
    s = workload(args.small, args.workload, args.n_want)
    if args.block:
        s = dataclasses.replace(s, block=args.block)
    prec = {"mixed": "mixed", "fp64": "fp64", "tf32": "tf32", "bf16x3": "bf16x3", "f16x2": "f16x2"}[args.prec]
    dt = torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.current_stream()
    ctx = Context(s.ncell, s.L, s.p, periodic=True, stream=stream)
    ctx.set_potential_gaussians(s.centres, s.depths, s.widths)
    if len(s.nl_centres):
        ctx.set_projectors(s.nl_centres, s.nl_h, s.nl_sigma, s.nl_rcut)
    ctx.build()
    ctx.set_blocking(s.block, 1)
    ctx.set_cell_tile(args.tile)
    ctx.set_cell_gather(args.gather)
    ctx.set_gemm_kernels(tall={"auto": -1, "narrow": 0, "wide": 1}[args.tall_kernel])
    if args.lanes:
        ctx.set_filter_lanes(args.lanes)
    ctx.set_fp64_operator(args.fp64_op)
    n, M = s.n_sub, ctx.ndofs
    b = ctx.bounds(20, s.seed)
    X = torch.empty((M, n), dtype=dt, device="cuda")
    ctx.fill_uniform(X, s.seed, prec=prec)
    tuned = None
    if not args.block and args.workload != "c3":
        # wavefunction block and cell tile picked by the library's autotuner
        blk, tile, cand = ctx.autotune(X, prec=prec)
        s = dataclasses.replace(s, block=blk)
        tuned = {"block": blk, "tile": tile,
                 "candidates_ms": {"%d/%d" % k: round(v, 3) for k, v in cand.items()}}
    ctx.cholgs(X, prec=prec)
    state = {"D": ctx.rayleigh_ritz(X, prec=prec)}
    phase = np.zeros(3)

    def step():
        D = state["D"]
        ctx.filter(X, s.degree, float(D[-1]), b, float(D[0]), prec=prec)
        phase[0] += ctx.last_timings()[0]
        ctx.cholgs(X, prec=prec)
        phase[1] += ctx.last_timings()[1]
        state["D"] = ctx.rayleigh_ritz(X, prec=prec)
        phase[2] += ctx.last_timings()[2]

    for _ in range(args.warmup):
        step()
    phase[:] = 0
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    ctx.set_kernel_timing(True)
    ctx.kernel_timings()
    l0 = _lib.kernel_launches()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    launches = _lib.kernel_launches() - l0
    kt = ctx.kernel_timings()          # [cell ms, assembly ms, cell launches, assembly launches]
    ctx.set_kernel_timing(False)
    clk = clocks.stop()
    t = e0.elapsed_time(e1) / 1e3
    t, value = job_seconds_per_iter(t, args.steps, dist, "cuda")

    # Rooflines (per-launch CUDA events on the context stream).
    nblocks = -(-n // s.block)
    ne = (s.p + 1) ** 3
    ncells = s.ncell ** 3
    sx = 8 if prec == "fp64" else 4
    filter_s = phase[0] / 1e3
    # cell launches in the timed region: every filter degree step and the RR
    # application, each over one column block
    steps_blocks = args.steps * (s.degree + 1)
    col_steps = steps_blocks * n                  # (vector, application) units
    peaks = load_peaks()
    cell_ms, asm_ms, cell_n, asm_n, nl_ms, nl_n = [float(v) for v in kt]
    roof, asm_roof, step_roof = rooflines(prec, s, n, M, peaks, col_steps, steps_blocks, nblocks,
                                          cell_ms, cell_n, asm_ms, asm_n, ctx.fp64_operator,
                                          gather=args.gather)
    alg_flops = col_steps * ncells * 2 * ne * ne
    phase_timed = phase.copy()
    # end to end through host buffers, inside the library (chfsi_step_host):
    # H2D of the pinned host block, one iteration, D2H of the block and the
    # Ritz values; wall time of the C-ABI call per step
    e2e = None
    if args.e2e_steps > 0:
        Xh = torch.empty((M, n), dtype=dt, pin_memory=True)
        Xh.copy_(X)
        torch.cuda.synchronize()

        def host_step(mode):
            D = state["D"]
            t0 = time.perf_counter()
            ev, ms = ctx.step_host(Xh, X, s.degree, float(D[-1]), b, float(D[0]), prec=prec,
                                   copy_mode=mode)
            wall = time.perf_counter() - t0
            state["D"] = ev
            return wall, ms

        walls, dms = [], []
        for _ in range(args.e2e_steps):
            w, ms = host_step(0)
            walls.append(w)
            dms.append(ms)
        wce, msce = host_step(1)                     # the same call with the copy engines
        nbytes = M * n * X.element_size()
        med = np.median(np.array(dms), axis=0)
        e2e = {"value": float(np.median(walls)), "unit": UNIT, "h2d_bytes_per_step": nbytes,
               "d2h_bytes_per_step": nbytes + n * 8,
               "device_ms": {"h2d": float(med[0]), "step": float(med[1]), "d2h": float(med[2])},
               "copy_gbs": {"h2d": nbytes / med[0] / 1e6, "d2h": nbytes / med[2] / 1e6},
               "copy_engine_step": {"wall_s": wce, "h2d_ms": float(msce[0]), "d2h_ms": float(msce[2])},
               "note": "chfsi_step_host on a pinned host block: the SMs move the rows over the "
                       "host link (copy_mode 0); copy_engine_step is the same call with the DMA "
                       "copy engines"}
        del Xh

    # the step after RR (Sec. 3.5, Algorithms rr and dc): spectrum-splitting RR on the
    # orthonormal block (n_fr = 15 % of the subspace), Fermi level and the
    # electron density at the Gauss points; timed with events, not in `value`
    split = None
    if prec != "tf32":
        from paper_1903_10959_gb300 import fermi_level
        n_fr = max(1, int(round(0.15 * n)))
        Xfr = torch.empty((M, n_fr), dtype=dt, device="cuda")
        q = s.p + 2
        rho = torch.empty(ncells * q ** 3, dtype=torch.float64, device="cuda")

        def ev_time(fn, reps=3):
            fn()
            torch.cuda.synchronize()
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            for _ in range(reps):
                fn()
            b_.record(stream)
            torch.cuda.synchronize()
            return a_.elapsed_time(b_) / reps

        dfr = {}
        t_split = ev_time(lambda: dfr.update(d=ctx.rayleigh_ritz_split(X, Xfr, prec=prec)))
        mu, occ = fermi_level(dfr["d"], n - n_fr, 2 * (n - n_fr) + n_fr, 0.01)
        t_den = ev_time(lambda: ctx.density(X, rho, Xfr, occ, prec=prec))
        n1 = s.p + 1
        den_flops = ncells * (n + n_fr) * 2 * (n1 ** 3 * q + n1 ** 2 * q ** 2 + n1 * q ** 3)
        # binary64 interpolation: GB300's 1.25 TFLOP/s; binary32: 152 SMs x 128
        # FP32 lanes x 2 flops x 2.07 GHz = 80.6 TFLOP/s
        den_peak = 1.25 if prec == "fp64" else 152 * 128 * 2 * 2.07e9 / 1e12
        achieved = den_flops / (t_den / 1e3) / 1e12
        split = {"n_fr": n_fr, "split_rr_ms": t_split,
                 "full_rr_ms": phase_timed[2] / args.steps, "fermi_level": mu,
                 "density_ms": t_den, "density_gflop": den_flops / 1e9,
                 "density_roofline": {"bound": "alu", "achieved": achieved, "peak": den_peak,
                                      "unit": "TFLOP/s", "frac": achieved / den_peak,
                                      "peak_note": "sum-factorised interpolation in the block's "
                                                   "precision; peak from unit counts and clock"}}
        del Xfr, rho

    # side arms (N = 1 only): the binary64 iteration / polish on this workload,
    # then the 20^3-cell p = 7 workload with projectors
    side = {}
    if world == 1 and not args.no_side_arms and args.workload == "chfsi" and prec != "fp64" \
            and not args.small:
        side["fp64_and_polish"] = fp64_polish_arm(ctx, s, X, b, state["D"], stream, value)
        ctx.destroy()
        del X
        torch.cuda.empty_cache()
        side["c3"] = c3_arm(stream, gather=args.gather, prec=prec if prec in ("bf16x3", "f16x2") else "bf16x3")
    if rank != 0:
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        # the same sample as the reference arm: all columns in one block
        tcpu, sample, parts = oracle_sample_seconds(dataclasses.replace(s, block=s.n_sub))
        cpu = {"value": tcpu, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
               "sample": sample, "phases_s": parts, "extrapolated": True}
    line = {
        "metric": METRIC if args.workload == "chfsi" else
        "ChFSI s/iter (filter + CholGS + RR), %s %d^3 cells p=%d" % (s.name.rsplit("-", 2)[0],
                                                                      s.ncell, s.p),
        "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": value * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp64": "f64", "mixed": "tf32x3", "tf32": "tf32", "bf16x3": "bf16x3", "f16x2": "f16x2"}[prec],
        "data": "synthetic",
        "config": workload_config(s, "inputs larger than L2: X %.1f GB, cell matrices %.1f GB"
                                  % (M * n * sx / 1e9, s.ncell ** 3 * ne * ne * 8 / 1e9)),
        "phases_ms_per_step": {"filter": phase_timed[0] / args.steps,
                               "cholgs": phase_timed[1] / args.steps,
                               "rr": phase_timed[2] / args.steps},
        "filter_tflops": {"algorithmic_per_filter_time": alg_flops / filter_s / 1e12,
                          "algorithmic_per_cell_kernel_time": alg_flops / (cell_ms / 1e3) / 1e12},
        "roofline": roof, "roofline_assembly": asm_roof, "roofline_filter_step": step_roof,
        "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": launches, "autotune": tuned, "spectrum_split_and_density": split,
        "projector_kernels_ms_per_step": nl_ms / args.steps if nl_n else None,
        "clocks": clk, "precision": prec, "parallelism": "replicas" if world > 1 else "single",
    }
    line.update(side)
    print(json.dumps(line), flush=True)
    if not side:
        ctx.destroy()


# ------------------------------------------------------------------ serving
SERVE_DEGREE, SERVE_ITERS, SERVE_WARM, SERVE_TOL = 30, 20, 6, 1.0e-5


def serve_stream(reqs, prec, slots, arrivals=None, budget=150 << 30):
    """Submit the requests (at the arrival times, seconds from now, or all at
    once) to a fresh server and wait for all; per-request results + makespan."""
    import threading
    from paper_1903_10959_gb300 import Server
    with Server(budget, slots) as sv:
        tickets = [None] * len(reqs)
        t_sub = [0.0] * len(reqs)
        t0 = time.perf_counter()

        def feeder():
            for i, (s, seq) in enumerate(reqs):
                if arrivals is not None:
                    dt = t0 + arrivals[i] - time.perf_counter()
                    if dt > 0:
                        time.sleep(dt)
                t_sub[i] = time.perf_counter()
                tickets[i] = sv.submit(((s.ncell,) * 3, (s.L,) * 3, s.p, True), s.n_sub, s.centres,
                                       s.depths, s.widths, depth_seq=seq, degree=SERVE_DEGREE,
                                       iters=SERVE_ITERS, warm_iters=SERVE_WARM, tol=SERVE_TOL,
                                       n_check=s.n_want, prec=prec, seed=s.seed)

        th = threading.Thread(target=feeder)
        th.start()
        th.join()
        res = [sv.poll(t, wait=True) for t in tickets]
        t_end = max(ts + r["total_ms"] * 1e-3 for ts, r in zip(t_sub, res))
    return res, t_end - t0


def serve_summary(res, makespan):
    ok = [r for r in res if r["status"] == 0]
    nsolves = sum(r["nsolves"] for r in ok)
    first = np.array([r["first_ms"] for r in ok])
    total = np.array([r["total_ms"] for r in ok])
    resolve = np.array([x for r in ok for x in r["solve_ms"][1:]])
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None  # noqa: E731
    return {"requests": len(res), "failed": len(res) - len(ok), "solves": nsolves,
            "makespan_s": makespan, "solves_per_s": nsolves / makespan,
            "first_solve_ms_p50": pct(first, 50), "first_solve_ms_p99": pct(first, 99),
            "request_ms_p50": pct(total, 50), "request_ms_p99": pct(total, 99),
            "warm_resolve_ms_p50": pct(resolve, 50), "warm_resolve_ms_p99": pct(resolve, 99),
            "queue_ms_max": max(r["queue_ms"] for r in ok) if ok else None,
            "iters_cold_mean": float(np.mean([r["iters"][0] for r in ok])) if ok else None,
            "iters_warm_mean": float(np.mean([x for r in ok for x in r["iters"][1:]])) if ok else None,
            "max_gresidual": max(max(r["max_gresidual"]) for r in ok) if ok else None,
            "frac_solves_gres_le_1e-6": float(np.mean([x <= 1e-6 for r in ok for x in r["max_gresidual"]]))
            if ok else None}


def run_serving(args):
    """Continuous-batching serving on a Poisson request stream: mixed-precision
    capacity (all requests at once), then arrival rates at fractions of it,
    against the plain FP64 path run one request at a time on the same stream."""
    import torch
    from paper_1903_10959_gb300 import workloads as W
    torch.cuda.init()
    sp = args.prec if args.prec != "fp64" else "bf16x3"     # the server's mixed precision
    reqs = W.serving_requests(seed=5, count=args.requests, dof_range=(2.0e4, args.dof_max),
                              degree=SERVE_DEGREE)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    warm, _ = serve_stream(reqs[:1], sp, 1)                     # builds, first-use costs
    res_cap, span_cap = serve_stream(reqs, sp, args.slots)
    cap = serve_summary(res_cap, span_cap)
    rate_cap = len(reqs) / span_cap                                    # requests / s
    sweep = {}
    for f in [float(x) for x in args.rates.split(",") if x]:
        arr = W.poisson_arrivals(5, len(reqs), f * rate_cap)
        r, span = serve_stream(reqs, sp, args.slots, arrivals=arr)
        sweep["%.2f" % f] = serve_summary(r, span)
    # plain FP64, one request at a time, against the mixed server on the same
    # subset (the smallest requests: binary64 cell products run ~50x slower)
    order = sorted(range(len(reqs)), key=lambda i: reqs[i][0].ndofs * reqs[i][0].n_sub)
    sub = [reqs[i] for i in order[:args.fp64_requests]]
    r64, span64 = serve_stream(sub, "fp64", 1)
    rmx, spanmx = serve_stream(sub, sp, args.slots)
    fp64 = {"subset": [s.name for s, _ in sub], "fp64_sequential": serve_summary(r64, span64),
            "mixed_server": serve_summary(rmx, spanmx)}
    errs = [float(np.abs(a["evals"][:, :s.n_want] - b["evals"][:, :s.n_want]).max())
            for a, b, (s, _) in zip(rmx, r64, sub) if a["status"] == 0 and b["status"] == 0]
    fp64["max_abs_eval_diff_mixed_vs_fp64"] = max(errs) if errs else None
    fp64["speedup_solves_per_s"] = (fp64["mixed_server"]["solves_per_s"]
                                    / fp64["fp64_sequential"]["solves_per_s"])
    clk = clocks.stop()
    s08 = sweep.get("0.80", cap)
    line = {
        "metric": "serving solves/s and p50/p99 latency (mixed, continuous batching)",
        "precision": sp,
        "value": cap["solves_per_s"], "unit": "solves/s", "n_gpus": 1, "steps": len(reqs),
        "warmup": 1, "ms_per_step": 1e3 / cap["solves_per_s"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+%s (f64 residual)" % {"mixed": "tf32x3"}.get(sp, sp),
        "data": "synthetic",
        "config": {"workload": "serving: %d periodic Gaussian-well requests, unknowns log-uniform "
                               "2e4-%.0e, p in {5,6,7}, N log-uniform 32-1000, 5 warm re-solves "
                               "(1%% depth noise), degree %d, stop at generalized residual %g"
                               % (len(reqs), args.dof_max, SERVE_DEGREE, SERVE_TOL),
                   "slots": args.slots, "budget_bytes": 150 << 30,
                   "iters_cap": [SERVE_ITERS, SERVE_WARM]},
        "capacity": cap, "arrival_sweep": sweep, "fp64_comparison": fp64,
        "p99_request_ms_mixed_at_0.8": s08["request_ms_p99"],
        "clocks": clk,
    }
    del warm
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ k-points
def mfk_flops_per_cell(p):
    """Flops of one Bloch sum-factorised cell apply per complex vector (two real
    columns): per real column the z / y / x passes of T = 1/2 K + 1/2 |k|^2 A and
    of G = k.G (3 + 5 + 4 FMAs per pencil entry: 24 n1^4 flops), the potential
    passes 4 (q n1^3 + q^2 n1^2 + q^3 n1) + q^3, and 3 n1^3 for the scaling and the
    combination of the parts."""
    n1, q = p + 1, p + 2
    return 2 * (24 * n1 ** 4 + 4 * (q * n1 ** 3 + q * q * n1 * n1 + q ** 3 * n1) + q ** 3 + 3 * n1 ** 3)


def run_kpoint(args):
    """Bloch ChFSI at one wavevector (binary64, complex Hermitian H~(k)): the
    8^3-cell p = 6 FCC box of the profiling case, N = 200 (+20) complex bands,
    degree 40; seconds per iteration (difference of 3- and 1-iteration solves,
    so the start block's CholGS / RR are excluded) and the roofline of the
    Bloch matrix-free apply against the binary64 rate."""
    import torch
    from paper_1903_10959_gb300 import Context, workloads as W
    s = W.fcc_periodic(ncell=8, p=6, L=15.0, n_fcc=2, n_want=200, degree=40, iters=3, block=220)
    kvec = [0.11, 0.07, 0.03]
    stream = torch.cuda.current_stream()
    ctx = Context(s.ncell, s.L, s.p, periodic=True, stream=stream)
    ctx.set_potential_gaussians(s.centres, s.depths, s.widths)
    ctx.build()
    ctx.set_kpoint(kvec)
    M, n = ctx.ndofs, s.n_sub
    b = ctx.bounds_kpoint(20, s.seed)
    re = torch.tensor(W.start_block(s.seed, M, n), device="cuda")
    im = torch.tensor(W.start_block(s.seed + 1, M, n), device="cuda")
    X0 = torch.complex(re, im)
    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    ctx.solve_kpoint(X0.clone(), 1, s.degree, b)                     # warm-up
    t1 = ev_seconds(stream, lambda: ctx.solve_kpoint(X0.clone(), 1, s.degree, b))
    t3 = ev_seconds(stream, lambda: ctx.solve_kpoint(X0.clone(), 3, s.degree, b))
    Y = torch.empty_like(X0)
    reps = max(3, args.steps)
    ctx.apply_kpoint(X0, Y)
    t_apply = ev_seconds(stream, lambda: [ctx.apply_kpoint(X0, Y) for _ in range(reps)]) / reps
    # BF16x3 filter (binary64 CholGS / RR): T~_e = H~_e + 1/2 |k|^2 A~ per cell and
    # the shared G~ on the tensor cores, binary32 column pairs
    Xb = X0.clone()
    ctx.solve_kpoint(Xb, 1, s.degree, b, prec="bf16x3")             # warm-up, packs
    m1 = ev_seconds(stream, lambda: ctx.solve_kpoint(X0.clone(), 1, s.degree, b, prec="bf16x3"))
    m3 = ev_seconds(stream, lambda: ctx.solve_kpoint(X0.clone(), 3, s.degree, b, prec="bf16x3"))
    X32 = X0.to(torch.complex64)
    Y32 = torch.empty_like(X32)
    ctx.apply_kpoint_mixed(X32, Y32)
    t_mixed = ev_seconds(stream, lambda: [ctx.apply_kpoint_mixed(X32, Y32) for _ in range(reps)]) / reps
    clk = clocks.stop()
    flops = s.ncell ** 3 * n * mfk_flops_per_cell(s.p)
    achieved = flops / t_apply / 1e12
    peak, note = dtype_peak("fp64", load_peaks())
    per_iter = (t3 - t1) / 2
    ne = (s.p + 1) ** 3
    mflops = s.ncell ** 3 * n * 8 * ne * ne          # complex n_e x n_e block per cell and band
    bpeak, bnote = dtype_peak("bf16x3", load_peaks())
    line = {
        "metric": "Bloch ChFSI s/iter (binary64, one k-point)", "value": per_iter, "unit": "s/iter",
        "n_gpus": 1, "steps": 2, "warmup": 1, "ms_per_step": per_iter * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "fcc-periodic 8^3 cells p=6 L=15, %d unknowns, 32 Gaussian wells, k = %s "
                               "bohr^-1, N=%d complex bands (+%d buffer), Chebyshev degree %d"
                               % (M, kvec, s.n_want, s.n_buffer, s.degree)},
        "solve_s": {"iters_1": t1, "iters_3": t3},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": None, "kernel": "mfk_cell_fp64_kernel (+ assembly)",
                     "avg_apply_ms": t_apply * 1e3, "flops_per_apply": flops,
                     "peak_note": note + "; achieved = executed Bloch sum-factorised flops (mfk_flops_per_cell) "
                                         "per application of H~(k) to the block / event time"},
        "bf16x3": {"s_per_iter": (m3 - m1) / 2, "solve_s": {"iters_1": m1, "iters_3": m3},
                   "apply_ms": t_mixed * 1e3,
                   "roofline": {"bound": "tensor", "achieved": mflops / t_mixed / 1e12, "peak": bpeak,
                                "unit": "TFLOP/s", "frac": mflops / t_mixed / 1e12 / bpeak,
                                "traffic": None,
                                "kernel": "tc_cell_bf16_rings_kernel (Bloch pairs) + tc_assemble_kernel",
                                "flops_per_apply": mflops,
                                "peak_note": bnote + "; achieved = algorithmic N_c 8 n_e^2 flops per complex "
                                                     "band (one complex n_e x n_e block per cell) / event time "
                                                     "of the whole application (cell products + assembly)"}},
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    ctx.destroy()


# ------------------------------------------------------------------ batching
def run_batch(args):
    """64 uneven Dirichlet systems (p = 5): the batched Chebyshev filter (one
    persistent launch per degree step for all systems, CUDA graph, autotuned
    tile) against filtering the systems one after another, and one batched
    ChFSI iteration (binary32 filter, binary64 CholGS/RR per system)."""
    import torch
    from paper_1903_10959_gb300 import Batch, Context, workloads as W
    systems = W.batched_systems()
    stream = torch.cuda.current_stream()
    ctxs, X, bnd = [], [], []
    for s in systems:
        c = Context(s.ncell, s.L, s.p, periodic=False, stream=stream)
        c.set_potential_gaussians(s.centres, s.depths, s.widths)
        c.build()
        x = torch.empty((c.ndofs, s.n_sub), dtype=torch.float32, device="cuda")
        c.fill_uniform(x, s.seed, prec="mixed")
        ctxs.append(c)
        X.append(x)
        bnd.append(c.bounds(20, s.seed))
    bnd = np.array(bnd)
    a, a0 = 0.2 * bnd, np.full(len(bnd), -3.0)
    m = systems[0].degree
    ne = (systems[0].p + 1) ** 3
    flops = sum(s.ncell ** 3 * 2 * ne * ne * s.n_sub for s in systems) * m
    bt = Batch(ctxs, stream=stream)
    choice, cand_ms = bt.autotune(X, prec="mixed")
    cands = bt.candidates()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / 1e3 / reps

    clocks = ClockSampler(int(os.environ.get("LOCAL_RANK", "0")))
    clocks.start()
    t_batch_tf = timed(lambda: bt.filter(X, m, a, bnd, a0, prec="mixed"), args.steps)
    t_batch = timed(lambda: bt.filter(X, m, a, bnd, a0, prec="bf16x3"), args.steps)

    def seq(prec):
        for c, x, ai, bi, a0i in zip(ctxs, X, a, bnd, a0):
            c.filter(x, m, float(ai), float(bi), float(a0i), prec=prec)
    t_seq = timed(lambda: seq("bf16x3"), args.steps)
    t_seq_tf = timed(lambda: seq("mixed"), args.steps)
    X64 = []
    for c, s, x in zip(ctxs, systems, X):            # fresh start blocks (the filtered ones are
        x64 = torch.empty(x.shape, dtype=torch.float64, device="cuda")   # nearly rank-deficient)
        c.fill_uniform(x64, s.seed + 1, prec="fp64")
        X64.append(x64)
    evs = bt.solve(X64, 1, m, bnd * 1.02)           # warm-up of the per-system solver state
    t_solve = timed(lambda: bt.solve(X64, 1, m, bnd * 1.02), 1)
    t_solve_mixed = timed(lambda: bt.solve(X64, 1, m, bnd * 1.02, orth_prec="mixed"), 1)
    t_solve_bf = timed(lambda: bt.solve(X64, 1, m, bnd * 1.02, filter_prec="bf16x3",
                                        orth_prec="bf16x3"), 1)
    clk = clocks.stop()
    peaks = load_peaks()
    tf32_peak, tf32_note = dtype_peak("mixed", peaks)
    bf16_peak, bf16_note = dtype_peak("bf16x3", peaks)
    achieved = flops / t_batch / 1e12
    achieved_tf = flops / t_batch_tf / 1e12
    line = {
        "metric": "batched Chebyshev filter aggregate TFLOP/s (64 Dirichlet systems, p=5)",
        "value": achieved, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_batch * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "bf16x3", "data": "synthetic",
        "config": {"workload": "64 Dirichlet Gaussian-well systems, 4-12 cells per side, p=5, "
                               "h=1.5, N log-uniform 16-400, degree %d" % m,
                   "unknowns_total": int(sum(c.ndofs for c in ctxs)),
                   "columns_total": int(sum(s.n_sub for s in systems))},
        "autotune": {"choice": cands[choice], "candidates_ms": {"%d/%d" % c: round(float(t), 3)
                                                                 for c, t in zip(cands, cand_ms)}},
        "filter_s_batched": t_batch, "filter_s_sequential": t_seq,
        "speedup_vs_sequential": t_seq / t_batch,
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": achieved / bf16_peak, "traffic": None,
                     "kernel": "tc_cell_bf16_rings_kernel<2, true> (multi-system) + tc_assemble_batched_kernel",
                     "peak_note": bf16_note + "; algorithmic flops N_c 2 n_e^2 per vector over the whole "
                                  "filter (cell + assembly launches)",
                     "executed_mma": {"passes_per_flop": 6, "frac_of_peak": 6 * achieved / bf16_peak}},
        "tf32x3": {"filter_s_batched": t_batch_tf, "filter_s_sequential": t_seq_tf,
                   "speedup_vs_sequential": t_seq_tf / t_batch_tf,
                   "roofline": {"bound": "tensor", "achieved": achieved_tf, "peak": tf32_peak,
                                "unit": "TFLOP/s", "frac": achieved_tf / tf32_peak,
                                "kernel": "autotuned TF32 batched cell kernel",
                                "peak_note": tf32_note}},
        "batched_chfsi_iteration_s": t_solve,
        "batched_chfsi_iteration_s_tf32x3_orth": t_solve_mixed,
        "batched_chfsi_iteration_s_bf16x3": t_solve_bf,
        "clocks": clk,
    }
    del evs
    print(json.dumps(line), flush=True)
    bt.destroy()
    for c in ctxs:
        c.destroy()


def main():
    args = parse()
    if args.workload == "serving" and args.impl != "reference":
        run_serving(args)
        return
    if args.workload == "kpoint" and args.impl != "reference":
        run_kpoint(args)
        return
    if args.workload == "batch" and args.impl != "reference":
        run_batch(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
