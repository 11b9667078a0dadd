"""Benchmark: batched BDF cell-solves per second on GB300.

Workload (default, one GPU): synthetic element- and charge-balanced network of
150 species / 1500 reactions (seed 1150), 16,384 cells with n_H log-uniform
[1e2, 1e6] cm^-3, T U[10, 300] K, A_V U[0, 20], G0 = 1, zeta = 1.3e-17 s^-1
(seed 7), initial abundances H2 0.5, He 0.1, C+ 1e-4, O 3e-4, N 7.5e-5,
e- = C+, others 1e-20; integrated 0 -> 1 Myr at rtol 1e-4, atol 1e-20 in
plain FP64. One step = one solve of the whole batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--cells C] [--only fp64|mixed] [--no-e2e] [--no-cpu-baseline]
                    [--no-large] [--no-extras] [--config large|adjoint|serving|zeta|track|peaks]

(--cells / --only / --no-e2e / --no-large / --no-extras shrink the run for
profiler captures; the default run is the benchmark.)

Besides the headline (FP64) the default line carries: the mixed-precision
path on the same cells; the measured FP64 and FP32 FMA peaks (the library's
probe kernel, run in this job) that the ALU rooflines divide by; 500 species /
6000 reactions in both precisions on the same 4,096 cells with the per-species
error against the FP64 oracle; the oracle parity sample with the converged
gate for cells on another step program; and compact runs of the adjoint
(1,024 cells, 1e5 yr), serving (Poisson requests at 200/s), time-dependent
environment tracks and the cosmic-ray sweep with sensitivities, all under the
same clock record.

With N > 1 (torchrun) each rank solves its own 16,384 cells of a batch of
N x 16,384 (weak scaling, no collective on the data path); the barrier and the
max over ranks are the only communication. ``--impl reference`` times the CPU
oracle (the plain FP64 restatement of the method) on the host cores.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2511_10558_gb300 import synth  # noqa: E402

METRIC = "cell-solves/s to 1 Myr at rtol 1e-4 (150/500 sp), FP64 vs mixed; p50/p99 latency"
S_SP, R_RX = 150, 1500
CELLS = 16384  # per GPU (overridden by --cells for profiler captures)
T_END = 1e6 * synth.YEAR
RTOL, ATOL = 1e-4, 1e-20
FP64_NOMINAL_TFLOPS = 1.26  # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (used only if the probe fails)
FP32_NOMINAL_TFLOPS = 80.5  # 152 SMs x 128 FP32 FMA/clk x 2 flop x 2.07 GHz (used only if the probe fails)


# ------------------------------------------------------------------ helpers

def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def network_counts(net):
    """(two-body reactions, one-body reactions, stoichiometric entries) of a network."""
    R_two = int(np.sum(net.rtype == synth.TWO_BODY))
    n_nu = int(sum(np.sum(net.reac >= 0, axis=1)) + sum(np.sum(net.prod >= 0, axis=1)))
    return R_two, net.n_reactions - R_two, n_nu


def algorithmic_flops(info, st, R_two, R_one, n_nu):
    """FP64 (and FP32) flops of the method for the given per-cell counters.

    Per unit: LU = F_LU of the symbolic fill; a triangular-solve pair =
    2 nnz(L+U); right-hand side = 2 R_two + R_one (rates) + n_nu (gather);
    Jacobian = 2 R_two + n_terms (approximated by 2 n_nu); refinement sweep =
    2 nnz(J) (FP64 residual) + 2 nnz(L+U) (FP32 solve).
    """
    lu = st["lu_factors"].astype(np.float64).sum() * info["lu_flops"]
    solve = st["newton_iters"].astype(np.float64).sum() * 2.0 * info["nnz_lu"]
    rhs = st["rhs_evals"].astype(np.float64).sum() * (2.0 * R_two + R_one + n_nu)
    jac = st["jac_evals"].astype(np.float64).sum() * (2.0 * R_two + 2.0 * n_nu)
    ref = st["refine_sweeps"].astype(np.float64).sum()
    return {"lu": lu, "solve": solve, "rhs": rhs, "jac": jac,
            "refine_fp64": ref * 2.0 * info["nnz_jac"], "refine_fp32": ref * 2.0 * info["nnz_lu"]}


def mixed_flops(info, st, R_two, R_one, n_nu):
    """(FP32, FP64) flops of the mixed path: the LU and every triangular-solve
    pair (the first solve of each Newton iteration and each refinement sweep)
    in FP32; rates, right-hand sides, Jacobians and the refinement residuals
    in FP64."""
    fl = algorithmic_flops(info, st, R_two, R_one, n_nu)
    sweeps = st["refine_sweeps"].astype(np.float64).sum()
    fp32 = fl["lu"] + fl["solve"] + sweeps * 2.0 * info["nnz_lu"]
    fp64 = fl["rhs"] + fl["jac"] + fl["refine_fp64"]
    return fp32, fp64


def measure_fma_peaks(carbox, dev, stream):
    """FP64 and FP32 FMA peaks (TFLOP/s, best of 3 launches) from the library's
    probe kernel: 8 CTAs of 256 threads per SM, 8 independent FMA chains each."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    grid, block = sms * 8, 256
    sink = torch.zeros(grid, dtype=torch.float64, device=dev)
    out = {"how": f"cbx_peak_fma: {grid} CTAs x {block} threads x 8 dependent-FMA chains, best of 3, CUDA events"}
    for name, fp64, iters in (("fp64", 1, 40000), ("fp32", 0, 2000000)):
        flops = carbox.lib.cbx_peak_fma_flops(grid, block, iters)
        best = 0.0
        for _ in range(4):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc = carbox.lib.cbx_peak_fma(fp64, grid, block, iters, carbox.C.c_void_p(stream.cuda_stream),
                                         carbox.C.c_void_p(sink.data_ptr()))
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if rc != 0:
                return None
            best = max(best, flops / (e0.elapsed_time(e1) / 1e3) / 1e12)
        out[name + "_tflops"] = best
    return out


def _oracle_job(args):
    net, phi, x0, t_end, rtol, atol = args
    from oracle import bdf
    return bdf.solve_cell(net, phi, x0, 0.0, t_end, rtol, atol).x


def oracle_map(net, phis, x0, t_end, rtol=RTOL, atol=ATOL):
    """Oracle results [S, n] for the cells phis (x0 shared), one spawn process per host core."""
    ctx = mp.get_context("spawn")
    n = len(phis)
    os.environ["OPENBLAS_NUM_THREADS"] = os.environ["OMP_NUM_THREADS"] = "1"
    with ctx.Pool(max(1, min(n, os.cpu_count() or 1))) as pool:
        out = pool.map(_oracle_job, [(net, phis[i], x0, t_end, rtol, atol) for i in range(n)])
    return np.stack(out, axis=1)


def flush_l2(buf):
    buf.add_(1.0)


def shard_cells(global_phi, rank, per_rank):
    """A rank's contiguous block of the global batch (weak scaling: per_rank cells each)."""
    return np.ascontiguousarray(global_phi[rank * per_rank:(rank + 1) * per_rank])


def max_over_ranks(seconds, device):
    """The slowest rank's time: an all-reduce (MAX) when a process group is up."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def weak_value(world, per_rank, steps, t_max):
    """Whole-job cell-solves/s: every rank solved per_rank cells per step."""
    return world * per_rank * steps / t_max


# ------------------------------------------------------------------ oracle timing

_NET_CACHE = {}


def _oracle_worker(args):
    S, R, idx, phis, x0 = args
    from oracle import bdf
    if (S, R) not in _NET_CACHE:
        _NET_CACHE[(S, R)] = synth.make_network(S, R)
    net = _NET_CACHE[(S, R)]
    return [(i, bdf.solve_cell(net, phi, x0, 0.0, T_END, RTOL, ATOL).x) for i, phi in zip(idx, phis)]


def time_oracle(n_cells, cores):
    """Oracle cell-solves/s on `cores` host processes over a seeded sample (the
    first n_cells cells), with the sample's results [S, n_cells]."""
    net = synth.make_network(S_SP, R_RX)
    x0 = synth.initial_abundances(net)
    phis = synth.cells(CELLS)[:n_cells]
    idx = np.arange(n_cells)
    chunks = [(S_SP, R_RX, idx[i::cores], phis[i::cores], x0) for i in range(cores)]
    ctx = mp.get_context("spawn")
    env_before = os.environ.get("OPENBLAS_NUM_THREADS")
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_worker, [(S_SP, R_RX, idx[:1], phis[:1], x0)] * cores)  # import + warm
            t = time.perf_counter()
            parts = pool.map(_oracle_worker, chunks)
            dt = time.perf_counter() - t
    finally:
        if env_before is None:
            os.environ.pop("OPENBLAS_NUM_THREADS", None)
        else:
            os.environ["OPENBLAS_NUM_THREADS"] = env_before
    xs = np.empty((S_SP, n_cells))
    for part in parts:
        for i, x in part:
            xs[:, i] = x
    return n_cells / dt, dt, xs


def parity_summary(x_gpu, x_ref, tol=1e-4, floor=1e-12, tight=None):
    """Per sampled cell, the largest relative difference over species above
    `floor`; how many cells are within `tol`. tight: {cell: rtol-1e-8 oracle
    result} for the cells outside tol, which then get the converged gate (the
    GPU's error against that reference at most twice the oracle's own)."""
    rel = []
    for c in range(x_ref.shape[1]):
        big = x_ref[:, c] > floor
        rel.append(float(np.max(np.abs(x_gpu[big, c] / x_ref[big, c] - 1))) if big.any() else 0.0)
    rel = np.array(rel)
    out = {"cells": int(rel.size), "tol": tol, "within_tol": int((rel <= tol).sum()),
           "max_rel": float(rel.max()), "median_rel": float(np.median(rel)), "converged_gate": []}
    for c, ref8 in (tight or {}).items():
        big = ref8 > floor
        e_gpu = float(np.max(np.abs(x_gpu[big, c] / ref8[big] - 1)))
        e_orc = float(np.max(np.abs(x_ref[big, c] / ref8[big] - 1)))
        out["converged_gate"].append({"cell": int(c), "twin_rel": float(rel[c]), "err_gpu_vs_rtol1e-8": e_gpu,
                                      "err_oracle_vs_rtol1e-8": e_orc, "pass": e_gpu <= 2.0 * e_orc})
    out["all_pass_gate"] = bool(all(g["pass"] for g in out["converged_gate"]) and
                                out["within_tol"] + len(out["converged_gate"]) == out["cells"])
    return out


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return
    cores = os.cpu_count() or 1
    n = max(cores, args.ref_cells)
    vals = []
    for _ in range(args.warmup if args.warmup < 1 else 1):
        time_oracle(cores, cores)
    for _ in range(args.steps):
        v, _, _ = time_oracle(n, cores)
        vals.append(v)
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "cell-solves/s", "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n / v,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"{S_SP} species / {R_RX} reactions, {CELLS} cells, 1 Myr, rtol 1e-4, "
                                   f"atol 1e-20, FP64 (each step a {n}-cell seeded sample)",
                       "cells_per_step": n},
            "cpu_baseline": {"value": v, "unit": "cell-solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"first {n} of the {CELLS} seeded cells per step, spawn pool of {cores}"},
            "e2e": {"value": v, "unit": "cell-solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    global CELLS
    CELLS = args.cells
    import torch
    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2511_10558_gb300 import build
    if rank == 0:
        build.build()
    if ws > 1:
        torch.distributed.barrier()
    from paper_2511_10558_gb300 import carbox

    net = synth.make_network(S_SP, R_RX)
    N = carbox.Network.from_synth(net)
    info = N.info()
    R_two, R_one, n_nu = network_counts(net)
    phi_h = shard_cells(synth.cells(CELLS * ws), rank, CELLS)
    x0_h = np.ascontiguousarray(np.repeat(synth.initial_abundances(net)[:, None], CELLS, axis=1))
    phi = torch.tensor(phi_h, device=dev)
    x0 = torch.tensor(x0_h, device=dev)
    x_out = torch.empty_like(x0)
    status = torch.empty(CELLS, dtype=torch.int32, device=dev)
    stats = carbox.stats_tensor(CELLS, dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream(dev)

    def step(prec):
        carbox.solve(N, phi, x0, 0.0, T_END, carbox.options(rtol=RTOL, atol=ATOL, precision=prec), stream=stream,
                     x_out=x_out, status=status, stats=stats)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def timed(prec, steps, warmup):
        for _ in range(warmup):
            step(prec)
        barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for k in range(steps):
            flush_l2(flush)
            ev[k][0].record(stream)
            step(prec)
            ev[k][1].record(stream)
        barrier()
        ms = [a.elapsed_time(b) for a, b in ev]
        return ms

    # ---- measured FMA peaks (the ALU roofline denominators), before the timed work
    peaks = None
    if rank == 0 and not args.no_peaks:
        with ClockSampler(local) as clk_peaks:
            peaks = measure_fma_peaks(carbox, dev, stream)
        if peaks is not None:
            peaks["clocks"] = clk_peaks.summary()
    fp64_peak = peaks["fp64_tflops"] if peaks else FP64_NOMINAL_TFLOPS
    fp32_peak = peaks["fp32_tflops"] if peaks else FP32_NOMINAL_TFLOPS
    peak_src = "measured in this run (FMA-chain probe)" if peaks else "nominal (probe unavailable)"

    # ---- FP64 (headline)
    with ClockSampler(local) as clk:
        ms64 = timed(carbox.CBX_FP64, args.steps, args.warmup) if args.only != "mixed" else [float("nan")]
    st64 = carbox.stats_dict(stats.cpu().numpy())
    ok64 = int((status == 0).sum().item())
    n_sample = min(CELLS, max(args.ref_cells, os.cpu_count() or 1))  # the oracle sample (cpu_baseline)
    x64_sample = x_out[:, :n_sample].cpu().numpy()
    t_max = max_over_ranks(sum(ms64) / 1e3, dev)
    value = weak_value(ws, CELLS, args.steps, t_max)
    ms_per_step = 1e3 * t_max / args.steps
    lat = (st64["t_end_ns"] - st64["t_begin_ns"]) / 1e6
    fl = algorithmic_flops(info, st64, R_two, R_one, n_nu)
    fp64_flops = fl["lu"] + fl["solve"] + fl["rhs"] + fl["jac"]
    achieved = fp64_flops / (ms_per_step / 1e3) / 1e12

    # ---- mixed precision, same workload
    if args.only == "fp64":
        print(json.dumps({"only": "fp64", "cells": CELLS, "ms_per_step": ms_per_step, "value": value}), flush=True)
        return
    with ClockSampler(local) as clk_mx:
        msmx = timed(carbox.CBX_MIXED, max(1, args.steps), 1 if args.only != "mixed" else args.warmup)
    if args.only == "mixed":
        print(json.dumps({"only": "mixed", "cells": CELLS, "ms_per_step": sum(msmx) / len(msmx),
                          "value": CELLS * len(msmx) / (sum(msmx) / 1e3)}), flush=True)
        return
    stmx = carbox.stats_dict(stats.cpu().numpy())
    okmx = int((status == 0).sum().item())
    xmx_sample = x_out[:, :n_sample].cpu().numpy()
    ms_mx = sum(msmx) / len(msmx)
    mixed_value = CELLS * len(msmx) / (sum(msmx) / 1e3)
    latmx = (stmx["t_end_ns"] - stmx["t_begin_ns"]) / 1e6
    f32, f64mx = mixed_flops(info, stmx, R_two, R_one, n_nu)
    ach32, ach64mx = f32 / (ms_mx / 1e3) / 1e12, f64mx / (ms_mx / 1e3) / 1e12

    # ---- 500 species / 6000 reactions (matrix in the CTAs' global workspace)
    large = None
    if not args.no_large and ws == 1:
        with ClockSampler(local) as clk_l:
            large = run_large_throughput(carbox, dev, stream, 4096, errors=rank == 0 and not args.no_cpu_baseline,
                                         peaks=peaks)
        large["clocks"] = clk_l.summary()

    # ---- end to end through the host-buffer C-ABI call (copies inside the timed region)
    opt = carbox.options(rtol=RTOL, atol=ATOL, precision=carbox.CBX_FP64)
    e2e_steps = max(1, min(args.steps, 2)) if not args.no_e2e else 0
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        xh, sh, _ = carbox.solve_host(N, phi_h, x0_h.reshape(S_SP, CELLS), 0.0, T_END, opt, stream=stream)
    barrier()
    e2e_t = max(time.perf_counter() - t0, 1e-9)
    e2e_value = weak_value(ws, CELLS, e2e_steps, max_over_ranks(e2e_t, dev)) if e2e_steps else None

    if rank != 0:
        return
    cpu = parity = None
    if ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        ncell = n_sample
        v, dt, x_ref = time_oracle(ncell, cores)
        cpu = {"value": v, "unit": "cell-solves/s", "cores": cores, "kind": "oracle",
               "sample": f"first {ncell} of the {CELLS} seeded cells, spawn pool of {cores} processes, {dt:.1f} s"}
        # cells outside 1e-4 in either precision get the converged gate (rtol-1e-8 oracle reference)
        out_tol = sorted(set(c for xs in (x64_sample, xmx_sample) for c in range(ncell)
                             if parity_summary(xs[:, c:c + 1], x_ref[:, c:c + 1])["within_tol"] == 0))
        tight = {}
        if out_tol:
            phis = synth.cells(CELLS)[out_tol]
            refs = oracle_map(net, phis, synth.initial_abundances(net), T_END, 1e-8, 1e-26)
            tight = {c: refs[:, k] for k, c in enumerate(out_tol)}
        parity = {}
        for name, xs in (("fp64", x64_sample), ("mixed", xmx_sample)):
            t_sub = {c: r for c, r in tight.items()
                     if parity_summary(xs[:, c:c + 1], x_ref[:, c:c + 1])["within_tol"] == 0}
            parity[name] = parity_summary(xs[:, :ncell], x_ref, tight=t_sub)
    extras = None
    if ws == 1 and not args.no_extras:
        blocks = (("adjoint", lambda: adjoint_block(carbox, dev, stream, n_checks=1)),
                  ("serving", lambda: serving_block(carbox, rate=200.0, duration=0.25)),
                  ("track", lambda: track_block(carbox, dev, stream, n_checks=1)),
                  ("zeta", lambda: zeta_block(carbox, dev, stream, n_checks=1)),
                  ("esdirk", lambda: esdirk_block(carbox, dev, stream)),
                  ("hmc", lambda: hmc_block(carbox, dev, stream)))
        extras = {}
        with ClockSampler(local) as clk_x:
            for name, run in blocks:
                try:
                    extras[name] = run()
                except Exception as exc:  # one failed side run must not lose the headline line
                    extras[name] = {"error": f"{type(exc).__name__}: {exc}"}
                    torch.cuda.synchronize(dev)
        extras["clocks"] = clk_x.summary()
    prof = os.path.join(ROOT, "profiles", "traffic.json")
    traffic = None
    if os.path.exists(prof):
        tr = json.load(open(prof)).get("solve_kernel_fp64_150")
        if tr and tr.get("kernel_hash") == build.source_hash():
            traffic = tr["dram_bytes_per_cell"] * CELLS
    line = {
        "metric": METRIC, "value": value, "unit": "cell-solves/s", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{S_SP} species / {R_RX} reactions (synthetic, seed 1150), {CELLS} cells per GPU, "
                               "0 -> 1 Myr, rtol 1e-4, atol 1e-20, FP64",
                   "cells_per_gpu": CELLS, "global_cells": CELLS * ws, "l2": "flushed (256 MB write) between steps",
                   "parallelism": f"cells sharded over {ws} GPU(s)"},
        "latency_ms": {"cell_p50": float(np.percentile(lat, 50)), "cell_p99": float(np.percentile(lat, 99)),
                       "batch_p50": float(np.percentile(ms64, 50)), "batch_max": float(max(ms64))},
        "cells_ok": ok64,
        "mixed": {"value": mixed_value, "unit": "cell-solves/s", "dtype": "f64 state + f32 LU",
                  "ms_per_step": ms_mx, "speedup_vs_fp64": mixed_value / (value / ws),
                  "cells_ok": okmx, "cell_p50_ms": float(np.percentile(latmx, 50)),
                  "cell_p99_ms": float(np.percentile(latmx, 99)),
                  "mean_refine_sweeps_per_newton": float(stmx["refine_sweeps"].sum() / max(1, stmx["newton_iters"].sum())),
                  "roofline": {"bound": "alu", "kernel": "solve_kernel<float> (FP32 LU and solves, FP64 rest)",
                               "fp32": {"achieved": ach32, "peak": fp32_peak, "unit": "TFLOP/s",
                                        "frac": ach32 / fp32_peak, "flops_per_launch": f32},
                               "fp64": {"achieved": ach64mx, "peak": fp64_peak, "unit": "TFLOP/s",
                                        "frac": ach64mx / fp64_peak, "flops_per_launch": f64mx},
                               "peak_source": peak_src},
                  "clocks": clk_mx.summary()},
        "large_500": large,
        "counters_per_cell": {k: float(st64[k].mean()) for k in carbox.STATS_FIELDS},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp64_peak, "traffic": traffic, "peak_source": peak_src,
                     "kernel": "solve_kernel<double> (FP64 pipe)",
                     "flops_per_launch": fp64_flops, "flop_split": {k: v for k, v in fl.items()}},
        "peaks": peaks,
        "cpu_baseline": cpu,
        "parity_sample": parity,
        "e2e": {"value": e2e_value, "unit": "cell-solves/s",
                "h2d_bytes_per_step": int(phi_h.nbytes + x0_h.nbytes),
                "d2h_bytes_per_step": int(x0_h.nbytes + CELLS * 4)},
        "configs": extras,
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def _gpu_setup():
    import torch
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    from paper_2511_10558_gb300 import build
    build.build()
    from paper_2511_10558_gb300 import carbox
    return torch, dev, carbox


def run_large_throughput(carbox, dev, stream, cells, errors=True, n_err=4, peaks=None):
    """500 species / 6000 reactions, 1 Myr: mixed and FP64 cell-solves/s on the same
    `cells` seeded cells (one timed step each), each with its roofline (the
    method's flops from the per-cell counters over the FMA peaks: `peaks` as
    measured by measure_fma_peaks, else nominal), and (errors) the per-species
    relative error of both against the FP64 oracle on the first n_err cells
    (species above 1e-12), with element and charge conservation."""
    import torch
    net = synth.make_network(500, 6000)
    N = carbox.Network.from_synth(net)
    info = N.info()
    counts = network_counts(net)
    fp64_peak = peaks["fp64_tflops"] if peaks else FP64_NOMINAL_TFLOPS
    fp32_peak = peaks["fp32_tflops"] if peaks else FP32_NOMINAL_TFLOPS
    peak_src = "measured in this run (FMA-chain probe)" if peaks else "nominal (probe not run)"
    phi_h = synth.cells(cells)
    x0_h = np.repeat(synth.initial_abundances(net)[:, None], cells, axis=1)
    phi = torch.tensor(phi_h, device=dev)
    x0 = torch.tensor(x0_h, device=dev).contiguous()
    out = {"workload": f"500 species / 6000 reactions (seed 1500), {cells} cells (the same for both precisions), "
                       "1 Myr, rtol 1e-4, atol 1e-20"}
    xs = {}
    for name, prec in [("mixed", carbox.CBX_MIXED), ("fp64", carbox.CBX_FP64)]:
        st = carbox.stats_tensor(cells, dev)
        o = carbox.options(rtol=RTOL, atol=ATOL, precision=prec)
        carbox.solve(N, phi[:152].contiguous(), x0[:, :152].contiguous(), 0.0, T_END, o, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, status, _ = carbox.solve(N, phi, x0, 0.0, T_END, o, stream=stream, stats=st)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        sd = carbox.stats_dict(st.cpu().numpy())
        lat = (sd["t_end_ns"] - sd["t_begin_ns"]) / 1e6
        xs[name] = x[:, :n_err].cpu().numpy()
        out[name] = {"cells": cells, "ms": ms, "value": cells / (ms / 1e3), "unit": "cell-solves/s",
                     "cells_ok": int((status == 0).sum().item()), "cell_p50_ms": float(np.percentile(lat, 50)),
                     "cell_p99_ms": float(np.percentile(lat, 99)),
                     "steps_per_cell": float(sd["steps"].mean()), "lu_per_cell": float(sd["lu_factors"].mean()),
                     "refine_sweeps_per_newton": float(sd["refine_sweeps"].sum() / max(1, sd["newton_iters"].sum()))}
        sec = ms / 1e3
        if name == "fp64":
            fl = algorithmic_flops(info, sd, *counts)
            tot = float(sum(fl.values()))
            out[name]["roofline"] = {"bound": "alu", "kernel": "solve_kernel<double, GM> (FP64 pipe)",
                                     "achieved": tot / sec / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                                     "frac": tot / sec / 1e12 / fp64_peak, "flops_per_launch": tot,
                                     "lu_share_of_flops": float(fl["lu"]) / tot, "peak_source": peak_src}
        else:
            f32, f64 = (float(v) for v in mixed_flops(info, sd, *counts))
            out[name]["roofline"] = {"bound": "alu", "kernel": "solve_kernel<float, GM> (FP32 LU and solves, FP64 rest)",
                                     "fp32": {"achieved": f32 / sec / 1e12, "peak": fp32_peak, "unit": "TFLOP/s",
                                              "frac": f32 / sec / 1e12 / fp32_peak, "flops_per_launch": f32},
                                     "fp64": {"achieved": f64 / sec / 1e12, "peak": fp64_peak, "unit": "TFLOP/s",
                                              "frac": f64 / sec / 1e12 / fp64_peak, "flops_per_launch": f64},
                                     "peak_source": peak_src}
    # the roofline counts F_LU of the symbolic fill; the global-memory LU
    # factors the whole matrix (lu_flops_dense per factorisation)
    out["lu_fill"] = {"nnz_lu": int(info["nnz_lu"]), "dense_fraction": info["nnz_lu"] / 500.0 ** 2,
                      "lu_flops": float(info["lu_flops"]), "lu_flops_dense": float(info["lu_flops_dense"])}
    out["mixed_speedup_vs_fp64"] = out["mixed"]["value"] / out["fp64"]["value"]
    if errors:
        ref = oracle_map(net, phi_h[:n_err], x0_h[:, 0], T_END)
        E = np.vstack([net.composition.T, net.charge[None, :]]).astype(float)
        e0 = E @ x0_h[:, 0]
        den = np.where(np.arange(E.shape[0]) == E.shape[0] - 1, np.abs(net.charge) @ x0_h[:, 0], e0)
        for name in ("mixed", "fp64"):
            rel, cons = [], 0.0
            for c in range(n_err):
                big = ref[:, c] > 1e-12
                rel.append(np.abs(xs[name][big, c] / ref[big, c] - 1))
                cons = max(cons, float(np.max(np.abs(E @ xs[name][:, c] - e0) / den)))
            r = np.concatenate(rel)
            out[name]["error_vs_fp64_oracle"] = {"cells": n_err, "species_values": int(r.size), "max": float(r.max()),
                                                 "median": float(np.median(r)), "p99": float(np.percentile(r, 99)),
                                                 "max_conservation_rel": cons}
    return out


def run_large(args):
    """Config 3 alone: 500 species, mixed vs FP64 on the same 4,096 cells, errors vs the FP64 oracle."""
    torch, dev, carbox = _gpu_setup()
    stream = torch.cuda.current_stream(dev)
    cells = args.cells if args.cells != 16384 else 4096
    print(json.dumps({"config": "large", **run_large_throughput(carbox, dev, stream, cells,
                                                                errors=not args.no_cpu_baseline)}), flush=True)


def run_adjoint(args):
    """Config 4 alone, with gradient checks on two cells (oracle adjoint and finite differences)."""
    torch, dev, carbox = _gpu_setup()
    print(json.dumps(adjoint_block(carbox, dev, torch.cuda.current_stream(dev), n_checks=2, fd=True)), flush=True)


def adjoint_block(carbox, dev, stream, n_checks=1, fd=False):
    """Config 4: 150 sp, 1024 cells, 1e5 yr; forward (recorded) and adjoint times;
    gradient checks on `n_checks` cells against the oracle adjoint of the GPU's
    program (and, fd, central finite differences of its exact replay)."""
    import torch
    from oracle import adjoint as adj
    net = synth.make_network(S_SP, R_RX)
    N = carbox.Network.from_synth(net)
    C = 1024
    t_end = 1e5 * synth.YEAR
    phi_h = synth.cells(C, seed=7)
    x0_h = np.repeat(synth.initial_abundances(net)[:, None], C, axis=1)
    phi = torch.tensor(phi_h, device=dev)
    x0 = torch.tensor(x0_h, device=dev).contiguous()
    tape = carbox.Tape(N, C, 2000)
    o = carbox.options(rtol=RTOL, atol=ATOL, precision=carbox.CBX_FP64)
    carbox.solve_record(N, tape, phi, x0, 0.0, t_end, o)   # warm-up
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    x, st = carbox.solve_record(N, tape, phi, x0, 0.0, t_end, o)
    e[1].record(stream)
    torch.cuda.synchronize()
    # loss: 10 seeded targets per cell (species above 1e-12 at t_f), targets +-0.5 dex
    xh = x.cpu().numpy()
    rng = np.random.default_rng(11)
    cot = np.zeros_like(xh)
    targets = []
    for c in range(C):
        cand = np.flatnonzero(xh[:, c] > 1e-12)
        tg = np.sort(rng.choice(cand, size=min(10, len(cand)), replace=False))
        yt = np.log10(xh[tg, c]) + rng.uniform(-0.5, 0.5, len(tg))
        targets.append((tg, yt))
        cot[:, c] = adj.log10_loss(xh[:, c], tg, yt)[1]
    cot_d = torch.tensor(cot, device=dev).contiguous()
    carbox.grad(tape, cot_d, C)  # warm-up
    torch.cuda.synchronize()
    e[2].record(stream)
    ga, gn, gt = carbox.grad(tape, cot_d, C)
    e[3].record(stream)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    gn_h, gt_h = gn.cpu().numpy(), gt.cpu().numpy()
    # checks on sampled cells: oracle adjoint of the GPU program, and central FD (step 1e-6)
    cells_checked = [0, 517][:n_checks]
    checks = []
    for c in cells_checked:
        prog = []
        for kind, q, v in tape.program(c):
            prog.append(("init", v) if kind == 0 else ("rescale", q, v) if kind == 1 else ("step", q, v, 0.0, None))
        tg, yt = targets[c]
        xr, prog_r = adj.replay(net, phi_h[c], x0_h[:, c], prog)
        _, cr = adj.log10_loss(xr, tg, yt)
        g = adj.adjoint(net, phi_h[c], x0_h[:, c], prog_r, cr)
        chk = {"cell": c, "rel_err_lnnH_vs_oracle_adjoint": abs(gn_h[c] / g[1] - 1),
               "rel_err_T_vs_oracle_adjoint": abs(gt_h[c] / g[2] - 1)}
        checks.append(chk)
        if not fd:
            continue
        eps = 1e-6
        pp, pm = phi_h[c].copy(), phi_h[c].copy()
        pp[0] *= np.exp(eps)
        pm[0] *= np.exp(-eps)
        fd_nH = (adj.log10_loss(adj.replay(net, pp, x0_h[:, c], prog)[0], tg, yt)[0] -
                 adj.log10_loss(adj.replay(net, pm, x0_h[:, c], prog)[0], tg, yt)[0]) / (2 * eps)
        pp, pm = phi_h[c].copy(), phi_h[c].copy()
        pp[1] += eps * phi_h[c, 1]
        pm[1] -= eps * phi_h[c, 1]
        fd_T = (adj.log10_loss(adj.replay(net, pp, x0_h[:, c], prog)[0], tg, yt)[0] -
                adj.log10_loss(adj.replay(net, pm, x0_h[:, c], prog)[0], tg, yt)[0]) / (2 * eps * phi_h[c, 1])
        chk.update({"rel_err_lnnH_vs_fd": abs(gn_h[c] / fd_nH - 1), "rel_err_T_vs_fd": abs(gt_h[c] / fd_T - 1)})
    res = {"config": "adjoint", "workload": f"{S_SP} species / {R_RX} reactions, {C} cells, 0 -> 1e5 yr, FP64, "
                                             "loss = sum over 10 seeded targets of (log10 x - y)^2",
           "forward_record_ms": fwd_ms, "adjoint_ms": bwd_ms, "backward_over_forward": bwd_ms / fwd_ms,
           "cells_ok": int((st == 0).sum().item()), "gradients": "ln alpha [1500] summed over cells, ln n_H [1024], T [1024]",
           "checks": checks}
    return res


def run_zeta(args):
    """The cosmic-ray sweep alone, with checks on three cells (oracle adjoint and finite differences)."""
    torch, dev, carbox = _gpu_setup()
    print(json.dumps(zeta_block(carbox, dev, torch.cuda.current_stream(dev), n_checks=3, fd=True)), flush=True)


def zeta_block(carbox, dev, stream, n_checks=1, fd=False):
    """Cosmic-ray sweep with sensitivities (synthetic analog of the paper's zeta study,
    Sec. 4 / Fig. 2): 150 sp, the reference cell (n_H 1e4, T 20 K, A_V 5, G0 1) at C
    values of zeta / zeta_0 log-spaced over [1e-2, 1e4], 0 -> 1e7 yr, FP64 forward with
    recording, then the adjoint of L = log10 x_e(t_f) per cell: d log10 x_e / d ln zeta
    (and d/d ln G0, d/dA_V, d/d ln n_H, d/dT) for every cell of the sweep."""
    import torch
    from oracle import adjoint as adj
    net = synth.make_network(S_SP, R_RX)
    N = carbox.Network.from_synth(net)
    C = 1024
    t_end = 1e7 * synth.YEAR
    ratio = 10.0 ** np.linspace(-2.0, 4.0, C)
    phi_h = np.repeat(synth.one_cell(), C, axis=0)
    phi_h[:, 4] = synth.ZETA0 * ratio
    x0_h = np.repeat(synth.initial_abundances(net)[:, None], C, axis=1)
    phi = torch.tensor(phi_h, device=dev).contiguous()
    x0 = torch.tensor(x0_h, device=dev).contiguous()
    tape = carbox.Tape(N, C, 3000)
    o = carbox.options(rtol=RTOL, atol=ATOL, precision=carbox.CBX_FP64)
    carbox.solve_record(N, tape, phi, x0, 0.0, t_end, o)   # warm-up
    torch.cuda.synchronize()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    x, st = carbox.solve_record(N, tape, phi, x0, 0.0, t_end, o)
    e[1].record(stream)
    torch.cuda.synchronize()
    xh = x.cpu().numpy()
    ie = net.index("e-")
    cot = np.zeros_like(xh)
    cot[ie, :] = 1.0 / (xh[ie, :] * np.log(10.0))   # L = log10 x_e
    cot_d = torch.tensor(cot, device=dev).contiguous()
    carbox.grad_env(tape, cot_d, C)  # warm-up
    torch.cuda.synchronize()
    e[2].record(stream)
    ga, gn, gt, gz, gg, gav = carbox.grad_env(tape, cot_d, C)
    e[3].record(stream)
    torch.cuda.synchronize()
    fwd_ms, bwd_ms = e[0].elapsed_time(e[1]), e[2].elapsed_time(e[3])
    gz_h = gz.cpu().numpy()
    # checks where the sensitivity is not saturated (|g| >= 0.1 of its largest
    # value; at high zeta this synthetic network is fully ionised and the
    # derivative is zero to rounding, where relative errors mean nothing)
    live = np.flatnonzero(np.abs(gz_h) >= 0.1 * np.abs(gz_h).max())
    checks = []
    for c in sorted({int(np.argmax(np.abs(gz_h))), int(live[0]), int(live[-1])})[:n_checks]:
        prog = []
        for kind, q, v in tape.program(c):
            prog.append(("init", v) if kind == 0 else ("rescale", q, v) if kind == 1 else ("step", q, v, 0.0, None))
        xr, prog_r = adj.replay(net, phi_h[c], x0_h[:, c], prog)
        cr = np.zeros(S_SP)
        cr[ie] = 1.0 / (xr[ie] * np.log(10.0))
        g = adj.adjoint(net, phi_h[c], x0_h[:, c], prog_r, cr)
        z_ref = adj.environment_gradients(net, g[0])[0]
        chk = {"cell": c, "zeta_over_zeta0": float(ratio[c]), "dlog10xe_dlnzeta": float(gz_h[c]),
               "rel_err_vs_oracle_adjoint": abs(gz_h[c] / z_ref - 1)}
        checks.append(chk)
        if not fd:
            continue
        eps = 1e-6
        pp, pm = phi_h[c].copy(), phi_h[c].copy()
        pp[4] *= np.exp(eps)
        pm[4] *= np.exp(-eps)
        fd = (np.log10(adj.replay(net, pp, x0_h[:, c], prog)[0][ie]) -
              np.log10(adj.replay(net, pm, x0_h[:, c], prog)[0][ie])) / (2 * eps)
        chk["rel_err_vs_fd"] = abs(gz_h[c] / fd - 1)
    ok = st.cpu().numpy() == 0
    grid = [0, C // 4, C // 2, 3 * C // 4, C - 1]
    res = {"config": "zeta", "workload": f"{S_SP} species / {R_RX} reactions, {C} cells, zeta/zeta0 log-spaced in "
                                          "[1e-2, 1e4], reference cell otherwise, 0 -> 1e7 yr, FP64; L = log10 x_e",
           "forward_record_ms": fwd_ms, "adjoint_ms": bwd_ms, "cells_ok": int(ok.sum()),
           "cell_solves_per_s_with_gradients": C / ((fwd_ms + bwd_ms) / 1e3),
           "x_e": {f"{ratio[c]:.3g}": float(xh[ie, c]) for c in grid},
           "sensitive_range_zeta_over_zeta0": [float(ratio[live[0]]), float(ratio[live[-1]])],
           "dlog10xe_dlnzeta": {f"{ratio[c]:.3g}": float(gz_h[c]) for c in grid},
           "checks": checks}
    return res


def run_track(args):
    """The time-dependent environment run alone, with two cells checked against the oracle."""
    torch, dev, carbox = _gpu_setup()
    print(json.dumps(track_block(carbox, dev, torch.cuda.current_stream(dev), n_checks=2)), flush=True)


def track_block(carbox, dev, stream, n_checks=1):
    """Time-dependent environment phi(t) (the generalised system of Sec. 2 with phi a function
    of time): 150 sp, 4096 seeded cells, each on a collapse-and-warming track (n_H x10, T x1.5,
    A_V +5 mag over 1 Myr, 4 knots); FP64 and mixed cell-solves/s next to the same cells at
    constant phi, and sampled cells against the oracle's solve_cell_track."""
    import torch
    from oracle import bdf
    net = synth.make_network(S_SP, R_RX)
    N = carbox.Network.from_synth(net)
    C = 4096
    phi_h = synth.cells(C)
    tr_h = synth.tracks(phi_h, T_END)
    x0_h = np.repeat(synth.initial_abundances(net)[:, None], C, axis=1)
    phi = torch.tensor(phi_h, device=dev).contiguous()
    tr = torch.tensor(tr_h, device=dev).contiguous()
    x0 = torch.tensor(x0_h, device=dev).contiguous()
    res = {"config": "track", "workload": f"{S_SP} species / {R_RX} reactions, {C} cells, 0 -> 1 Myr, rtol 1e-4, "
                                          "atol 1e-20; tracks: n_H x10 (geometric), T x1.5, A_V +5 mag, 4 knots"}
    for name, prec in (("fp64", carbox.CBX_FP64), ("mixed", carbox.CBX_MIXED)):
        o = carbox.options(rtol=RTOL, atol=ATOL, precision=prec)
        out = {}
        for kind in ("track", "constant"):
            run = (lambda: carbox.solve_track(N, tr, x0, 0.0, T_END, o)) if kind == "track" else \
                  (lambda: carbox.solve(N, phi, x0, 0.0, T_END, o))
            run()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, st, _ = run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            out[kind] = {"ms": ms, "value": C / (ms / 1e3), "unit": "cell-solves/s",
                         "cells_ok": int((st == 0).sum().item())}
            if kind == "track":
                xt = x.cpu().numpy()
        out["track_over_constant_time"] = out["track"]["ms"] / out["constant"]["ms"]
        res[name] = out
        if name == "fp64":
            checks = []
            for c in [0, 7][:n_checks]:
                ref = bdf.solve_cell_track(net, tr_h[c], x0_h[:, c], 0.0, T_END, RTOL, ATOL).x
                big = ref > 1e-12
                checks.append({"cell": c, "max_rel_vs_oracle": float(np.max(np.abs(xt[big, c] / ref[big] - 1)))})
            res["checks_fp64"] = checks
    return res


def esdirk_block(carbox, dev, stream, n_err=3):
    """ESDIRK 4(3) of Kvaerno's family (the paper's kind of solver) next to the BDF on the
    same 4,096 cells of the 150-species network, 1 Myr, FP64 and mixed; and both methods'
    error against an rtol-1e-8 oracle reference on n_err cells (cross-method parity)."""
    import torch
    net = synth.make_network(S_SP, R_RX)
    N = carbox.Network.from_synth(net)
    C = 4096
    phi_h = synth.cells(C)
    x0_h = np.repeat(synth.initial_abundances(net)[:, None], C, axis=1)
    phi = torch.tensor(phi_h, device=dev).contiguous()
    x0 = torch.tensor(x0_h, device=dev).contiguous()
    res = {"config": "esdirk", "workload": f"{S_SP} species / {R_RX} reactions, {C} cells, 0 -> 1 Myr, rtol 1e-4, "
                                           "atol 1e-20; ESDIRK 4(3) (5 stages, L-stable) vs BDF, same cells"}
    xs = {}
    for method, mname in ((carbox.CBX_METHOD_ESDIRK, "esdirk"), (carbox.CBX_METHOD_BDF, "bdf")):
        for prec, pname in ((carbox.CBX_FP64, "fp64"), (carbox.CBX_MIXED, "mixed")):
            o = carbox.options(rtol=RTOL, atol=ATOL, precision=prec, method=method)
            carbox.solve(N, phi[:152].contiguous(), x0[:, :152].contiguous(), 0.0, T_END, o, stream=stream)
            st = carbox.stats_tensor(C, dev)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x, status, _ = carbox.solve(N, phi, x0, 0.0, T_END, o, stream=stream, stats=st)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            sd = carbox.stats_dict(st.cpu().numpy())
            res[f"{mname}_{pname}"] = {"ms": ms, "value": C / (ms / 1e3), "unit": "cell-solves/s",
                                       "cells_ok": int((status == 0).sum().item()),
                                       "steps_per_cell": float(sd["steps"].mean()),
                                       "lu_per_cell": float(sd["lu_factors"].mean()),
                                       "rhs_per_cell": float(sd["rhs_evals"].mean())}
            if pname == "fp64":
                xs[mname] = x[:, :n_err].cpu().numpy()
    tight = oracle_map(net, phi_h[:n_err], x0_h[:, 0], T_END, 1e-8, 1e-26)
    errs = {}
    for m in ("esdirk", "bdf"):
        e = []
        for c in range(n_err):
            big = tight[:, c] > 1e-12
            e.append(float(np.max(np.abs(xs[m][big, c] / tight[big, c] - 1))))
        errs[m] = e
    res["error_vs_rtol1e-8_oracle"] = {"cells": n_err, **errs}
    return res


def hmc_block(carbox, dev, stream, transitions=4, leapfrog=4):
    """Rate-uncertainty sampling (HMC over ln alpha, the posterior gradient from one recorded
    solve and the discrete adjoint): 150 species, 64 cells, 1e5 yr, 5 target species per
    cell; time per transition and per posterior-gradient evaluation."""
    import torch
    from paper_2511_10558_gb300 import hmc
    net = synth.make_network(S_SP, R_RX)
    N = carbox.Network.from_synth(net)
    C = 64
    t_end = 1e5 * synth.YEAR
    phi = torch.tensor(synth.cells(C, seed=31), device=dev).contiguous()
    x0 = torch.tensor(np.repeat(synth.initial_abundances(net)[:, None], C, axis=1), device=dev).contiguous()
    theta0 = np.log(net.alpha)
    rng = np.random.default_rng(5)
    theta_true = theta0 + 0.2 * rng.standard_normal(net.n_reactions)
    xt, _ = carbox.solve_with_alpha(N, torch.tensor(np.exp(theta_true), device=dev), phi, x0, 0.0, t_end)
    xt = xt.cpu().numpy()
    targets = np.array([np.sort(rng.choice(np.flatnonzero(xt[:, c] > 1e-10), 5, replace=False)) for c in range(C)])
    y = np.log10(xt[targets, np.arange(C)[:, None]])
    post = hmc.RatePosterior(N, phi, x0, t_end, targets, y, 0.1, 0.5, theta0)
    U, g = post(theta0)
    t0 = time.perf_counter()
    U, g = post(theta0)
    t_eval = time.perf_counter() - t0
    th, acc_n = theta0.copy(), 0
    rng2 = np.random.default_rng(9)
    t0 = time.perf_counter()
    for _ in range(transitions):
        th, U, g, acc, dH = hmc.hmc_step(th, U, g, post, 1e-3, leapfrog, rng2)
        acc_n += int(acc)
    dt = time.perf_counter() - t0
    return {"config": "hmc", "workload": f"{S_SP} species / {R_RX} reactions, {C} cells, 0 -> 1e5 yr, FP64; "
                                         f"theta = ln alpha [{net.n_reactions}], 5 targets per cell, sigma 0.1 dex, "
                                         f"prior sd 0.5; {transitions} transitions of {leapfrog} leapfrog steps",
            "s_per_posterior_gradient": t_eval, "s_per_transition": dt / transitions,
            "accepted": acc_n, "transitions": transitions, "final_U": float(U)}


def run_serving(args):
    """Config 5 alone, at the given rate and duration of arrivals."""
    torch, dev, carbox = _gpu_setup()
    print(json.dumps(serving_block(carbox, args.rate, args.duration)), flush=True)


def serving_block(carbox, rate, duration):
    """Config 5: Poisson requests over 32/150/500-species networks through cbx_server."""
    import threading
    nets = {}
    for S, R in [(32, 200), (150, 1500), (500, 6000)]:
        net = synth.make_network(S, R)
        nets[S] = (net, carbox.Network.from_synth(net))
    rng = np.random.default_rng(13)
    n_req = max(1, int(rng.poisson(rate * duration)))
    arrivals = np.sort(rng.uniform(0.0, duration, n_req))
    reqs = []
    for k in range(n_req):
        S = int(rng.choice([32, 150, 500]))
        C = int(np.clip(np.round(np.exp(rng.uniform(0.0, np.log(4096.0)))), 1, 4096))
        t_end = 10.0 ** rng.uniform(3.0, 7.0) * synth.YEAR
        phi = synth.cells(C, seed=1000 + k)
        x0 = np.repeat(synth.initial_abundances(nets[S][0])[:, None], C, axis=1)
        reqs.append((arrivals[k], S, phi, x0, t_end))
    opt = carbox.options(rtol=RTOL, atol=ATOL, precision=carbox.CBX_MIXED)
    srv = carbox.Server(mem_budget=64 << 30, n_streams=8, max_ctas=76)
    ids = [None] * n_req
    t0 = time.perf_counter()

    def submitter():
        for k, (ta, S, phi, x0, t_end) in enumerate(reqs):
            d = ta - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            ids[k] = srv.submit(nets[S][1], phi, x0, 0.0, t_end, opt)

    th = threading.Thread(target=submitter)
    th.start()
    th.join()
    lat, cells, ok = [], 0, 0
    for k in range(n_req):
        x, st, (ts, tb, td) = srv.wait(ids[k])
        lat.append(td - ts)
        cells += len(st)
        ok += int((st == 0).sum())
    wall = time.perf_counter() - t0
    stats = srv.stats()
    srv.close()
    lat = np.array(lat)
    by = {}
    for S in (32, 150, 500):
        sel = np.array([r[1] == S for r in reqs])
        if sel.any():
            by[str(S)] = {"requests": int(sel.sum()), "p50_s": float(np.percentile(lat[sel], 50)),
                          "p99_s": float(np.percentile(lat[sel], 99))}
    res = {"config": "serving", "workload": f"Poisson arrivals at {rate}/s for {duration} s; networks "
           "32/150/500 species uniform; cells log-uniform 1..4096; spans log-uniform 1e3..1e7 yr; mixed precision",
           "requests": n_req, "cells": cells, "cells_ok": ok, "wall_s": wall,
           "throughput_cells_per_s": cells / wall, "throughput_requests_per_s": n_req / wall,
           "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
           "by_network": by, "server": {"mem_budget": 64 << 30, "streams": 8, "max_ctas": 76, **stats}}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="carbox", choices=["carbox", "reference"])
    ap.add_argument("--ref-cells", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cells", type=int, default=16384)
    ap.add_argument("--only", choices=["fp64", "mixed"], default=None)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-large", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the compact config 4/5, track and zeta runs")
    ap.add_argument("--no-peaks", action="store_true", help="skip the FMA peak probe (nominal peaks)")
    ap.add_argument("--config", choices=["bench", "large", "adjoint", "serving", "zeta", "track", "peaks", "esdirk",
                                         "hmc"], default="bench")
    ap.add_argument("--duration", type=float, default=2.0, help="serving: seconds of Poisson arrivals")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: mean requests per second")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == "large":
        run_large(args)
    elif args.config == "adjoint":
        run_adjoint(args)
    elif args.config == "serving":
        run_serving(args)
    elif args.config == "zeta":
        run_zeta(args)
    elif args.config == "track":
        run_track(args)
    elif args.config in ("esdirk", "hmc"):
        torch, dev, carbox = _gpu_setup()
        blk = esdirk_block if args.config == "esdirk" else hmc_block
        print(json.dumps(blk(carbox, dev, torch.cuda.current_stream(dev))), flush=True)
    elif args.config == "peaks":
        torch, dev, carbox = _gpu_setup()
        with ClockSampler(0) as clk:
            pk = measure_fma_peaks(carbox, dev, torch.cuda.current_stream(dev))
        print(json.dumps({"config": "peaks", **(pk or {}), "clocks": clk.summary()}), flush=True)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
