"""Benchmark: batched BDF cell-solves per second on GB300.

Workload (default, one GPU): synthetic element- and charge-balanced network of
150 species / 1500 reactions (seed 1150), 16,384 cells with n_H log-uniform
[1e2, 1e6] cm^-3, T U[10, 300] K, A_V U[0, 20], G0 = 1, zeta = 1.3e-17 s^-1
(seed 7), initial abundances H2 0.5, He 0.1, C+ 1e-4, O 3e-4, N 7.5e-5,
e- = C+, others 1e-20; integrated 0 -> 1 Myr at rtol 1e-4, atol 1e-20 in
plain FP64. One step = one solve of the whole batch.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                    [--cells C] [--only fp64|mixed] [--no-e2e] [--no-cpu-baseline]

(--cells / --only / --no-e2e shrink the run for profiler captures; the default
run is the benchmark.)

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
FP64_PEAK_TFLOPS = 1.25  # nominal GB300 FP64 (152 SMs x 2 FMA/clk x 2.07 GHz); 1.19 measured by FMA chains


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


def flush_l2(buf):
    buf.add_(1.0)


# ------------------------------------------------------------------ oracle timing

_NET_CACHE = {}


def _oracle_worker(args):
    S, R, phis, x0 = args
    from oracle import bdf
    if (S, R) not in _NET_CACHE:
        _NET_CACHE[(S, R)] = synth.make_network(S, R)
    net = _NET_CACHE[(S, R)]
    for phi in phis:
        bdf.solve_cell(net, phi, x0, 0.0, T_END, RTOL, ATOL)
    return len(phis)


def time_oracle(n_cells, cores):
    """Oracle cell-solves/s on `cores` host processes over a seeded sample."""
    net = synth.make_network(S_SP, R_RX)
    x0 = synth.initial_abundances(net)
    phis = synth.cells(CELLS)[:n_cells]
    chunks = [(S_SP, R_RX, phis[i::cores], x0) for i in range(cores)]
    ctx = mp.get_context("spawn")
    env_before = os.environ.get("OPENBLAS_NUM_THREADS")
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    try:
        with ctx.Pool(cores) as pool:
            pool.map(_oracle_worker, [(S_SP, R_RX, phis[:1], x0)] * cores)  # import + warm
            t = time.perf_counter()
            done = sum(pool.map(_oracle_worker, chunks))
            dt = time.perf_counter() - t
    finally:
        if env_before is None:
            os.environ.pop("OPENBLAS_NUM_THREADS", None)
        else:
            os.environ["OPENBLAS_NUM_THREADS"] = env_before
    return done / dt, dt


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
        v, _ = time_oracle(n, cores)
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
    R_two = int(np.sum(net.rtype == synth.TWO_BODY))
    R_one = net.n_reactions - R_two
    n_nu = int(sum(np.sum(net.reac >= 0, axis=1)) + sum(np.sum(net.prod >= 0, axis=1)))
    allphi = synth.cells(CELLS * ws)
    phi_h = np.ascontiguousarray(allphi[rank * CELLS:(rank + 1) * CELLS])
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

    # ---- FP64 (headline)
    with ClockSampler(local) as clk:
        ms64 = timed(carbox.CBX_FP64, args.steps, args.warmup) if args.only != "mixed" else [float("nan")]
    st64 = carbox.stats_dict(stats.cpu().numpy())
    ok64 = int((status == 0).sum().item())
    t_local = sum(ms64) / 1e3
    t_max = t_local
    if ws > 1:
        tt = torch.tensor([t_local], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    value = ws * CELLS * args.steps / t_max
    ms_per_step = 1e3 * t_max / args.steps
    lat = (st64["t_end_ns"] - st64["t_begin_ns"]) / 1e6
    fl = algorithmic_flops(info, st64, R_two, R_one, n_nu)
    fp64_flops = fl["lu"] + fl["solve"] + fl["rhs"] + fl["jac"]
    achieved = fp64_flops / (ms_per_step / 1e3) / 1e12

    # ---- mixed precision, same workload
    if args.only == "fp64":
        print(json.dumps({"only": "fp64", "cells": CELLS, "ms_per_step": ms_per_step, "value": value}), flush=True)
        return
    msmx = timed(carbox.CBX_MIXED, max(1, args.steps), 1 if args.only != "mixed" else args.warmup)
    if args.only == "mixed":
        print(json.dumps({"only": "mixed", "cells": CELLS, "ms_per_step": sum(msmx) / len(msmx),
                          "value": CELLS * len(msmx) / (sum(msmx) / 1e3)}), flush=True)
        return
    stmx = carbox.stats_dict(stats.cpu().numpy())
    okmx = int((status == 0).sum().item())
    mixed_value = CELLS * len(msmx) / (sum(msmx) / 1e3)
    latmx = (stmx["t_end_ns"] - stmx["t_begin_ns"]) / 1e6

    # ---- end to end through the host-buffer C-ABI call (copies inside the timed region)
    opt = carbox.options(rtol=RTOL, atol=ATOL, precision=carbox.CBX_FP64)
    e2e_steps = max(1, min(args.steps, 2)) if not args.no_e2e else 0
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        xh, sh, _ = carbox.solve_host(N, phi_h, x0_h.reshape(S_SP, CELLS), 0.0, T_END, opt, stream=stream)
    barrier()
    e2e_t = max(time.perf_counter() - t0, 1e-9)
    e2e_value = ws * CELLS * e2e_steps / e2e_t if ws == 1 and e2e_steps else None
    if ws > 1:
        tt = torch.tensor([e2e_t], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        e2e_value = ws * CELLS * e2e_steps / float(tt.item())

    if rank != 0:
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        ncell = max(cores, args.ref_cells)
        v, dt = time_oracle(ncell, cores)
        cpu = {"value": v, "unit": "cell-solves/s", "cores": cores, "kind": "oracle",
               "sample": f"first {ncell} of the {CELLS} seeded cells, spawn pool of {cores} processes, {dt:.1f} s"}
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
                  "ms_per_step": sum(msmx) / len(msmx), "speedup_vs_fp64": mixed_value / (value / ws),
                  "cells_ok": okmx, "cell_p50_ms": float(np.percentile(latmx, 50)),
                  "cell_p99_ms": float(np.percentile(latmx, 99)),
                  "mean_refine_sweeps_per_newton": float(stmx["refine_sweeps"].sum() / max(1, stmx["newton_iters"].sum()))},
        "counters_per_cell": {k: float(st64[k].mean()) for k in carbox.STATS_FIELDS},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": achieved / FP64_PEAK_TFLOPS, "traffic": traffic,
                     "kernel": "solve_kernel<double> (FP64 pipe)",
                     "flops_per_launch": fp64_flops, "flop_split": {k: v for k, v in fl.items()}},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "cell-solves/s",
                "h2d_bytes_per_step": int(phi_h.nbytes + x0_h.nbytes),
                "d2h_bytes_per_step": int(x0_h.nbytes + CELLS * 4)},
        "gpu_launches": args.steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
