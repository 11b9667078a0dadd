"""Parity helpers for the GPU tests: oracle runs in a spawn pool and the gate.

Gate (per cell, species above 1e-12 per n_H):
  * twin parity: the GPU result within 1e-4 relative of the oracle run with
    the same algorithm, constants and tolerances; else
  * converged gate: against an oracle reference at rtol 1e-8 (atol 1e-26),
    the GPU's error is at most twice the oracle's own error at the working
    tolerance. This is the case where a rounding-level difference flipped a
    threshold decision of the step controller, so that the two runs follow
    different, equally valid step programs; the GPU result must then be as
    accurate as the oracle's, with no absolute floor.

The pool is started with the ``spawn`` method (a process forked after CUDA
has been initialised can hang), one worker per host core, one BLAS thread each.
"""
from __future__ import annotations

import multiprocessing as mp
import os

import numpy as np

TOL = 1e-4
FLOOR = 1e-12
TIGHT = (1e-8, 1e-26)


def _worker(args):
    net, phi, x0, t_end, rtol, atol, track, method = args
    from oracle import bdf, esdirk
    mod = esdirk if method == "esdirk" else bdf
    if track is None:
        return mod.solve_cell(net, phi, x0, 0.0, t_end, rtol, atol).x
    return mod.solve_cell_track(net, track, x0, 0.0, t_end, rtol, atol).x


def oracle_cells(net, phis, x0s, t_end, rtol=1e-4, atol=1e-20, tracks=None, method="bdf"):
    """Oracle results [S, n] for cells phis[i] (or tracks[i]) with x0s[:, i],
    by the BDF (method "bdf") or the ESDIRK ("esdirk") oracle."""
    n = len(phis) if tracks is None else len(tracks)
    jobs = [(net, None if tracks is not None else np.asarray(phis[i]), np.asarray(x0s[:, i]), t_end, rtol, atol,
             None if tracks is None else np.asarray(tracks[i]), method) for i in range(n)]
    old = {k: os.environ.get(k) for k in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS")}
    os.environ["OPENBLAS_NUM_THREADS"] = os.environ["OMP_NUM_THREADS"] = "1"
    try:
        with mp.get_context("spawn").Pool(max(1, min(n, os.cpu_count() or 1))) as pool:
            out = pool.map(_worker, jobs)
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return np.stack(out, axis=1)


def max_rel(x, ref, floor=FLOOR):
    big = ref > floor
    return float(np.max(np.abs(x[big] / ref[big] - 1))) if big.any() else 0.0


def gate(x_gpu, ref, net, phis, x0s, t_end, tracks=None):
    """Apply the gate to every cell (columns); returns a per-cell report.

    Raises AssertionError naming the first cell that fails."""
    twin = [max_rel(x_gpu[:, c], ref[:, c]) for c in range(ref.shape[1])]
    flipped = [c for c, r in enumerate(twin) if not r <= TOL]
    report = {"cells": len(twin), "within_tol": len(twin) - len(flipped), "max_twin": max(twin),
              "converged_gate": []}
    if flipped:
        tight = oracle_cells(net, None if phis is None else [phis[c] for c in flipped], x0s[:, flipped], t_end,
                             *TIGHT, tracks=None if tracks is None else [tracks[c] for c in flipped])
        for k, c in enumerate(flipped):
            big = tight[:, k] > FLOOR
            e_gpu = float(np.max(np.abs(x_gpu[big, c] / tight[big, k] - 1)))
            e_orc = float(np.max(np.abs(ref[big, c] / tight[big, k] - 1)))
            report["converged_gate"].append({"cell": c, "twin": twin[c], "err_gpu": e_gpu, "err_oracle": e_orc})
            assert e_gpu <= 2.0 * e_orc, (c, twin[c], e_gpu, e_orc)
    return report
