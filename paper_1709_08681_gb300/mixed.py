"""Batched solves over a mixed set of solution intervals: uneven lengths,
three array types, offsets of 10-60 arcsec with 2 arcmin outliers
(``inputs.mixed_intervals``).  All intervals run as one batch: one persistent
fused launch per LM iteration over every interval's bricks, the iteration
captured in a CUDA graph, launch shapes picked by the batch autotuner.

``run`` builds the batch, simulates the observed data on the GPU, and
measures (CUDA events on the batch's stream) the time of one batched LM
iteration and of the full solve from zero offsets; it reports visibilities
per second, intervals per second and the accuracy against the true offsets.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _abi
from . import inputs as I
from . import roofline as RL
from .session import MixedSession


def run(n_intervals=256, seed=0, t_range=(30, 600), arrays=("y27", "disk64", "disk197"), iters_timed=3,
        log=None):
    t_start = time.perf_counter()
    A = I.mixed_arrays(seed, arrays)
    ivs = I.mixed_intervals(A, n_intervals, seed, t_range)
    stream = torch.cuda.current_stream()
    sess = MixedSession(A, ivs, stream=stream)
    vis = sess.simulate()
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_start
    w_scale = [1.0 / A[iv.array].sigma_noise ** 2 for iv in ivs]
    batch = _abi.Batch(sess.ctxs, vis, None, w_scale=w_scale, stream=stream)
    t = time.perf_counter()
    tiling = batch.psc_batch_autotune()
    t_tune = time.perf_counter() - t
    zeros = [np.zeros((A[iv.array].n_ant, 2)) for iv in ivs]
    # one batched iteration (restart + iterate), graph-replayed, event-timed
    batch.psc_batch_begin(zeros)
    for _ in range(2):
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(iters_timed):
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_iter = e0.elapsed_time(e1) / iters_timed / 1e3
    batch.psc_batch_profile(True)
    batch.psc_batch_restart()
    batch.psc_batch_iterate(1)
    batch.psc_batch_profile(False)
    k_ms, k_n = batch.psc_batch_profile_read()
    batch.close()
    # full solves from zero, all intervals in one batch
    torch.cuda.synchronize()
    e0.record(stream)
    sols, reps = _abi.psc_solve_batch(sess.ctxs, vis, None, w_scale=w_scale)
    e1.record(stream)
    torch.cuda.synchronize()
    t_solve = e0.elapsed_time(e1) / 1e3
    err_in, err_out, iters, reasons = [], [], [], {}
    for k, iv in enumerate(ivs):
        d = (sols[k] - iv.lm_true) / I.ARCSEC
        mask = np.zeros(len(d), dtype=bool)
        mask[iv.outliers] = True
        err_in.append(np.sqrt(np.mean(d[~mask] ** 2)))
        if mask.any():
            err_out.append(np.max(np.abs(d[mask])))
        iters.append(reps[k].n_iter)
        r = _abi.STOP_REASONS[reps[k].reason]
        reasons[r] = reasons.get(r, 0) + 1
    n_vis = sess.n_vis()
    taps = {a: float(np.sum(RL.taps_per_channel(A[a]))) for a in arrays}
    flops = sum(iv.n_time * A[iv.array].n_bl * taps[iv.array] for iv in ivs) * RL.FLOPS_PER_TAP
    k_avg = k_ms / max(k_n, 1)
    rep = {
        "n_intervals": n_intervals, "n_vis": int(n_vis),
        "arrays": {a: sum(1 for iv in ivs if iv.array == a) for a in arrays},
        "t_range": list(t_range),
        "tiling": sorted({tuple(x) for x in tiling}),
        "t_setup_s": t_setup, "t_autotune_s": t_tune,
        "iteration_ms": 1e3 * t_iter, "gvis_per_s_iteration": n_vis / t_iter / 1e9,
        "fused_launch_ms": k_avg, "flops_per_launch": flops,
        "fused_tflops": flops / (k_avg * 1e-3) / 1e12,
        "solve_s": t_solve, "intervals_per_s": n_intervals / t_solve,
        "mean_lm_iters": float(np.mean(iters)), "max_lm_iters": int(np.max(iters)), "stop_reasons": reasons,
        "rms_err_arcsec_median": float(np.median(err_in)), "rms_err_arcsec_max": float(np.max(err_in)),
        "outlier_max_err_arcsec": float(np.max(err_out)) if err_out else None,
        "n_outliers": int(sum(len(iv.outliers) for iv in ivs)),
    }
    if log:
        log(rep)
    sess.close()
    return rep, sols


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--intervals", type=int, default=256)
    ap.add_argument("--t-min", type=int, default=30)
    ap.add_argument("--t-max", type=int, default=600)
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args()
    rep, _ = run(a.intervals, a.seed, (a.t_min, a.t_max))
    print(json.dumps(rep))
