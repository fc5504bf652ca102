"""Time-varying pointing solved interval by interval with a warm start.

The pointing of every antenna drifts (``inputs.drifting_offsets``: a mean
offset plus a random walk, constant within a solution interval).  Two ways
to solve all intervals are compared on the same data:

* cold: every interval from zero offsets, all intervals as one batch (one
  persistent fused launch per LM iteration over all of them);
* warm: the intervals in time order, each starting from the previous
  interval's solution (the paper's use of earlier solutions as the initial
  guess), one solve at a time.

Both must reach the same minimiser.  ``run`` reports the LM iterations and
the CUDA-event time of each, the accuracy against the true offsets, and the
throughput of one batched evaluation over all the data.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _abi
from . import inputs as I
from . import roofline as RL
from .session import Session


def run(name="drift197_l128ch", seed=0, log=None, **over):
    t0 = time.perf_counter()
    wl = I.make_workload(name, seed=seed, **over)
    stream = torch.cuda.current_stream()
    sess = Session(wl, stream=stream)
    vis = sess.simulate()
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n_int = len(wl.intervals)
    w_scale = [1.0 / wl.sigma_noise ** 2] * n_int
    vk = [sess.vis_slice(vis, k) for k in range(n_int)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    # one batched evaluation over all intervals (graph replay), with autotuned shapes
    batch = _abi.Batch(sess.ctxs, vk, None, w_scale=w_scale, stream=stream)
    batch.psc_batch_autotune()
    zeros = [np.zeros((wl.n_ant, 2)) for _ in range(n_int)]
    batch.psc_batch_begin(zeros)
    batch.psc_batch_iterate(2)
    torch.cuda.synchronize()
    reps_t = 3
    e0.record(stream)
    for _ in range(reps_t):
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)
    e1.record(stream)
    torch.cuda.synchronize()
    t_iter = e0.elapsed_time(e1) / reps_t / 1e3
    batch.psc_batch_profile(True)
    batch.psc_batch_restart()
    batch.psc_batch_iterate(1)
    batch.psc_batch_profile(False)
    k_ms, k_n = batch.psc_batch_profile_read()
    batch.close()

    # cold: all intervals from zero, one batch
    torch.cuda.synchronize()
    e0.record(stream)
    cold, cold_reps = _abi.psc_solve_batch(sess.ctxs, vk, None, w_scale=w_scale)
    e1.record(stream)
    torch.cuda.synchronize()
    t_cold = e0.elapsed_time(e1) / 1e3

    # warm: in time order, each from the previous solution (contexts keep the
    # shapes the autotuner gave them)
    warm, warm_iters = [], []
    torch.cuda.synchronize()
    e0.record(stream)
    prev = np.zeros((wl.n_ant, 2))
    for k in range(n_int):
        sol, rep = sess.ctxs[k].psc_solve_offsets(vk[k], None, w_scale[k], lm0=prev)
        warm.append(sol)
        warm_iters.append(rep.n_iter)
        prev = sol
    e1.record(stream)
    torch.cuda.synchronize()
    t_warm = e0.elapsed_time(e1) / 1e3

    def rms(a, b):
        return float(np.sqrt(np.mean((np.asarray(a) - np.asarray(b)) ** 2)) / I.ARCSEC)

    taps = float(np.sum(RL.taps_per_channel(wl)))
    flops = sum(nt for _, nt in wl.intervals) * wl.n_bl * taps * RL.FLOPS_PER_TAP
    k_avg = k_ms / max(k_n, 1)
    rep = {
        "n_ant": wl.n_ant, "n_chan": wl.n_chan, "n_time": wl.n_time, "n_intervals": n_int, "n_vis": int(wl.n_vis),
        "t_setup_s": t_setup,
        "iteration_ms": 1e3 * t_iter, "gvis_per_s_iteration": wl.n_vis / t_iter / 1e9,
        "fused_launch_ms": k_avg, "fused_tflops": flops / (k_avg * 1e-3) / 1e12,
        "cold_batched_s": t_cold, "cold_mean_lm_iters": float(np.mean([r.n_iter for r in cold_reps])),
        "warm_sequential_s": t_warm, "warm_mean_lm_iters": float(np.mean(warm_iters)),
        "warm_vs_cold_max_arcsec": float(max(np.max(np.abs(a - b)) for a, b in zip(warm, cold)) / I.ARCSEC),
        "rms_err_arcsec_cold": float(np.median([rms(a, b) for a, b in zip(cold, wl.lm_true)])),
        "rms_err_arcsec_warm": float(np.median([rms(a, b) for a, b in zip(warm, wl.lm_true)])),
        "walk_step_arcsec": float(np.std(np.diff(wl.lm_true, axis=0)) / I.ARCSEC),
    }
    if log:
        log(rep)
    sess.close()
    return rep


if __name__ == "__main__":
    import argparse
    import json
    ap = argparse.ArgumentParser()
    ap.add_argument("--n-time", type=int, default=None, help="time steps (reduced sizes; 60 per interval)")
    ap.add_argument("--seed", type=int, default=0)
    args = ap.parse_args()
    over = {}
    if args.n_time:
        over = {"n_time": args.n_time, "n_interval": max(1, args.n_time // 60)}
    print(json.dumps(run(seed=args.seed, **over)))
