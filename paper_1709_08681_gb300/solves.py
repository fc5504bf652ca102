"""Solves per second of a small workload: many independent intervals.

The plain-method case ("vla27_l1ch": 27 antennas, one channel, 60 time steps
over +-1 h, 21,060 visibilities per interval) is latency-bound on a GPU, so
its throughput is counted in solves.  ``run`` draws ``n_draws`` sets of true
offsets and noise on the workload's one geometry and sky (one model grid and
one uvw array shared by every context), simulates each interval with the GPU
predictor, and times with CUDA events

* one batched solve of all draws (one persistent fused launch per LM
  iteration over all of them, graph-replayed), and
* the same draws solved one at a time,

both plain Levenberg-Marquardt from zero offsets.  It reports solves/s, the
mean LM iterations and the RMS error against the true offsets.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi
from . import inputs as I
from .session import Session


def run(name="vla27_l1ch", n_draws=64, seed=0, stream=None, n_single=16):
    stream = stream if stream is not None else torch.cuda.current_stream()
    wl = I.make_workload(name, seed=seed)
    base = Session(wl, stream=stream)
    t0, nt = wl.intervals[0]
    row = wl.n_bl * 3 * 8
    ctxs, vis, truth = [], [], []
    for k in range(n_draws):
        c = _abi.Context(wl.n_ant, nt, wl.n_chan, base.uvw.data_ptr() + t0 * row, wl.freq_hz, wl.ap_kind,
                         wl.diam_m, wl.alpha_per_dlambda, wl.decorrelation, wl.image.shape[0], wl.n_grid,
                         wl.cell_rad, wl.support, wl.oversample, base.grid.data_ptr(), stream)
        lm = I.true_offsets(wl.n_ant, wl.sigma_pt, seed, 1000 + k)
        v = torch.empty((nt, wl.n_bl, wl.n_chan), dtype=torch.complex64, device=base.device)
        c.psc_predict(lm, v)
        v += torch.from_numpy(I.complex_noise(v.shape, wl.sigma_noise, seed, 2000 + k)).to(base.device)
        ctxs.append(c)
        vis.append(v)
        truth.append(lm)
    w_scale = [1.0 / wl.sigma_noise ** 2] * n_draws
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    _abi.psc_solve_batch(ctxs, vis, None, w_scale=w_scale)          # warm
    torch.cuda.synchronize()
    e0.record(stream)
    sols, reps = _abi.psc_solve_batch(ctxs, vis, None, w_scale=w_scale)
    e1.record(stream)
    torch.cuda.synchronize()
    t_batch = e0.elapsed_time(e1) / 1e3
    ctxs[0].psc_solve_offsets(vis[0], None, w_scale[0])            # warm
    torch.cuda.synchronize()
    e0.record(stream)
    single = [ctxs[k].psc_solve_offsets(vis[k], None, w_scale[k]) for k in range(n_single)]
    e1.record(stream)
    torch.cuda.synchronize()
    t_single = e0.elapsed_time(e1) / 1e3
    rms = [float(np.sqrt(np.mean((sols[k] - truth[k]) ** 2)) / I.ARCSEC) for k in range(n_draws)]
    out = {
        "workload": name, "n_vis_per_interval": int(nt * wl.n_bl * wl.n_chan), "n_draws": n_draws,
        "solves_per_s_batched": n_draws / t_batch, "batched_s": t_batch,
        "solves_per_s_single": n_single / t_single, "single_ms_per_solve": 1e3 * t_single / n_single,
        "mean_lm_iters": float(np.mean([r.n_iter for r in reps])),
        "mean_lm_iters_single": float(np.mean([r.n_iter for _, r in single])),
        "rms_err_arcsec_median": float(np.median(rms)),
        "within_1arcsec": float(np.mean(np.asarray(rms) <= 1.0)),
        "init": "zero (plain LM)",
    }
    for c in ctxs:
        c.close()
    base.close()
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(run()))
