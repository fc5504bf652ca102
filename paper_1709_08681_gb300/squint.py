"""Beam squint from the two parallel-hand polarisations solved separately.

Each antenna's R and L beams point at the mechanical offset displaced by
plus and minus half of a squint vector.  The two polarisations' visibilities
are simulated with their own offsets and independent noise, and each
polarisation is solved for its own offsets, as the paper does for the two
parallel hands.  Their half-sum is the mechanical offset and their difference
is the squint.  Both polarisations of every interval run as one batch: one
persistent launch per LM iteration over 2 x the intervals.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi
from . import inputs as I
from .session import Session


def run(name="vla27_l64ch", seed=0, sigma_mech_arcsec=20.0, squint_arcsec=60.0, **over):
    wl = I.make_workload(name, seed=seed, **over)
    n_int = len(wl.intervals)
    offs = [I.squinted_offsets(wl.n_ant, sigma_mech_arcsec * I.ARCSEC, squint_arcsec * I.ARCSEC, seed, 200 + k)
            for k in range(n_int)]
    stream = torch.cuda.current_stream()
    sess_r = Session(wl, stream=stream)
    sess_l = Session(wl, stream=stream, grid=sess_r.grid)      # second set of contexts on the same data layout
    vis = []
    for pol, sess in ((2, sess_r), (3, sess_l)):
        v = sess.predict([o[pol] for o in offs])
        v += torch.from_numpy(wl.noise(10 + pol)).to(v.device)  # independent noise per polarisation
        vis.append(v)
    ctxs = sess_r.ctxs + sess_l.ctxs
    vk = [sess_r.vis_slice(vis[0], k) for k in range(n_int)] + [sess_l.vis_slice(vis[1], k) for k in range(n_int)]
    w_scale = [1.0 / wl.sigma_noise ** 2] * (2 * n_int)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sols, reps = _abi.psc_solve_batch(ctxs, vk, None, w_scale=w_scale)
    e1.record(stream)
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    mech_err, sq_err = [], []
    for k in range(n_int):
        r, l = sols[k], sols[n_int + k]
        mech_err.append(np.sqrt(np.mean((0.5 * (r + l) - offs[k][0]) ** 2)) / I.ARCSEC)
        sq_err.append(np.sqrt(np.mean(((r - l) - offs[k][1]) ** 2)) / I.ARCSEC)
    rep = {"n_intervals": n_int, "polarisations": 2, "n_vis": 2 * int(wl.n_vis), "squint_arcsec": squint_arcsec,
           "solve_s": t, "solves_per_s": 2 * n_int / t,
           "mean_lm_iters": float(np.mean([x.n_iter for x in reps])),
           "mechanical_rms_err_arcsec": float(np.max(mech_err)), "squint_rms_err_arcsec": float(np.max(sq_err))}
    sess_r.close()
    sess_l.close()
    return rep, sols, offs


if __name__ == "__main__":
    import json
    print(json.dumps(run()[0]))
