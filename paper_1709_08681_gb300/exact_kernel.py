"""The exact disk kernel (``psc_set_kernel_model(PSC_KERNEL_EXACT_DISK)``)
on a workload: throughput of the fused evaluation with it, and the offsets it
recovers against those of the Gaussian model of Eq. AIJPOINTING, both solved
on data simulated with the exact kernel.

Data: the workload's geometry and sky, offsets drawn with ``sigma_arcsec``
(larger than the workload's own, where the models differ), visibilities
predicted by the GPU with the exact kernel plus the workload's seeded
thermal noise.  The brick shape of the exact kernel (one visibility per
thread) is chosen among a few candidates by timing one evaluation of the
first interval; the candidates include flat bricks (consecutive (channel,
time) items per block, psc_set_flat_tiling).
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi, inputs as I, roofline as RL
from .session import Session

# (t_tile, c_group) rectangles, and flat bricks of n items ("flat", n)
TILINGS = [(128, 2), (64, 4), (256, 1), (32, 8), (64, 2), ("flat", 256), ("flat", 192), ("flat", 128), ("flat", 64)]


def _apply(ctx, tl):
    if tl[0] == "flat":
        ctx.psc_set_flat_tiling(tl[1], 1)
    else:
        ctx.psc_set_tiling(tl[0], tl[1], 1)


def _eval_ms(ctx, lm, vis, w_scale, n):
    ctx.psc_profile(True)
    ctx.psc_residual_grad(lm, vis, None, w_scale)              # warm
    ctx.psc_profile_read()
    for _ in range(n):
        ctx.psc_residual_grad(lm, vis, None, w_scale)
    ms, k = ctx.psc_profile_read()
    ctx.psc_profile(False)
    return ms / max(k, 1)


def run(name="vla27_l64ch", seed=0, sigma_arcsec=60.0, n_eval=5, **over):
    wl = I.make_workload(name, seed=seed, sigma_pt_arcsec=sigma_arcsec, **over)
    sess = Session(wl)
    for ctx in sess.ctxs:
        ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)
    vis = sess.predict(wl.lm_true)
    vis += torch.from_numpy(wl.noise(5)).to(vis.device)
    w_scale = 1.0 / wl.sigma_noise ** 2
    lm_eval = [0.5 * x for x in wl.lm_true]
    # brick shape: one timed evaluation of the first interval per candidate
    best, best_ms = TILINGS[0], float("inf")
    for tl in TILINGS:
        _apply(sess.ctxs[0], tl)
        ms = _eval_ms(sess.ctxs[0], lm_eval[0], sess.vis_slice(vis, 0), w_scale, 1)
        if ms < best_ms:
            best, best_ms = tl, ms
    for ctx in sess.ctxs:
        _apply(ctx, best)
    eval_ms = sum(_eval_ms(ctx, lm_eval[k], sess.vis_slice(vis, k), w_scale, n_eval)
                  for k, ctx in enumerate(sess.ctxs))
    taps = RL.taps_per_channel(wl)
    flops = sum(nt * wl.n_bl * float(np.sum(taps)) * RL.FLOPS_PER_TAP_EXACT for _, nt in wl.intervals)
    props = torch.cuda.get_device_properties(vis.device)
    peak = RL.fp32_peak_tflops(props.multi_processor_count)
    tflops = flops / (eval_ms * 1e-3) / 1e12
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {}
    for label, model in (("exact", _abi.PSC_KERNEL_EXACT_DISK), ("gauss", _abi.PSC_KERNEL_GAUSS)):
        errs, iters = [], []
        torch.cuda.synchronize()
        e0.record()
        for k, ctx in enumerate(sess.ctxs):
            ctx.psc_set_kernel_model(model)
            _apply(ctx, best)
            sol, rep = ctx.psc_solve_offsets(sess.vis_slice(vis, k), None, w_scale)
            errs.append(float(np.sqrt(np.mean((sol - wl.lm_true[k]) ** 2)) / I.ARCSEC))
            iters.append(rep.n_iter)
        e1.record()
        torch.cuda.synchronize()
        out[label] = {"rms_err_arcsec_max": max(errs), "mean_lm_iters": float(np.mean(iters)),
                      "solve_s": e0.elapsed_time(e1) / 1e3}
    sess.close()
    return {"n_intervals": len(wl.intervals), "n_vis": int(wl.n_vis), "sigma_pt_arcsec": sigma_arcsec,
            "tiling": list(best), "eval_ms": eval_ms, "gvis_per_s": wl.n_vis / (eval_ms * 1e-3) / 1e9,
            "flops_per_eval": flops, "fused_tflops": tflops,
            "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                         "flops_per_tap": RL.FLOPS_PER_TAP_EXACT},
            "solve_exact": out["exact"], "solve_gauss_model": out["gauss"]}


if __name__ == "__main__":
    import json
    print(json.dumps(run()))
