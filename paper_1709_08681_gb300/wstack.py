"""Residual-w stack on a workload: the whole observation solved as one long
interval, over which the array is not co-planar (Sec. 6.1 and the
conclusions: there the w-term adds to the cost; W-snapshots alone cover
short intervals).

Set-up, all through the C ABI: the interval's least-squares uvw plane
(``psc_snapshot_plane``), the components in the snapshot frame with each
one's n - 1 (``psc_wstack_components``, beam ratio at the band centre), the
residual-w extent (``psc_wstack_range``, scaled by the band's edges), the
plane spacing from the interpolation bound (2 pi max|n - 1| dw)^2 / 8 = eps,
the plane grids on the tensor cores (``psc_model_grid_wstack``) and the
context reading them (``psc_set_wstack``).

``run`` reports the stack (planes, spacing, bytes, build time), the fused
evaluation's time with the stack and with the snapshot grid alone (same
context and brick shape), how far apart the two models are, and the offsets
both recover from data predicted by a stack eight times finer.
``batched_intervals`` covers the workload's own short intervals instead: per
interval a plane, a snapshot grid and a stack of what the plane leaves, all
contexts in one batch (one persistent launch of the stacked kernel per LM
iteration), timed with and without the stacks.
"""
from __future__ import annotations

import math
import time

import numpy as np
import torch

from . import _abi, inputs as I, roofline as RL

C_LIGHT = 299_792_458.0
# candidate brick shapes: ("rect", t_tile, c_group, kv) or ("flat", items, kv)
TILINGS = [("rect", 32, 4, 1), ("rect", 64, 2, 1), ("rect", 16, 8, 1), ("rect", 32, 4, 2),
           ("flat", 128, 1), ("flat", 256, 1), ("flat", 128, 2), ("flat", 256, 2)]


class StackSession:
    """One context over all time steps of a workload, degridding from a stack."""

    def __init__(self, wl: I.Workload, eps: float = 1e-6, device: str = "cuda:0", stream=None):
        self.wl = wl
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.uvw = torch.from_numpy(np.ascontiguousarray(wl.uvw_m)).to(self.device)
        rows = wl.n_time * wl.n_bl
        f_lo, f_hi = float(np.min(wl.freq_hz)), float(np.max(wl.freq_hz))
        self.a, self.b = _abi.psc_snapshot_plane(self.uvw, rows, self.stream)
        lo_m, hi_m = _abi.psc_wstack_range(self.uvw, rows, self.a, self.b, self.stream)
        self.comp = _abi.psc_wstack_components(wl.sky, self.a, self.b, wl.ap_kind, wl.diam_m, wl.alpha_per_dlambda,
                                               0.5 * (f_lo + f_hi))
        self.w_lo = min(lo_m * f_lo, lo_m * f_hi) / C_LIGHT
        self.w_hi = max(hi_m * f_lo, hi_m * f_hi) / C_LIGHT
        self.grid = torch.empty((wl.n_grid, wl.n_grid), dtype=torch.complex64, device=self.device)
        _abi.psc_model_grid_components(self.comp[:, :3], wl.n_grid, wl.cell_rad, self.grid, self.stream)
        self.ctx = _abi.Context(wl.n_ant, wl.n_time, wl.n_chan, self.uvw, wl.freq_hz, wl.ap_kind, wl.diam_m,
                                wl.alpha_per_dlambda, wl.decorrelation, wl.image.shape[0], wl.n_grid, wl.cell_rad,
                                wl.support, wl.oversample, self.grid, self.stream)
        self.stacks = {}
        self.use(eps)

    def build(self, eps: float):
        """Plane grids for interpolation error eps (relative, per source)."""
        if eps in self.stacks:
            return self.stacks[eps]
        w0, dw, n = _stack_extent(self.comp, self.w_lo, self.w_hi, eps)
        planes = torch.empty((n, self.wl.n_grid, self.wl.n_grid), dtype=torch.complex64, device=self.device)
        torch.cuda.synchronize(self.device)
        t = time.perf_counter()
        _abi.psc_model_grid_wstack(self.comp, self.wl.n_grid, self.wl.cell_rad, n, w0, dw, planes, self.stream)
        st = {"planes": planes, "n": n, "w0": w0, "dw": dw, "build_s": time.perf_counter() - t}
        self.stacks[eps] = st
        return st

    def use(self, eps):
        """Degrid from the stack for eps, or from the snapshot grid (eps None)."""
        if eps is None:
            self.ctx.psc_set_wstack(None, 0)
            return
        st = self.build(eps)
        self.ctx.psc_set_wstack(st["planes"], st["n"], st["w0"], st["dw"], self.a, self.b)

    def close(self):
        self.ctx.close()
        self.stacks = {}


def _stack_extent(comp, w_lo, w_hi, eps):
    """(w0, dw, n_planes) covering [w_lo, w_hi] with interpolation error eps."""
    dw = math.sqrt(8.0 * eps) / (2.0 * math.pi * float(np.max(np.abs(comp[:, 3]))))
    w0 = math.floor(w_lo / dw) * dw
    return w0, dw, max(2, int(math.ceil((w_hi - w0) / dw)) + 1)


def batched_intervals(wl: I.Workload, eps: float = 1e-6, n_iter: int = 5, stream=None):
    """W-snapshots plus a residual-w stack per solution interval, batched."""
    dev = torch.device("cuda:0")
    stream = stream if stream is not None else torch.cuda.current_stream(dev)
    uvw = torch.from_numpy(np.ascontiguousarray(wl.uvw_m)).to(dev)
    row = wl.n_bl * 3 * 8
    f_lo, f_hi = float(np.min(wl.freq_hz)), float(np.max(wl.freq_hz))
    ctxs, keep, n_planes = [], [], []
    for (t0, nt) in wl.intervals:
        ptr = uvw.data_ptr() + t0 * row
        a, b = _abi.psc_snapshot_plane(ptr, nt * wl.n_bl, stream)
        lo_m, hi_m = _abi.psc_wstack_range(ptr, nt * wl.n_bl, a, b, stream)
        comp = _abi.psc_wstack_components(wl.sky, a, b, wl.ap_kind, wl.diam_m, wl.alpha_per_dlambda,
                                          0.5 * (f_lo + f_hi))
        w0, dw, n = _stack_extent(comp, min(lo_m * f_lo, lo_m * f_hi) / C_LIGHT,
                                  max(hi_m * f_lo, hi_m * f_hi) / C_LIGHT, eps)
        grid = torch.empty((wl.n_grid, wl.n_grid), dtype=torch.complex64, device=dev)
        _abi.psc_model_grid_components(comp[:, :3], wl.n_grid, wl.cell_rad, grid, stream)
        planes = torch.empty((n, wl.n_grid, wl.n_grid), dtype=torch.complex64, device=dev)
        _abi.psc_model_grid_wstack(comp, wl.n_grid, wl.cell_rad, n, w0, dw, planes, stream)
        ctx = _abi.Context(wl.n_ant, nt, wl.n_chan, ptr, wl.freq_hz, wl.ap_kind, wl.diam_m, wl.alpha_per_dlambda,
                           wl.decorrelation, wl.image.shape[0], wl.n_grid, wl.cell_rad, wl.support, wl.oversample,
                           grid.data_ptr(), stream)
        ctx.psc_set_wstack(planes, n, w0, dw, a, b)
        ctxs.append(ctx)
        keep.append((grid, planes, (w0, dw, n, a, b)))
        n_planes.append(n)
    vis = torch.empty((wl.n_time, wl.n_bl, wl.n_chan), dtype=torch.complex64, device=dev)
    vk = []
    for k, ((t0, nt), ctx) in enumerate(zip(wl.intervals, ctxs)):
        vk.append(vis[t0:t0 + nt])
        ctx.psc_predict(wl.lm_true[k], vk[-1])

    def iteration_ms():
        batch = _abi.Batch(ctxs, vk, None, w_scale=[1.0 / wl.sigma_noise ** 2] * len(ctxs), stream=stream)
        batch.psc_batch_autotune()
        batch.psc_batch_begin([np.zeros((wl.n_ant, 2))] * len(ctxs))
        for _ in range(2):
            batch.psc_batch_restart()
            batch.psc_batch_iterate(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(n_iter):
            batch.psc_batch_restart()
            batch.psc_batch_iterate(1)
        e1.record(stream)
        torch.cuda.synchronize()
        batch.close()
        return e0.elapsed_time(e1) / n_iter

    ms_stack = iteration_ms()
    for ctx in ctxs:
        ctx.psc_set_wstack(None, 0)
    ms_snap = iteration_ms()
    for ctx in ctxs:
        ctx.close()
    n_vis = wl.n_time * wl.n_bl * wl.n_chan
    return {"n_intervals": len(wl.intervals), "planes_per_interval": n_planes,
            "stack_bytes": int(sum(n_planes)) * wl.n_grid * wl.n_grid * 8,
            "batched_iteration_ms_stack": ms_stack, "gvis_per_s_stack": n_vis / (ms_stack * 1e-3) / 1e9,
            "batched_iteration_ms_snapshot_grids": ms_snap, "gvis_per_s_snapshot_grids": n_vis / (ms_snap * 1e-3) / 1e9}


def _apply(ctx, tl):
    if tl[0] == "rect":
        ctx.psc_set_tiling(*tl[1:])
    else:
        ctx.psc_set_flat_tiling(*tl[1:])


def _eval_ms(ctx, lm, vis, w_scale, n):
    ctx.psc_profile(True)
    ctx.psc_residual_grad(lm, vis, None, w_scale)              # warm
    ctx.psc_profile_read()
    for _ in range(n):
        ctx.psc_residual_grad(lm, vis, None, w_scale)
    ms, k = ctx.psc_profile_read()
    ctx.psc_profile(False)
    return ms / max(k, 1)


def run(name="vla27_l64ch", seed=0, eps=1e-6, n_eval=5, **over):
    wl = I.make_workload(name, seed=seed, **over)
    torch.cuda.synchronize()
    sess = StackSession(wl, eps)
    ctx = sess.ctx
    w_scale = 1.0 / wl.sigma_noise ** 2
    lm_true = wl.lm_true[0]
    # data: a stack eight times finer in w (error bound 64 times lower) plus noise
    sess.use(eps / 64)
    vis = torch.empty((wl.n_time, wl.n_bl, wl.n_chan), dtype=torch.complex64, device=sess.device)
    ctx.psc_predict(lm_true, vis)
    vis += torch.from_numpy(wl.noise(5)).to(vis.device)
    fine = sess.stacks.pop(eps / 64)
    fine_info = {"planes": fine["n"], "dw": fine["dw"]}
    del fine
    # brick shape for the stack: one timed evaluation per candidate
    sess.use(eps)
    lm_eval = 0.5 * lm_true
    best, best_ms = None, float("inf")
    for tl in TILINGS:
        try:
            _apply(ctx, tl)
        except _abi.PscError:
            continue                                           # e.g. kv = 2 not allowed
        ms = _eval_ms(ctx, lm_eval, vis, w_scale, 1)
        if ms < best_ms:
            best, best_ms = tl, ms
    _apply(ctx, best)
    ms_stack = _eval_ms(ctx, lm_eval, vis, w_scale, n_eval)
    v_stack = torch.empty_like(vis)
    ctx.psc_predict(lm_true, v_stack)
    sess.use(None)
    ms_snap = _eval_ms(ctx, lm_eval, vis, w_scale, n_eval)
    v_snap = torch.empty_like(vis)
    ctx.psc_predict(lm_true, v_snap)
    model_gap = float(torch.linalg.vector_norm(v_stack - v_snap) / torch.linalg.vector_norm(v_stack))
    # offsets from both models (same data, same brick shape)
    solves = {}
    for label, e in (("stack", eps), ("snapshot_only", None)):
        sess.use(e)
        torch.cuda.synchronize()
        t = time.perf_counter()
        sol, rep = ctx.psc_solve_offsets(vis, None, w_scale)
        solves[label] = {"rms_err_arcsec": float(np.sqrt(np.mean((sol - lm_true) ** 2)) / I.ARCSEC),
                         "lm_iters": rep.n_iter, "solve_s": time.perf_counter() - t}
    st = sess.stacks[eps]
    sess.close()
    batched = batched_intervals(wl, eps)
    taps = RL.taps_per_channel(wl)
    flops = wl.n_time * wl.n_bl * float(np.sum(taps)) * RL.FLOPS_PER_TAP_WSTACK
    props = torch.cuda.get_device_properties(vis.device)
    peak = RL.fp32_peak_tflops(props.multi_processor_count)
    tflops = flops / (ms_stack * 1e-3) / 1e12
    n_vis = wl.n_time * wl.n_bl * wl.n_chan
    out = {"n_time": wl.n_time, "n_vis": int(n_vis), "plane": [sess.a, sess.b],
           "residual_w_lambda": [sess.w_lo, sess.w_hi], "eps": eps, "n_planes": st["n"], "dw_lambda": st["dw"],
           "stack_bytes": st["n"] * wl.n_grid * wl.n_grid * 8, "stack_build_s": st["build_s"],
           "tiling": list(best), "eval_ms_stack": ms_stack, "gvis_per_s_stack": n_vis / (ms_stack * 1e-3) / 1e9,
           "eval_ms_snapshot_grid": ms_snap, "gvis_per_s_snapshot_grid": n_vis / (ms_snap * 1e-3) / 1e9,
           "model_gap_rel_l2": model_gap, "data_stack": fine_info, "solve": solves,
           "roofline": {"bound": "alu", "achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
                        "flops_per_tap": RL.FLOPS_PER_TAP_WSTACK},
           "batched_short_intervals": batched}
    return out


if __name__ == "__main__":
    import json
    print(json.dumps(run()))
