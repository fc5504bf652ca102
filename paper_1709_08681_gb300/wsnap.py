"""W-snapshots on a workload (Sec. 6.1: for short solution intervals the
array may be treated as co-planar): per interval, the least-squares uvw plane
(``psc_snapshot_plane``), the model's components moved to the snapshot frame
(``psc_snapshot_components``, beam ratio at the band centre) and their model
grid on the tensor cores (``psc_model_grid_components``); each interval's
context gets its own grid, and the batch runs unchanged.

``run`` reports the per-interval set-up time, the component GEMM's rate, the
fitted planes and how far each interval departs from its plane (the part of
the w-term the method neglects), and the time of one batched LM iteration
over the snapshot contexts.
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import _abi
from . import inputs as I

C_LIGHT = 299_792_458.0


class SnapshotSession:
    """Contexts of a workload's intervals, each with its snapshot model grid."""

    def __init__(self, wl: I.Workload, device: str = "cuda:0", stream=None):
        self.wl = wl
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.uvw = torch.from_numpy(np.ascontiguousarray(wl.uvw_m)).to(self.device)
        f_ref = 0.5 * (float(wl.freq_hz[0]) + float(wl.freq_hz[-1]))
        row = wl.n_bl * 3 * 8
        self.grids, self.ctxs, self.planes, self.t_plane, self.t_grid = [], [], [], [], []
        for (t0, nt) in wl.intervals:
            uvw_k = self.uvw.data_ptr() + t0 * row
            t = time.perf_counter()
            a, b = _abi.psc_snapshot_plane(uvw_k, nt * wl.n_bl, self.stream)
            comp = _abi.psc_snapshot_components(wl.sky, a, b, wl.ap_kind, wl.diam_m, wl.alpha_per_dlambda, f_ref)
            self.t_plane.append(time.perf_counter() - t)
            grid = torch.empty((wl.n_grid, wl.n_grid), dtype=torch.complex64, device=self.device)
            t = time.perf_counter()
            _abi.psc_model_grid_components(comp, wl.n_grid, wl.cell_rad, grid, self.stream)
            self.t_grid.append(time.perf_counter() - t)
            self.grids.append(grid)
            self.planes.append((a, b))
            self.ctxs.append(_abi.Context(
                wl.n_ant, nt, wl.n_chan, uvw_k, wl.freq_hz, wl.ap_kind, wl.diam_m, wl.alpha_per_dlambda,
                wl.decorrelation, wl.image.shape[0], wl.n_grid, wl.cell_rad, wl.support, wl.oversample,
                grid.data_ptr(), self.stream))

    def vis_slice(self, vis, k):
        t0, nt = self.wl.intervals[k]
        return vis[t0:t0 + nt]

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []


def run(name="vla27_l64ch", seed=0, **over):
    wl = I.make_workload(name, seed=seed, **over)
    torch.cuda.synchronize()
    sess = SnapshotSession(wl)
    # departure of each interval from its plane, in wavelengths at the top frequency
    resid = []
    for (t0, nt), (a, b) in zip(wl.intervals, sess.planes):
        x = wl.uvw_m[t0:t0 + nt].reshape(-1, 3)
        resid.append(float(np.max(np.abs(x[:, 2] - a * x[:, 0] - b * x[:, 1]))) * float(wl.freq_hz[-1]) / C_LIGHT)
    # the batch over the snapshot contexts: one LM iteration, event-timed
    vis = torch.empty((wl.n_time, wl.n_bl, wl.n_chan), dtype=torch.complex64, device=sess.device)
    for k, ctx in enumerate(sess.ctxs):
        ctx.psc_predict(wl.lm_true[k], sess.vis_slice(vis, k))
    vk = [sess.vis_slice(vis, k) for k in range(len(sess.ctxs))]
    batch = _abi.Batch(sess.ctxs, vk, None, w_scale=[1.0 / wl.sigma_noise ** 2] * len(sess.ctxs), stream=sess.stream)
    batch.psc_batch_autotune()
    batch.psc_batch_begin([np.zeros((wl.n_ant, 2))] * len(sess.ctxs))
    for _ in range(2):
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(sess.stream)
    for _ in range(5):
        batch.psc_batch_restart()
        batch.psc_batch_iterate(1)
    e1.record(sess.stream)
    torch.cuda.synchronize()
    it_ms = e0.elapsed_time(e1) / 5
    batch.close()
    n_comp = wl.sky.shape[0]
    kp = max(8, (n_comp + 7) // 8 * 8)
    gemm_flops = 8.0 * wl.n_grid * wl.n_grid * kp              # complex multiply-adds of the component GEMM
    t_grid = float(np.median(sess.t_grid))
    rep = {"n_intervals": len(wl.intervals), "n_components": int(n_comp), "grid": wl.n_grid,
           "planes": [[round(a, 6), round(b, 6)] for a, b in sess.planes],
           "max_departure_from_plane_wavelengths": max(resid),
           "plane_and_components_ms": 1e3 * float(np.median(sess.t_plane)),
           "component_grid_ms": 1e3 * t_grid, "component_grid_tflops": gemm_flops / t_grid / 1e12,
           "batched_iteration_ms": it_ms, "gvis_per_s_iteration": wl.n_vis / (it_ms * 1e-3) / 1e9}
    sess.close()
    return rep


if __name__ == "__main__":
    import json
    print(json.dumps(run()))
