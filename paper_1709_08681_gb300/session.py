"""Device-resident setup of a workload for the C ABI.

Uploads the inputs of a ``inputs.Workload`` with torch (device memory and
streams only), builds the model grid with ``psc_model_grid`` and creates one
``psc_ctx`` per solution interval (each borrows a time slice of the shared
uvw array and the shared grid).  ``simulate`` predicts observed visibilities
with the GPU predictor at the workload's true offsets and adds the seeded
thermal noise drawn by ``inputs`` -- the way the paper simulates data
(Sec. 4.1), with the predictor standing in for its direct Fourier transform.
"""
from __future__ import annotations

import numpy as np
import torch

from . import _abi
from .inputs import Workload


class Session:
    def __init__(self, wl: Workload, device: str = "cuda:0", stream=None, grid=None):
        self.wl = wl
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.uvw = torch.from_numpy(np.ascontiguousarray(wl.uvw_m)).to(self.device)
        n_img = wl.image.shape[0]
        self.grid_args = dict(n_img=n_img, n_grid=wl.n_grid, cell_rad=wl.cell_rad, support=wl.support,
                              oversample=wl.oversample)
        if grid is None:
            img = torch.from_numpy(np.ascontiguousarray(wl.image, dtype=np.float32)).to(self.device)
            self.grid = torch.empty((wl.n_grid, wl.n_grid), dtype=torch.complex64, device=self.device)
            _abi.psc_model_grid(n_img, wl.n_grid, wl.cell_rad, wl.support, wl.oversample, img, self.grid,
                                self.stream)
            del img
        else:
            self.grid = grid
        self.ctxs = []
        row = wl.n_bl * 3 * 8
        for (t0, nt) in wl.intervals:
            self.ctxs.append(_abi.Context(
                wl.n_ant, nt, wl.n_chan, self.uvw.data_ptr() + t0 * row, wl.freq_hz, wl.ap_kind, wl.diam_m,
                wl.alpha_per_dlambda, wl.decorrelation, n_img, wl.n_grid, wl.cell_rad, wl.support,
                wl.oversample, self.grid.data_ptr(), self.stream))

    def vis_slice(self, vis: torch.Tensor, k: int) -> torch.Tensor:
        t0, nt = self.wl.intervals[k]
        return vis[t0:t0 + nt]

    def empty_vis(self) -> torch.Tensor:
        return torch.empty((self.wl.n_time, self.wl.n_bl, self.wl.n_chan), dtype=torch.complex64, device=self.device)

    def predict(self, lm_per_interval) -> torch.Tensor:
        out = self.empty_vis()
        for k, ctx in enumerate(self.ctxs):
            ctx.psc_predict(lm_per_interval[k], self.vis_slice(out, k))
        return out

    def simulate(self, noise: bool = True, noise_stream: int = 5, device_noise=None) -> torch.Tensor:
        """Observed visibilities at the true offsets plus thermal noise.  The
        noise comes from ``inputs`` (host, the same numbers on every machine)
        unless the data are too large to draw on the host (more than 2e8
        visibilities, or device_noise=True): then from a device generator
        seeded with (seed, noise_stream), one interval at a time."""
        v = self.predict(self.wl.lm_true)
        if noise and self.wl.sigma_noise > 0:
            if device_noise is None:
                device_noise = self.wl.n_vis > 200_000_000
            if not device_noise:
                v += torch.from_numpy(self.wl.noise(noise_stream)).to(self.device)
            else:
                g = torch.Generator(device=self.device)
                g.manual_seed(int(self.wl.seed) * 1000003 + int(noise_stream))
                for k in range(len(self.wl.intervals)):
                    sl = self.vis_slice(v, k)
                    sl += torch.view_as_complex(torch.randn(sl.shape + (2,), generator=g, device=self.device)
                                                * self.wl.sigma_noise)
        return v

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []


class MixedSession:
    """Device-resident setup of a mixed batch (``inputs.mixed_arrays`` /
    ``inputs.mixed_intervals``): one model grid per array type, and per
    interval its own uvw upload, context and observed visibilities -- the GPU
    predictor at the interval's true offsets plus thermal noise from a seeded
    device generator (the data are too large to draw on the host)."""

    def __init__(self, arrays: dict, intervals: list, device: str = "cuda:0", stream=None):
        from . import inputs as I
        self.arrays = arrays
        self.intervals = intervals
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.grids = {}
        for name, arr in arrays.items():
            n_img = arr.image.shape[0]
            img = torch.from_numpy(np.ascontiguousarray(arr.image, dtype=np.float32)).to(self.device)
            g = torch.empty((arr.n_grid, arr.n_grid), dtype=torch.complex64, device=self.device)
            _abi.psc_model_grid(n_img, arr.n_grid, arr.cell_rad, arr.support, arr.oversample, img, g, self.stream)
            self.grids[name] = g
            del img
        self.uvw, self.ctxs = [], []
        for iv in intervals:
            arr = arrays[iv.array]
            u = torch.from_numpy(I.mixed_uvw(arr, iv)).to(self.device)
            self.uvw.append(u)
            self.ctxs.append(_abi.Context(
                arr.n_ant, iv.n_time, len(arr.freq_hz), u, arr.freq_hz, arr.ap_kind, arr.diam_m,
                arr.alpha_per_dlambda, arr.decorrelation, arr.image.shape[0], arr.n_grid, arr.cell_rad,
                arr.support, arr.oversample, self.grids[iv.array], self.stream))

    def shape(self, k):
        iv = self.intervals[k]
        arr = self.arrays[iv.array]
        return (iv.n_time, arr.n_bl, len(arr.freq_hz))

    def n_vis(self, k=None):
        if k is None:
            return sum(self.n_vis(j) for j in range(len(self.intervals)))
        s = self.shape(k)
        return s[0] * s[1] * s[2]

    def simulate(self, noise: bool = True):
        """Observed visibilities of every interval (list of device tensors)."""
        out = []
        for k, iv in enumerate(self.intervals):
            v = torch.empty(self.shape(k), dtype=torch.complex64, device=self.device)
            self.ctxs[k].psc_predict(iv.lm_true, v)
            if noise:
                g = torch.Generator(device=self.device)
                g.manual_seed(iv.noise_seed)
                sig = self.arrays[iv.array].sigma_noise
                v += torch.view_as_complex(torch.randn(v.shape + (2,), generator=g, device=self.device) * sig)
            out.append(v)
        return out

    def close(self):
        for c in self.ctxs:
            c.close()
        self.ctxs = []
