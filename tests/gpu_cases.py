"""Helpers that put a tiny oracle problem (``cases.problem``) on the GPU
through the C ABI.  The GPU side builds its own model grid from the same
image with ``psc_model_grid``; nothing computed by the oracle is handed to
the CUDA path except when a test says so (``use_oracle_grid``)."""
import numpy as np
import torch

from paper_1709_08681_gb300 import _abi


class GpuProblem:
    def __init__(self, m, img, use_oracle_grid=False, t_tile=None, c_group=None, kv=None):
        self.m = m
        dev = torch.device("cuda:0")
        self.uvw = torch.from_numpy(np.ascontiguousarray(m.uvw_m)).to(dev)
        ng = m.grid.shape[0]
        n_img = img.shape[0]
        if use_oracle_grid:
            self.grid = torch.from_numpy(m.grid.astype(np.complex64)).to(dev)
        else:
            self.grid = torch.empty((ng, ng), dtype=torch.complex64, device=dev)
            image = torch.from_numpy(np.ascontiguousarray(img, dtype=np.float32)).to(dev)
            _abi.psc_model_grid(n_img, ng, m.cell_rad, m.support, m.oversample, image, self.grid)
        nt, nbl, _ = m.uvw_m.shape
        self.shape = (nt, nbl, len(m.freq_hz))
        self.ctx = _abi.Context(m.n_ant, nt, len(m.freq_hz), self.uvw, m.freq_hz, m.ap_kind, m.diam_m,
                                m.alpha_per_dlambda, m.decorrelation, n_img, ng, m.cell_rad, m.support,
                                m.oversample, self.grid, ap_table=getattr(m, "ap_table", None))
        if t_tile or c_group or kv:
            self.ctx.psc_set_tiling(t_tile or 0, c_group or 0, kv or 0)

    def predict(self, lm, derivs=True):
        v = torch.empty(self.shape, dtype=torch.complex64, device="cuda:0")
        d = torch.empty((4,) + self.shape, dtype=torch.complex64, device="cuda:0") if derivs else None
        self.ctx.psc_predict(lm, v, d)
        return v.cpu().numpy(), (d.cpu().numpy() if derivs else None)

    def upload(self, arr, dtype=torch.complex64):
        return torch.from_numpy(np.ascontiguousarray(arr)).to("cuda:0").to(dtype)
