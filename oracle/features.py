"""Oracle: per-antenna input features of the learned initialiser (FP64).

Test infrastructure only (see ``oracle/__init__``).

Not a construct of the paper: the learned initial estimate is an addition to
the method.  Its input per antenna i is the chi^2 gradient and a 5 x 5
trial-offset stencil, read as 2 + 25 + 25 = 52 numbers:

* gradient: the block Newton step -H_ii^{-1} g_i at zero offsets (Eq. DCHIDD
  gradient and the Gauss-Newton 2x2 block of antenna i), over sigma_prior;
* for each trial offset delta_s = sigma_prior (a, b), a, b in -2..2, applied to
  antenna i alone (all other antennas at zero), with V_s the model of Eq.
  AIJPOINTING at that offset, over the baselines of antenna i:
    amplitude ratio  A_i(s) = sum w Re(conj(V_obs) V_s) / sum w |V_s|^2
    chi^2 change     C_i(s) = (chi2_i(delta_s) - chi2_i(0)) / sum w |V_0|^2,
    chi2_i(delta) = sum w |V_obs - V_s|^2 (C is zero at the centre and stays
    finite on noiseless data, where chi2_i(0) can vanish).
  Because the model of baseline (i, j) depends on the offsets only through
  l_i + l_j and |l_i - l_j| (ramp and decorrelation), putting delta on i or on
  j gives the same V_s: one evaluation per baseline serves both antennas.

Only time steps t with t % time_stride == 0 enter the sums (the gradient
block as well as the stencil).  Feature
order: [step_l, step_m, A(s) for s in row-major (b, a), C(s) likewise], with
a indexing the l offset and b the m offset.
"""
from __future__ import annotations

import math

import numpy as np

from . import psc
from .degrid import degrid_sums

N_FEAT = 52
STENCIL = [(a, b) for b in range(-2, 3) for a in range(-2, 3)]   # row-major over (b, a)


def stencil_model(model: psc.Model, sigma_prior: float, time_stride: int = 1):
    """V_s for every stencil point: complex128 [25][nt'][nbl][nc] over the kept time steps."""
    uvw = model.uvw_m[::time_stride]
    nt, nbl, _ = uvw.shape
    nc = len(model.freq_hz)
    shape = (nt, nbl, nc)
    u, v = psc.uv_lambda(uvw, model.freq_hz)
    chan = np.broadcast_to(np.arange(nc)[None, None, :], shape)
    a2 = (model.alpha() ** 2)[None, None, :]
    tables = model.tables()
    out = []
    for a, b in STENCIL:
        dl, dm = a * sigma_prior, b * sigma_prior
        L = np.full(shape, dl)          # l_i + l_j with only one antenna offset
        M = np.full(shape, dm)
        t0, _, _ = degrid_sums(u, v, L, M, chan, tables, model.grid, model.du, model.support, model.oversample)
        D = np.exp(-a2 * (dl * dl + dm * dm) / 2.0) if model.decorrelation else 1.0
        out.append(D * t0)
    return np.stack(out)


def features(model: psc.Model, vis_obs, w, sigma_prior: float, time_stride: int = 1):
    """float64 [n_ant][52] features (see module docstring)."""
    vis_obs = np.asarray(vis_obs, dtype=np.complex128)
    w = np.ones(vis_obs.shape) if w is None else np.asarray(w, dtype=np.float64)
    n = model.n_ant
    strided = psc.Model(**{**model.__dict__, "uvw_m": model.uvw_m[::time_stride]})
    chi2, g, H, X = psc.chi2_grad_normal(strided, np.zeros((n, 2)), vis_obs[::time_stride], w[::time_stride])
    step = np.zeros((n, 2))
    for i in range(n):
        Hi = np.array([[H[i, 0], H[i, 1]], [H[i, 1], H[i, 2]]])
        if np.linalg.det(Hi) > 0 and Hi[0, 0] > 0:
            step[i] = -np.linalg.solve(Hi, g[i])
    Vs = stencil_model(model, sigma_prior, time_stride)
    vo = vis_obs[::time_stride]
    ww = w[::time_stride]
    Xb = np.sum(ww[None] * np.real(np.conj(vo)[None] * Vs), axis=(1, 3))      # [25][nbl]
    Yb = np.sum(ww[None] * np.abs(Vs) ** 2, axis=(1, 3))
    Zb = np.sum(ww * np.abs(vo) ** 2, axis=(0, 2))                            # [nbl]
    ij = model.antenna_pairs()
    Xa = np.zeros((n, 25))
    Ya = np.zeros((n, 25))
    Za = np.zeros(n)
    for bl, (i, j) in enumerate(ij):
        for a in (i, j):
            Xa[a] += Xb[:, bl]
            Ya[a] += Yb[:, bl]
            Za[a] += Zb[bl]
    centre = STENCIL.index((0, 0))
    amp = Xa / Ya
    chi = Za[:, None] - 2.0 * Xa + Ya
    chi = (chi - chi[:, centre:centre + 1]) / Ya[:, centre:centre + 1]
    return np.concatenate([step / sigma_prior, amp, chi], axis=1)
