"""Oracle: model visibilities, their pointing derivatives, residuals, chi^2,
and the per-antenna gradient and 2x2 normal-equation blocks, in FP64.

Test infrastructure only (see ``oracle/__init__``).

Paper basis (Bhatnagar & Cornwell 2017)
---------------------------------------
* Algorithm 1, inner loop: compute A_ij and grad_i A_ij (Eqs. AIJPOINTING,
  DAIJPOINTING), degrid V^M = A_ij * V° and grad_i V^M = grad_i A_ij * V°,
  form R_ij = V^Obs - V^M and accumulate Chi and dChi.
* Eq. AIJPOINTING: A_ij = A° exp(-(l_i - l_j)^2 alpha^2 / 2) exp(i pi u (l_i + l_j)),
  written for l and extended the same way to m (Sec. 3).
* Eq. DAIJPOINTING: dA_ij/dl_i = A_ij [(l_j - l_i) alpha^2 + i pi u].
* Eq. Chisq: chi^2 = sum R^dag W R (one parallel-hand product here: sum w |R|^2).
* Eq. DCHIDD: d chi^2 / d a_i = -2 sum_j Re(R_ij^dag W_ij grad_i V^M_ij).

Readings: each measured visibility is one baseline i < j, so chi^2 sums over
i < j and every baseline feeds both of its antennas' gradients; the normal
blocks are the Gauss-Newton ones, H_pq = 2 sum w Re(conj(dV/dp) dV/dq), for
p, q in {l_a, m_a} of one antenna a.  alpha scales with frequency as
alpha = alpha_per_dlambda * D nu / c.  With ``decorrelation = 0`` the bracketed
amplitude factor of Eq. AIJPOINTING is dropped and so is its derivative term.
With ``kernel = "exact"`` (uniform disks only) the kernel is the exact
transform of the two shifted disk patterns' product (``oracle/exact``), which
carries the amplitude's dependence on l_i - l_j itself; ``decorrelation`` is
then not used.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

from . import aperture
from .degrid import degrid_sums
from .exact import degrid_sums_exact

C_LIGHT = 299_792_458.0


@dataclasses.dataclass
class Model:
    """The fixed part of one solve: geometry, model grid and aperture."""
    uvw_m: np.ndarray          # [nt][nbl][3] metres
    freq_hz: np.ndarray        # [nc]
    n_ant: int
    grid: np.ndarray           # complex128 [Ng][Ng]
    cell_rad: float            # image pixel; du = 1 / (Ng cell)
    support: int
    oversample: int
    ap_kind: str               # "disk" | "gauss"
    diam_m: float
    alpha_per_dlambda: float
    decorrelation: int
    kernel: str = "gauss"      # "gauss": Eq. AIJPOINTING; "exact": the disks' exact kernel
    ap_table: object = None    # ap_kind "table": dish-scale samples of A° (oracle.aperture)

    @property
    def du(self) -> float:
        return 1.0 / (self.grid.shape[0] * self.cell_rad)

    def alpha(self) -> np.ndarray:
        return self.alpha_per_dlambda * aperture.d_lambda(self.diam_m, self.freq_hz)

    def tables(self):
        dl = aperture.d_lambda(self.diam_m, self.freq_hz)
        al = self.alpha()
        return [aperture.radial_table(self.ap_kind, dl[c], al[c], self.du, self.oversample, self.support,
                                      self.ap_table)
                for c in range(len(self.freq_hz))]

    def antenna_pairs(self):
        ij = [(i, j) for i in range(self.n_ant) for j in range(i + 1, self.n_ant)]
        return np.asarray(ij, dtype=np.int64)


def uv_lambda(uvw_m: np.ndarray, freq_hz: np.ndarray):
    """(u, v) in wavelengths, shaped [nt][nbl][nc]: uvw * nu / c."""
    s = np.asarray(freq_hz, dtype=np.float64) / C_LIGHT
    return uvw_m[..., 0:1] * s, uvw_m[..., 1:2] * s


def predict(model: Model, lm: np.ndarray, with_derivs: bool = True):
    """Model visibilities V [nt][nbl][nc] and, optionally, the derivative planes
    [4][nt][nbl][nc] = dV/dl_i, dV/dm_i, dV/dl_j, dV/dm_j (complex128)."""
    lm = np.asarray(lm, dtype=np.float64)
    nt, nbl, _ = model.uvw_m.shape
    nc = len(model.freq_hz)
    ij = model.antenna_pairs()
    li, mi = lm[ij[:, 0], 0], lm[ij[:, 0], 1]
    lj, mj = lm[ij[:, 1], 0], lm[ij[:, 1], 1]
    shape = (nt, nbl, nc)
    u, v = uv_lambda(model.uvw_m, model.freq_hz)
    L = np.broadcast_to((li + lj)[None, :, None], shape)
    M = np.broadcast_to((mi + mj)[None, :, None], shape)
    chan = np.broadcast_to(np.arange(nc)[None, None, :], shape)
    if model.kernel == "exact":
        dlx = np.broadcast_to((li - lj)[None, :, None], shape)
        dly = np.broadcast_to((mi - mj)[None, :, None], shape)
        return _exact_out(model, u, v, L, M, dlx, dly, chan, with_derivs)
    t0, tu, tv = degrid_sums(u, v, L, M, chan, model.tables(), model.grid, model.du,
                             model.support, model.oversample)
    a2 = (model.alpha() ** 2)[None, None, :]
    if model.decorrelation:
        dsq = ((li - lj) ** 2 + (mi - mj) ** 2)[None, :, None]
        D = np.exp(-a2 * dsq / 2.0)
        dl = (lj - li)[None, :, None] * a2      # (l_j - l_i) alpha^2
        dm = (mj - mi)[None, :, None] * a2
    else:
        D = np.ones((1, nbl, 1))
        dl = np.zeros((1, nbl, 1))
        dm = np.zeros((1, nbl, 1))
    V = D * t0
    if not with_derivs:
        return V, None
    ipi = 1j * math.pi
    dV = np.stack([D * (dl * t0 + ipi * tu),      # d/dl_i
                   D * (dm * t0 + ipi * tv),      # d/dm_i
                   D * (-dl * t0 + ipi * tu),     # d/dl_j
                   D * (-dm * t0 + ipi * tv)])    # d/dm_j
    return V, dV


def _exact_out(model: Model, u, v, L, M, dlx, dly, chan, with_derivs):
    """V and dV with the exact disk kernel: V = T0, dV/dl_i = TX + i pi Tu,
    dV/dl_j = -TX + i pi Tu (m likewise with TY, Tv)."""
    if model.ap_kind != "disk":
        raise ValueError("the exact kernel is defined for uniform disks")
    dl = aperture.d_lambda(model.diam_m, model.freq_hz)
    lens = np.asarray([aperture.table_len("disk", d, model.du, model.oversample, model.support) for d in dl])
    chan = np.asarray(chan)
    t0, tu, tv, tx, ty = degrid_sums_exact(u, v, L, M, dlx, dly, 0.5 * dl[chan], lens[chan], model.grid,
                                           model.du, model.support, model.oversample)
    if not with_derivs:
        return t0, None
    ipi = 1j * math.pi
    return t0, np.stack([tx + ipi * tu, ty + ipi * tv, -tx + ipi * tu, -ty + ipi * tv])


def predict_points(model: Model, lm, t_idx, bl_idx, ch_idx):
    """V and dV (dV/dl_i, dV/dm_i, dV/dl_j, dV/dm_j) of selected visibilities
    (index arrays into [nt][nbl][nc]), by the same formulas as ``predict``."""
    lm = np.asarray(lm, dtype=np.float64)
    t_idx, bl_idx, ch_idx = (np.asarray(x, dtype=np.int64) for x in (t_idx, bl_idx, ch_idx))
    ij = model.antenna_pairs()[bl_idx]
    li, mi = lm[ij[:, 0], 0], lm[ij[:, 0], 1]
    lj, mj = lm[ij[:, 1], 0], lm[ij[:, 1], 1]
    f = np.asarray(model.freq_hz, dtype=np.float64)[ch_idx] / C_LIGHT
    u = model.uvw_m[t_idx, bl_idx, 0] * f
    v = model.uvw_m[t_idx, bl_idx, 1] * f
    if model.kernel == "exact":
        return _exact_out(model, u, v, li + lj, mi + mj, li - lj, mi - mj, ch_idx, True)
    t0, tu, tv = degrid_sums(u, v, li + lj, mi + mj, ch_idx, model.tables(), model.grid, model.du,
                             model.support, model.oversample)
    a2 = model.alpha()[ch_idx] ** 2
    if model.decorrelation:
        D = np.exp(-a2 * ((li - lj) ** 2 + (mi - mj) ** 2) / 2.0)
        dl, dm = (lj - li) * a2, (mj - mi) * a2
    else:
        D, dl, dm = np.ones_like(u), np.zeros_like(u), np.zeros_like(u)
    ipi = 1j * math.pi
    V = D * t0
    dV = np.stack([D * (dl * t0 + ipi * tu), D * (dm * t0 + ipi * tv),
                   D * (-dl * t0 + ipi * tu), D * (-dm * t0 + ipi * tv)])
    return V, dV


def chi2_grad_normal(model: Model, lm, vis_obs, w=None):
    """chi^2, gradient g [n_ant][2] (d/dl, d/dm), diagonal normal blocks
    H [n_ant][3] = (H_ll, H_lm, H_mm) and per-baseline cross blocks
    X [n_bl][4] = (H_{l_i l_j}, H_{l_i m_j}, H_{m_i l_j}, H_{m_i m_j}) at ``lm``."""
    V, dV = predict(model, lm)
    return reduce_terms(model, V, dV, vis_obs, w)


def reduce_terms(model: Model, V, dV, vis_obs, w=None):
    vis_obs = np.asarray(vis_obs, dtype=np.complex128)
    w = np.ones(V.shape) if w is None else np.asarray(w, dtype=np.float64)
    R = vis_obs - V
    chi2 = float(np.sum(w * np.abs(R) ** 2))
    ij = model.antenna_pairs()
    g = np.zeros((model.n_ant, 2))
    H = np.zeros((model.n_ant, 3))

    def nsum(p, q):           # 2 sum w Re(conj(dV_p) dV_q) per baseline
        return 2.0 * np.sum(w * np.real(np.conj(dV[p]) * dV[q]), axis=(0, 2))

    # per-baseline sums over time and channel, then scattered to antennas
    gp = -2.0 * np.sum(w[None] * np.real(np.conj(R)[None] * dV), axis=(1, 3))        # [4][nbl]
    hi = np.stack([nsum(0, 0), nsum(0, 1), nsum(1, 1)], axis=1)
    hj = np.stack([nsum(2, 2), nsum(2, 3), nsum(3, 3)], axis=1)
    X = np.stack([nsum(0, 2), nsum(0, 3), nsum(1, 2), nsum(1, 3)], axis=1)
    for b, (i, j) in enumerate(ij):
        g[i] += gp[0, b], gp[1, b]
        g[j] += gp[2, b], gp[3, b]
        H[i] += hi[b]
        H[j] += hj[b]
    return chi2, g, H, X


def assemble_full(n_ant: int, g, H, X):
    """Full gradient [2n] and Gauss-Newton matrix [2n][2n] (order l_0, m_0,
    l_1, m_1, ...) from the per-antenna and per-baseline 2x2 blocks."""
    n = 2 * n_ant
    G = np.asarray(g, dtype=np.float64).reshape(n)
    A = np.zeros((n, n))
    for a in range(n_ant):
        A[2 * a, 2 * a], A[2 * a, 2 * a + 1], A[2 * a + 1, 2 * a + 1] = H[a]
        A[2 * a + 1, 2 * a] = H[a][1]
    b = 0
    for i in range(n_ant):
        for j in range(i + 1, n_ant):
            blk = np.asarray(X[b]).reshape(2, 2)
            A[2 * i:2 * i + 2, 2 * j:2 * j + 2] = blk
            A[2 * j:2 * j + 2, 2 * i:2 * i + 2] = blk.T
            b += 1
    return G, A


def full_normal(model: Model, lm, vis_obs, w=None):
    """chi^2, full gradient [2 n_ant] and full Gauss-Newton matrix [2n][2n]
    (parameter order l_0, m_0, l_1, m_1, ...), built visibility by visibility
    from the Jacobian rows -- an independent route to the blocks above."""
    V, dV = predict(model, lm)
    vis_obs = np.asarray(vis_obs, dtype=np.complex128)
    w = np.ones(V.shape) if w is None else np.asarray(w, dtype=np.float64)
    R = vis_obs - V
    chi2 = float(np.sum(w * np.abs(R) ** 2))
    ij = model.antenna_pairs()
    n = 2 * model.n_ant
    g = np.zeros(n)
    H = np.zeros((n, n))
    for b, (i, j) in enumerate(ij):
        idx = [2 * i, 2 * i + 1, 2 * j, 2 * j + 1]
        J = dV[:, :, b, :].reshape(4, -1)
        wb = w[:, b, :].reshape(-1)
        rb = R[:, b, :].reshape(-1)
        g[idx] += -2.0 * np.real(np.conj(rb)[None, :] * J) @ wb
        H[np.ix_(idx, idx)] += 2.0 * np.real((np.conj(J) * wb[None, :]) @ J.T)
    return chi2, g, H
