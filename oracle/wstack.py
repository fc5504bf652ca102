"""Oracle: the residual w-term of long solution intervals, by a stack of
model grids in w (test infrastructure only, see ``oracle/__init__``).

Paper basis (Bhatnagar & Cornwell 2017, Sec. 6.1 and the conclusions): when
the array is not co-planar over an interval the w-term adds to the cost of
the method; W-snapshots remove it for intervals short enough to be treated as
co-planar.  This module covers what W-snapshots leave: the departure of each
visibility from the interval's plane.

With the plane w = a u + b v (``wsnap.plane_fit``) and the sources moved to
the snapshot frame (``wsnap.snapshot_sources``: positions l', m', fluxes S'),
the phase of source k still carries

    w_r (n_k - 1),    w_r = (w - a u - b v) nu / c  (wavelengths),

with n_k = sqrt(1 - l_k^2 - m_k^2) of the source's true direction.  Readings
(the paper names the problem, not a formula):
* plane p of the stack is the model grid of the snapshot sources with the
  complex fluxes S'_k exp(2 pi i w_p (n_k - 1)), at w_p = w0 + p dw,
  p = 0 .. P-1 (P >= 2);
* a visibility with residual w_r is degridded from
  (1 - f) G_p + f G_{p+1},  q = (w_r - w0) / dw,  p = min(floor(q), P - 2),
  f = q - p,
  which interpolates exp(2 pi i w (n_k - 1)) linearly in w between the two
  planes around w_r; the error per source is at most
  (2 pi |n_k - 1| dw)^2 / 8 of its flux;
* the stack must cover every visibility: w0 <= w_r <= w0 + (P - 1) dw, else
  the evaluation is refused;
* the pointing offsets enter only through the kernel, as in the co-planar
  path: the w-screen belongs to the sky, so the derivative formulas are
  unchanged and V, dV are linear in the grid.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import model_grid, psc, wsnap


def residual_w(uvw_m, freq_hz, a: float, b: float) -> np.ndarray:
    """w_r [nt][nbl][nc] in wavelengths."""
    uvw_m = np.asarray(uvw_m, dtype=np.float64)
    wr = uvw_m[..., 2] - a * uvw_m[..., 0] - b * uvw_m[..., 1]
    return wr[..., None] * (np.asarray(freq_hz, dtype=np.float64) / psc.C_LIGHT)


def stack_sources(src, a: float, b: float, kind: str, freq_hz: float, diam_m: float,
                  alpha_per_dlambda: float) -> np.ndarray:
    """[n][4] rows (l', m', S', n - 1): the snapshot sources and each source's
    n - 1 at its true direction."""
    src = np.asarray(src, dtype=np.float64)
    snap = wsnap.snapshot_sources(src, a, b, kind, freq_hz, diam_m, alpha_per_dlambda)
    nm1 = np.sqrt(1.0 - src[:, 0] ** 2 - src[:, 1] ** 2) - 1.0
    return np.concatenate([snap, nm1[:, None]], axis=1)


def plane_grids(src4, n_grid: int, du: float, w0: float, dw: float, n_planes: int) -> np.ndarray:
    """complex128 [P][Ng][Ng]: plane p is the grid of fluxes S' exp(2 pi i w_p (n - 1))."""
    src4 = np.asarray(src4, dtype=np.float64)
    out = np.empty((n_planes, n_grid, n_grid), dtype=np.complex128)
    for p in range(n_planes):
        wp = w0 + p * dw
        flux = src4[:, 2] * np.exp(2j * np.pi * wp * src4[:, 3])
        out[p] = model_grid.grid_from_components(src4[:, :3], n_grid, du, flux=flux)
    return out


def plane_weights(wr, w0: float, dw: float, n_planes: int):
    """(p, f): the lower plane and the weight of the upper one, per visibility."""
    if n_planes < 2 or not dw > 0:
        raise ValueError("a stack needs at least two planes and dw > 0")
    wr = np.asarray(wr, dtype=np.float64)
    q = (wr - w0) / dw
    if np.any(q < 0) or np.any(q > n_planes - 1):
        raise ValueError("the w-planes do not cover every visibility")
    p = np.minimum(np.floor(q).astype(np.int64), n_planes - 2)
    return p, q - p


def predict(model: psc.Model, planes, w0: float, dw: float, a: float, b: float, lm, with_derivs: bool = True):
    """V [nt][nbl][nc] and dV [4][nt][nbl][nc] from the stack: each plane's
    prediction (``psc.predict`` with that plane as the grid) weighted by the
    visibility's interpolation weight, which by linearity in the grid equals
    degridding the interpolated grid."""
    wr = residual_w(model.uvw_m, model.freq_hz, a, b)
    p, f = plane_weights(wr, w0, dw, len(planes))
    V = np.zeros(wr.shape, dtype=np.complex128)
    dV = np.zeros((4,) + wr.shape, dtype=np.complex128) if with_derivs else None
    for k in range(len(planes)):
        h = np.where(p == k, 1.0 - f, 0.0) + np.where(p + 1 == k, f, 0.0)
        if not np.any(h):
            continue
        Vk, dVk = psc.predict(dataclasses.replace(model, grid=planes[k]), lm, with_derivs)
        V += h * Vk
        if with_derivs:
            dV += h[None] * dVk
    return V, dV


def chi2_grad_normal(model: psc.Model, planes, w0, dw, a, b, lm, vis_obs, w=None):
    """chi^2, g, H and the cross blocks X (as ``psc.chi2_grad_normal``) with the stack."""
    V, dV = predict(model, planes, w0, dw, a, b, lm)
    return psc.reduce_terms(model, V, dV, vis_obs, w)
