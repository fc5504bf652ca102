"""Oracle: W-snapshots for one solution interval (test infrastructure only,
see ``oracle/__init__``).

Paper basis (Bhatnagar & Cornwell 2017, Sec. 6.1 and the conclusions): for
short solution intervals the cost of the w-term can be avoided by treating
the array as co-planar within each interval (the W-snapshots algorithm).

With the w-term the phase of source k is u l_k + v m_k + w (n_k - 1).  If the
interval's baselines lie in the plane w = a u + b v, it equals
u l'_k + v m'_k with

    l'_k = l_k + a (n_k - 1),   m'_k = m_k + b (n_k - 1),

so the co-planar degridding path applies to the sky with its sources moved to
(l', m').  Readings (no formula in the paper):
* (a, b) is the least-squares plane of the interval's (u, v, w) in metres
  (all baselines and time steps);
* the degridding kernel weights a source by the primary beam at the grid
  position (l', m'), so each flux is rescaled by PB(l_k) / PB(l'_k), PB the
  pointing-free power pattern of the antenna pair (the disk's Airy pattern
  squared, or the Gaussian's), evaluated per channel group at the channel
  given; the pointing offsets then enter only through the kernel, as in the
  co-planar path;
* what stays of the w-term is w - a u - b v, the interval's departure from the
  plane, which this method neglects.
"""
from __future__ import annotations

import math

import numpy as np

from . import aperture


def plane_fit(uvw_m) -> tuple:
    """(a, b) minimising sum (w - a u - b v)^2 over all rows of uvw [..., 3]."""
    x = np.asarray(uvw_m, dtype=np.float64).reshape(-1, 3)
    A = x[:, :2]
    sol, *_ = np.linalg.lstsq(A, x[:, 2], rcond=None)
    return float(sol[0]), float(sol[1])


def distort(src, a: float, b: float) -> np.ndarray:
    """Sources (l, m, S) moved to the snapshot frame: (l + a (n-1), m + b (n-1), S)."""
    src = np.asarray(src, dtype=np.float64)
    l, m = src[:, 0], src[:, 1]
    nm1 = np.sqrt(1.0 - l * l - m * m) - 1.0
    return np.stack([l + a * nm1, m + b * nm1, src[:, 2]], axis=1)


def power_beam(kind: str, rho, freq_hz: float, diam_m: float, alpha_per_dlambda: float):
    dl = float(aperture.d_lambda(diam_m, freq_hz))
    if kind == "disk":
        return aperture.efp_disk(rho, dl) ** 2
    return aperture.efp_gauss(rho, alpha_per_dlambda * dl) ** 2


def snapshot_sources(src, a: float, b: float, kind: str, freq_hz: float, diam_m: float,
                     alpha_per_dlambda: float) -> np.ndarray:
    """Distorted sources with fluxes rescaled by PB(l) / PB(l') at ``freq_hz``."""
    src = np.asarray(src, dtype=np.float64)
    out = distort(src, a, b)
    pb0 = power_beam(kind, np.hypot(src[:, 0], src[:, 1]), freq_hz, diam_m, alpha_per_dlambda)
    pb1 = power_beam(kind, np.hypot(out[:, 0], out[:, 1]), freq_hz, diam_m, alpha_per_dlambda)
    out[:, 2] = src[:, 2] * pb0 / pb1
    return out
