"""Algorithmic work of the fused evaluation, for roofline figures.

Per visibility the fused kernel visits the grid cells inside the aperture's
support, pi rho_max^2 of them (rho_max in cells: the radial table's reach,
clipped to the S x S window).  The algorithmic work per such tap is
FLOPS_PER_TAP = 24 FP32 flops: the tap's kernel value A° K with its phase ramp
(a complex weight), and the three complex multiply-adds of V = sum K G and the
two derivative sums sum du K G, sum dv K G.  The kernels here factor the ramp
per cell and per visibility, which leaves FLOPS_PER_TAP_IMPL = 15 flops per
tap in the inner loop: s = dx^2 + dy^2 (2), the square root (1), t = rho ov (1),
the A° interpolation (2), P += A° G (4), A° dx (1), Q += (A° dx) G (4).  Rates
are reported against the algorithmic count; the implemented count is given
beside it.  The bound is the FP32 ALU: SMs x 128 lanes x 2 flops (FMA) x clock.
"""
from __future__ import annotations

import math

import numpy as np

FLOPS_PER_TAP = 24
FLOPS_PER_TAP_IMPL = 15
# Exact disk kernel (exact.cu), per tap: s (2), square root (1), seven
# interpolated series coefficients (14), 1 / s (1), (dl.du)/|du|^2 (1),
# A = (dl.e)^2 (1), O (6), dO/dA (6), dO/ds (4), its product with
# (dl.du)/|du|^2 (1), O dx and W dx (2), five complex accumulations (20), the
# two per-tap steps (2).
FLOPS_PER_TAP_EXACT = 61
# Residual-w stack: the Gaussian-model tap plus the interpolation between the
# two planes' cells, G_p + f (G_{p+1} - G_p) (2 subtractions, 2 FMAs).
FLOPS_PER_TAP_WSTACK = FLOPS_PER_TAP_IMPL + 4
FP32_LANES_PER_SM = 128
C_LIGHT = 299_792_458.0


def taps_per_channel(geom) -> np.ndarray:
    """Non-zero taps per visibility for each channel of ``geom`` (any object
    with n_grid, cell_rad, freq_hz, diam_m, ap_kind, support, oversample)."""
    du = 1.0 / (geom.n_grid * geom.cell_rad)
    out = []
    for f in geom.freq_hz:
        dl = geom.diam_m * f / C_LIGHT
        rho = dl / du if geom.ap_kind == "disk" else 0.5 * geom.support * math.sqrt(2)
        L = math.floor(geom.oversample * rho) + 2
        r = (L - 1) / geom.oversample
        out.append(min(math.pi * r * r, geom.support * geom.support))
    return np.asarray(out)


def fp32_peak_tflops(n_sm: int, clock_hz: float = 2.070e9) -> float:
    return n_sm * FP32_LANES_PER_SM * 2 * clock_hz / 1e12


def flops_per_eval(geom, intervals, n_bl, per_tap=FLOPS_PER_TAP) -> float:
    """Algorithmic FP32 flops of one fused evaluation of the given intervals
    ((t0, n_time) pairs of one geometry)."""
    taps = float(np.sum(taps_per_channel(geom)))
    return sum(nt for _, nt in intervals) * n_bl * taps * per_tap
