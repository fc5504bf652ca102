"""Oracle: closed-form (direct-sum) visibilities of point sources seen through
antenna beams with shifted pointing centres.

Test infrastructure only (see ``oracle/__init__``).

Paper basis: Eq. ME with the direction-independent term set to one and the
direction-dependent term E_i E_j* (real voltage patterns), evaluated as a
direct Fourier sum over point sources -- the way the paper simulates its
test data (Sec. 4.1: "direct Fourier transform and a model for the antenna
PB with pointing offsets"):

    V_ij(u, v) = sum_k S_k E(s_k - p_i) E(s_k - p_j) exp(+2 pi i (u l_k + v m_k))

where p_i = (l_i, m_i) is antenna i's pointing offset.  By default the w term
and n - 1 are left out (co-planar model, the same as the degridding path);
with ``w_term=True`` the phase also carries w (n_k - 1), n_k = sqrt(1 - l_k^2 - m_k^2)
(the non-coplanar measurement equation, for the W-snapshot pins).
"""
from __future__ import annotations

import math

import numpy as np

from . import aperture
from .psc import uv_lambda


def efp(kind: str, rho, freq_hz: float, diam_m: float, alpha_per_dlambda: float, blockage: float = 0.0):
    dl = float(aperture.d_lambda(diam_m, freq_hz))
    if kind == "disk":
        return aperture.efp_disk(rho, dl)
    if kind == "gauss":
        return aperture.efp_gauss(rho, alpha_per_dlambda * dl)
    if kind == "annulus":
        return aperture.efp_annulus(rho, dl, blockage)
    raise ValueError(kind)


def visibilities(uvw_m, freq_hz, n_ant, src, lm, kind, diam_m, alpha_per_dlambda, w_term=False, blockage=0.0):
    """complex128 [nt][nbl][nc] direct-sum visibilities (see module docstring)."""
    lm = np.asarray(lm, dtype=np.float64)
    uvw_m = np.asarray(uvw_m, dtype=np.float64)
    u, v = uv_lambda(uvw_m, freq_hz)
    w = uvw_m[..., 2:3] * (np.asarray(freq_hz, dtype=np.float64) / 299_792_458.0)
    ij = np.asarray([(i, j) for i in range(n_ant) for j in range(i + 1, n_ant)])
    out = np.zeros(u.shape, dtype=np.complex128)
    for c, f in enumerate(np.asarray(freq_hz, dtype=np.float64)):
        for lk, mk, sk in np.asarray(src, dtype=np.float64):
            rho = np.hypot(lk - lm[:, 0], mk - lm[:, 1])           # per antenna
            e = efp(kind, rho, f, diam_m, alpha_per_dlambda, blockage)
            amp = sk * e[ij[:, 0]] * e[ij[:, 1]]                    # [nbl]
            ph = u[:, :, c] * lk + v[:, :, c] * mk
            if w_term:
                ph = ph + w[:, :, c] * (math.sqrt(1.0 - lk * lk - mk * mk) - 1.0)
            out[:, :, c] += amp[None, :] * np.exp(2j * math.pi * ph)
    return out
