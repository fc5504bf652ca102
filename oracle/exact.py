"""Oracle: the exact per-baseline kernel of two uniform disks with different
pointing offsets (ctypes front of ``exact.c``).

Test infrastructure only (see ``oracle/__init__``).

Paper basis (Bhatnagar & Cornwell 2017, Sec. 3): A_ij is the transform of the
baseline's primary beam E_i E_j, the pattern of each antenna shifted by its
pointing offset.  Eq. AIJPOINTING models the main lobe as a Gaussian, which
turns the offsets into a phase ramp and an amplitude factor; the paper notes
that a more accurate pattern may replace the Gaussian.  For the uniform disk
the transform is exactly

    A_ij(du) = exp(i pi du.(l_i + l_j)) O(du; l_i - l_j) / (pi R^2)^2,

with O the integral of cos(2 pi w.dl) over the lens where the two apertures,
centred du apart, overlap (``exact.c`` derives it).  At l_i = l_j it is the
radial A° of ``aperture.aperture_disk``.  The derivatives follow from the
same integral: dA_ij/dl_i = A_ij i pi du + ramp dO/d(dl) / (pi R^2)^2 and
dA_ij/dl_j = A_ij i pi du - ramp dO/d(dl) / (pi R^2)^2 (m likewise).
"""
from __future__ import annotations

import ctypes

import numpy as np

from .degrid import _load, _p


def overlap(rho, a, b, R: float):
    """O(rho; a, b) and dO/da, dO/db for disks of radius R, at the points of
    the broadcast arrays rho (centre separation, wavelengths), a = dl.e_par,
    b = dl.e_perp (radians), by 32-node Gauss-Legendre quadrature."""
    lib = _load()
    rho, a, b = np.broadcast_arrays(*(np.asarray(x, dtype=np.float64) for x in (rho, a, b)))
    shape = rho.shape
    rho, a, b = (np.ascontiguousarray(x.ravel()) for x in (rho, a, b))
    O, Oa, Ob = (np.zeros(rho.size) for _ in range(3))
    dp = ctypes.c_double
    lib.oracle_exact_overlap(rho.size, _p(rho, dp), _p(a, dp), _p(b, dp), float(R), _p(O, dp), _p(Oa, dp),
                             _p(Ob, dp))
    return O.reshape(shape), Oa.reshape(shape), Ob.reshape(shape)


def degrid_sums_exact(u, v, L, M, dlx, dly, R, lens, grid, du, support, ov):
    """Per-visibility (T0, Tu, Tv, TX, TY) with the exact kernel (complex128,
    shaped like ``u``): T0 = sum K G ramp, Tu / Tv the same weighted by the
    tap offset (wavelengths), TX / TY = sum dK/d(dl_x | dl_y) G ramp, where
    K is normalised like the radial table (times du^2 / (pi R^2)^2) and
    interpolated linearly in radius at ``ov`` samples per cell.  R (disk
    radius, wavelengths) and lens (table length) are per visibility."""
    lib = _load()
    shape = np.shape(u)
    f64 = lambda x: np.ascontiguousarray(np.ravel(np.broadcast_to(x, shape)), dtype=np.float64)
    u, v, L, M, dlx, dly, R = (f64(x) for x in (u, v, L, M, dlx, dly, R))
    lens = np.ascontiguousarray(np.ravel(np.broadcast_to(lens, shape)), dtype=np.int32)
    g = np.ascontiguousarray(grid, dtype=np.complex128)
    n = u.size
    out = [np.zeros(n, dtype=np.complex128) for _ in range(5)]
    dp, ip = ctypes.c_double, ctypes.c_int
    lib.oracle_exact_degrid(n, _p(u, dp), _p(v, dp), _p(L, dp), _p(M, dp), _p(dlx, dp), _p(dly, dp),
                            _p(R, dp), _p(lens, ip), int(ov), _p(g.view(np.float64), dp), g.shape[0],
                            float(du), int(support), *(_p(o.view(np.float64), dp) for o in out))
    return tuple(o.reshape(shape) for o in out)
