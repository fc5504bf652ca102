"""Oracle: antenna voltage patterns, the a-priori aperture kernel A° and its
radial table.  Test infrastructure only (see ``oracle/__init__``).

Paper basis
-----------
* Sec. 3: the main lobe of an antenna's far-field pattern is modelled as
  exp(-(l - l_i)^2 alpha^2), alpha = 2^-1/2 / sigma; A_ij is the Fourier
  transform of the baseline's primary beam, and A°_ij is its pre-computed,
  pointing-free part.  Algorithm 1 pre-computes A° once.
* Eq. ME: V = int E_i E_j* I exp(+2 pi i s.b) ds, so with the same sign
  convention A°(q) = int PB(l) exp(+2 pi i q.l) dl.

For a uniform disk of diameter D the voltage pattern is 2 J1(x)/x,
x = pi D_lambda rho, and the power beam's transform is the disk's
autocorrelation divided by its area squared (so that int A° dq = PB(0) = 1).
For the Gaussian model the power beam exp(-2 alpha^2 rho^2) transforms to
(pi / (2 alpha^2)) exp(-pi^2 q^2 / (2 alpha^2)).

Table rule (shared definition, implemented independently on the GPU side):
the table of a channel holds A°(n du / ov) du^2, n = 0 .. len-1, with
len = floor(ov * rho_max) + 2 where rho_max (in grid cells) is D_lambda/du for
the disk and (S/2) sqrt(2) for the Gaussian.  A tap at radius rho cells reads
t = rho * ov, n = floor(t), f = t - n, value (1-f) tab[n] + f tab[n+1] when
n + 1 < len, else 0.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

C_LIGHT = 299_792_458.0


def d_lambda(diam_m: float, freq_hz):
    """Aperture diameter in wavelengths."""
    return diam_m * np.asarray(freq_hz, dtype=np.float64) / C_LIGHT


def efp_disk(rho, dl):
    """Voltage pattern of a uniform disk: 2 J1(x)/x with x = pi D_lambda rho (1 at rho = 0)."""
    x = math.pi * dl * np.asarray(rho, dtype=np.float64)
    out = np.ones_like(x)
    nz = np.abs(x) > 1e-12
    out[nz] = 2.0 * special.j1(x[nz]) / x[nz]
    return out


def efp_gauss(rho, alpha):
    """Main-lobe Gaussian voltage pattern exp(-alpha^2 rho^2) (Sec. 3)."""
    return np.exp(-(alpha ** 2) * np.asarray(rho, dtype=np.float64) ** 2)


def airy_half_power_x() -> float:
    """x_h with (2 J1(x_h)/x_h)^2 = 1/2, by bisection on [1, 2]."""
    lo, hi = 1.0, 2.0
    f = lambda x: (2.0 * special.j1(x) / x) ** 2 - 0.5
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if f(lo) * f(mid) <= 0.0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


def alpha_per_dlambda_disk() -> float:
    """alpha / D_lambda of the Gaussian power beam with the Airy half-power width:
    exp(-2 alpha^2 rho_h^2) = 1/2 at rho_h = x_h / (pi D_lambda)."""
    return math.pi * math.sqrt(math.log(2.0) / 2.0) / airy_half_power_x()


def aperture_disk(q, dl):
    """A°(q) for the uniform disk, q in wavelengths: overlap area of two disks
    of radius R = D_lambda/2 whose centres are q apart, over (pi R^2)^2."""
    R = 0.5 * dl
    q = np.minimum(np.abs(np.asarray(q, dtype=np.float64)), 2.0 * R)
    ovl = 2.0 * R * R * np.arccos(q / (2.0 * R)) - 0.5 * q * np.sqrt(np.maximum(4.0 * R * R - q * q, 0.0))
    return ovl / (math.pi * R * R) ** 2


def aperture_gauss(q, alpha):
    """A°(q) for the Gaussian model: (pi / 2 alpha^2) exp(-pi^2 q^2 / (2 alpha^2))."""
    q = np.asarray(q, dtype=np.float64)
    return (math.pi / (2.0 * alpha ** 2)) * np.exp(-(math.pi ** 2) * q * q / (2.0 * alpha ** 2))


def table_len(kind: str, dl: float, du: float, ov: int, support: int) -> int:
    rho_max = dl / du if kind == "disk" else 0.5 * support * math.sqrt(2.0)
    return int(math.floor(ov * rho_max)) + 2


def radial_table(kind: str, dl: float, alpha: float, du: float, ov: int, support: int) -> np.ndarray:
    """A°(n du / ov) * du^2 for n = 0 .. len-1 (FP64)."""
    n = np.arange(table_len(kind, dl, du, ov, support), dtype=np.float64)
    q = n * du / ov
    if kind == "disk":
        a = aperture_disk(q, dl)
        a[q >= dl] = 0.0
    elif kind == "gauss":
        a = aperture_gauss(q, alpha)
    else:
        raise ValueError(kind)
    return a * du * du
