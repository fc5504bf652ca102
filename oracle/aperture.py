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

A tabulated A° (Sec. 3: A° may hold a-priori primary-beam effects; Alg. 1
pre-computes it) is given on the scale of the dish: samples T_k of
T(x) = A°(x D_lambda) D_lambda^2 at x = k / (K - 1), linear between samples,
and A° = 0 from q = D_lambda on (the autocorrelation of an aperture of
diameter D ends at one diameter).  The samples are used as given.

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


def efp_annulus(rho, dl, eps):
    """Voltage pattern of a uniformly illuminated disk with a central blockage
    of eps times its diameter: the disk's Airy pattern less the blockage's,
    [2 J1(x)/x - eps^2 2 J1(eps x)/(eps x)] / (1 - eps^2), x = pi D_lambda rho
    (1 at rho = 0)."""
    if eps <= 0.0:
        return efp_disk(rho, dl)
    return (efp_disk(rho, dl) - eps * eps * efp_disk(rho, eps * dl)) / (1.0 - eps * eps)


def circle_overlap(a, b, d):
    """Area common to two disks of radii a and b whose centres are d apart."""
    d = np.abs(np.asarray(d, dtype=np.float64))
    out = np.zeros_like(d)
    inside = d <= abs(a - b)
    out[inside] = math.pi * min(a, b) ** 2
    part = (~inside) & (d < a + b)
    dd = d[part]
    c1 = np.clip((dd * dd + a * a - b * b) / (2.0 * dd * a), -1.0, 1.0)
    c2 = np.clip((dd * dd + b * b - a * a) / (2.0 * dd * b), -1.0, 1.0)
    k = np.maximum((-dd + a + b) * (dd + a - b) * (dd - a + b) * (dd + a + b), 0.0)
    out[part] = a * a * np.arccos(c1) + b * b * np.arccos(c2) - 0.5 * np.sqrt(k)
    return out


def annulus_table_samples(n: int, eps: float) -> np.ndarray:
    """A° D_lambda^2 of the blocked disk (efp_annulus) on the dish scale, n
    samples over x = q / D_lambda in [0, 1]: the autocorrelation of the
    annulus of outer radius 1/2 and inner radius eps/2, over its area squared."""
    x = np.linspace(0.0, 1.0, n)
    R, r = 0.5, 0.5 * eps
    auto = circle_overlap(R, R, x) - 2.0 * circle_overlap(R, r, x) + circle_overlap(r, r, x)
    area = math.pi * (R * R - r * r)
    return auto / (area * area)


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


def aperture_table(q, dl, samples):
    """A°(q) from dish-scale samples T_k (see the module docstring)."""
    x = np.abs(np.asarray(q, dtype=np.float64)) / dl
    T = np.asarray(samples, dtype=np.float64)
    xk = np.linspace(0.0, 1.0, T.size)
    out = np.interp(x, xk, T) / (dl * dl)
    out[x >= 1.0] = 0.0
    return out


def disk_table_samples(n: int) -> np.ndarray:
    """The uniform disk on the dish scale: T(x) = (8 / pi^2)(acos x - x sqrt(1 - x^2)),
    n samples over [0, 1]."""
    x = np.linspace(0.0, 1.0, n)
    return 8.0 / math.pi ** 2 * (np.arccos(x) - x * np.sqrt(np.maximum(1.0 - x * x, 0.0)))


def table_len(kind: str, dl: float, du: float, ov: int, support: int) -> int:
    rho_max = 0.5 * support * math.sqrt(2.0) if kind == "gauss" else dl / du
    return int(math.floor(ov * rho_max)) + 2


def radial_table(kind: str, dl: float, alpha: float, du: float, ov: int, support: int, samples=None) -> np.ndarray:
    """A°(n du / ov) * du^2 for n = 0 .. len-1 (FP64); kind "table" takes the
    dish-scale samples."""
    n = np.arange(table_len(kind, dl, du, ov, support), dtype=np.float64)
    q = n * du / ov
    if kind == "disk":
        a = aperture_disk(q, dl)
        a[q >= dl] = 0.0
    elif kind == "gauss":
        a = aperture_gauss(q, alpha)
    elif kind == "table":
        a = aperture_table(q, dl, samples)
    else:
        raise ValueError(kind)
    return a * du * du
