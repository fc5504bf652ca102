"""Pins of the oracle's exact disk kernel (the transform of two shifted
uniform-disk patterns' product, Sec. 3's "more accurate function").

Each test checks ``oracle.exact`` against something other than itself: the
closed-form lens area and the disk's own transform (Airy, scipy Bessel J1),
scipy's adaptive double quadrature over the lens, finite differences, and the
direct-sum visibilities of Eq. ME (``oracle.closed_form``), which the exact
kernel must reproduce at any offset to the gridding error of the zero-offset
case, where the Gaussian approximation of Eq. AIJPOINTING drifts away.
"""
import dataclasses
import math

import numpy as np
import pytest
from scipy import integrate, special

from paper_1709_08681_gb300 import inputs as I
from oracle import aperture, closed_form, exact, psc

import cases

R = 45.0   # disk radius in wavelengths (25 m at 1.08 GHz)


def test_zero_offset_gives_the_lens_area():
    rho = np.linspace(0.0, 2.2 * R, 57)
    O, Oa, Ob = exact.overlap(rho, 0.0, 0.0, R)
    area = aperture.aperture_disk(rho, 2 * R) * (math.pi * R * R) ** 2
    area[rho >= 2 * R] = 0.0
    assert np.allclose(O, area, rtol=1e-13, atol=1e-9 * R * R)
    assert np.all(Oa == 0.0) and np.all(Ob == 0.0)


@pytest.mark.parametrize("dl", [1e-5, 3e-4, 2e-3, 2e-2])
def test_zero_separation_gives_the_disk_transform(dl):
    """At du = 0 the lens is the whole disk: O = pi R^2 2 J1(x) / x, x = 2 pi R |dl|."""
    for ang in (0.0, 0.7, 2.0):
        a, b = dl * math.cos(ang), dl * math.sin(ang)
        O, _, _ = exact.overlap(0.0, a, b, R)
        x = 2 * math.pi * R * dl
        assert O == pytest.approx(math.pi * R * R * 2 * special.j1(x) / x, rel=1e-12)


@pytest.mark.parametrize("rho,a,b", [(10.0, 3e-4, 1e-4), (47.0, -2e-4, 5e-4), (85.0, 1e-3, -7e-4),
                                     (30.0, 4e-3, 2.5e-3)])
def test_overlap_matches_adaptive_double_quadrature(rho, a, b):
    """scipy dblquad over the lens |w -+ du/2| <= R in the du-aligned frame."""
    W = R - rho / 2

    def hh(wp):
        return math.sqrt(max(R * R - (abs(wp) + rho / 2) ** 2, 0.0))

    kw = dict(epsabs=1e-10, epsrel=1e-12)
    O_ref = integrate.dblquad(lambda wq, wp: math.cos(2 * math.pi * (a * wp + b * wq)), -W, W,
                              lambda wp: -hh(wp), hh, **kw)[0]
    Oa_ref = integrate.dblquad(lambda wq, wp: -2 * math.pi * wp * math.sin(2 * math.pi * (a * wp + b * wq)),
                               -W, W, lambda wp: -hh(wp), hh, **kw)[0]
    Ob_ref = integrate.dblquad(lambda wq, wp: -2 * math.pi * wq * math.sin(2 * math.pi * (a * wp + b * wq)),
                               -W, W, lambda wp: -hh(wp), hh, **kw)[0]
    O, Oa, Ob = exact.overlap(rho, a, b, R)
    scale = math.pi * R * R
    assert abs(O - O_ref) < 1e-9 * scale
    assert abs(Oa - Oa_ref) < 1e-9 * scale * 2 * math.pi * R
    assert abs(Ob - Ob_ref) < 1e-9 * scale * 2 * math.pi * R


def test_overlap_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    rho = rng.uniform(0, 2 * R, 40)
    a = rng.uniform(-1e-3, 1e-3, 40)
    b = rng.uniform(-1e-3, 1e-3, 40)
    h = 1e-7
    O, Oa, Ob = exact.overlap(rho, a, b, R)
    fa = (exact.overlap(rho, a + h, b, R)[0] - exact.overlap(rho, a - h, b, R)[0]) / (2 * h)
    fb = (exact.overlap(rho, a, b + h, R)[0] - exact.overlap(rho, a, b - h, R)[0]) / (2 * h)
    scale = math.pi * R * R * 2 * math.pi * R
    assert np.max(np.abs(Oa - fa)) < 1e-7 * scale
    assert np.max(np.abs(Ob - fb)) < 1e-7 * scale


def test_overlap_is_even_in_each_offset_component():
    rho, a, b = 33.0, 6e-4, -2e-4
    ref = exact.overlap(rho, a, b, R)[0]
    for s in ((-1, 1), (1, -1), (-1, -1)):
        assert exact.overlap(rho, s[0] * a, s[1] * b, R)[0] == pytest.approx(ref, rel=1e-14)


@pytest.mark.parametrize("sigma", [0.0, 20.0, 120.0, 300.0])
def test_exact_kernel_matches_direct_sum_at_any_offset(sigma):
    """The exact kernel leaves only the gridding error of the zero-offset case
    (7e-5 here) at every offset; the Gaussian factor of Eq. AIJPOINTING does
    not (9e-4 at 120", 1e-2 at 300")."""
    m, sky, lm, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=sigma, freqs=(1.2e9, 1.4e9))
    Vc = closed_form.visibilities(m.uvw_m, m.freq_hz, m.n_ant, sky, lm, "disk", 25.0, m.alpha_per_dlambda)
    Ve, _ = psc.predict(dataclasses.replace(m, kernel="exact"), lm, False)
    assert cases.rel_l2(Ve, Vc) < 1e-4
    if sigma >= 120.0:
        Vg, _ = psc.predict(m, lm, False)
        assert cases.rel_l2(Vg, Vc) > 5e-4


def test_exact_kernel_at_zero_offset_equals_the_radial_kernel():
    m, _, lm, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=0.0, freqs=(1.2e9, 1.4e9))
    V, dV = psc.predict(m, lm)
    Ve, dVe = psc.predict(dataclasses.replace(m, kernel="exact"), lm)
    assert cases.rel_l2(Ve, V) < 1e-13
    assert cases.rel_l2(dVe, dV) < 1e-12


def test_exact_derivatives_match_finite_differences():
    m, _, lm, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=120.0)
    m = dataclasses.replace(m, kernel="exact")
    _, dV = psc.predict(m, lm)
    ij = m.antenna_pairs()
    h = 1e-3 * I.ARCSEC
    for a in (0, 3):
        for ax in (0, 1):
            lp, ln = lm.copy(), lm.copy()
            lp[a, ax] += h
            ln[a, ax] -= h
            fd = (psc.predict(m, lp, False)[0] - psc.predict(m, ln, False)[0]) / (2 * h)
            an = np.zeros_like(fd)
            for bl, (i, j) in enumerate(ij):
                if i == a:
                    an[:, bl] = dV[ax][:, bl]
                elif j == a:
                    an[:, bl] = dV[2 + ax][:, bl]
            assert cases.rel_l2(an, fd) < 1e-6


def test_predict_points_equals_predict_with_the_exact_kernel():
    m, _, lm, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=60.0, freqs=(1.2e9, 1.4e9))
    m = dataclasses.replace(m, kernel="exact")
    V, dV = psc.predict(m, lm)
    rng = np.random.default_rng(1)
    t, b, c = rng.integers(0, V.shape[0], 20), rng.integers(0, V.shape[1], 20), rng.integers(0, V.shape[2], 20)
    Vp, dVp = psc.predict_points(m, lm, t, b, c)
    assert np.allclose(Vp, V[t, b, c], rtol=1e-13, atol=1e-15)
    assert np.allclose(dVp, dV[:, t, b, c], rtol=1e-13, atol=1e-12)
