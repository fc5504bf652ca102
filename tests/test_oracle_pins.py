"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a library
routine (numpy FFT, scipy Bessel functions and quadrature), a closed form
(the direct-sum visibilities of Eq. ME, Hankel-transform identities), an
invariant (Hermitian symmetry, the beam-centre null of Sec. 5), finite
differences (Eqs. DAIJPOINTING and DCHIDD), the statistics of the thermal
noise, or numbers the paper prints (tests/golden/paper_values.json).
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate, special

from paper_1709_08681_gb300 import inputs as I
from oracle import aperture, closed_form, lm as LM, model_grid, psc

import cases

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


# ------------------------------------------------------------------ model grid

def test_grid_matches_numpy_fft():
    rng = np.random.default_rng(0)
    N, Ng = 16, 40
    img = rng.normal(size=(N, N))
    G = model_grid.grid_from_image(img, Ng)
    P = np.zeros((Ng, Ng))
    r = (np.arange(N) - N // 2) % Ng
    P[np.ix_(r, r)] = img
    ref = np.fft.fftshift(Ng * Ng * np.fft.ifft2(P))
    assert np.max(np.abs(G - ref)) < 1e-11 * np.max(np.abs(ref))


def test_grid_single_pixel_is_plane_wave():
    N, Ng, cell = 32, 96, 5.0 * I.ARCSEC
    img = np.zeros((N, N))
    row, col = 21, 9
    img[row, col] = 0.7
    G = model_grid.grid_from_image(img, Ng)
    du = 1.0 / (Ng * cell)
    u = (np.arange(Ng) - Ng // 2) * du
    l, m = (col - N // 2) * cell, (row - N // 2) * cell
    ref = 0.7 * np.exp(2j * np.pi * (u[None, :] * l + u[:, None] * m))
    assert np.max(np.abs(G - ref)) < 1e-10


def test_grid_image_equals_components():
    N, Ng, cell = 64, 128, 10.0 * I.ARCSEC
    sky = I.sky_points(12, 4 * I.ARCMIN, N, cell, ("loguniform", 0.01, 1.0), 3)
    G1 = model_grid.grid_from_image(I.sky_image(sky, N, cell).astype(np.float64), Ng)
    G2 = model_grid.grid_from_components(sky, Ng, 1.0 / (Ng * cell))
    # the image is stored as float32 pixels
    assert cases.rel_l2(G1, G2) < 1e-6


# ------------------------------------------------------------------ aperture

@pytest.mark.parametrize("dl", [50.0, 116.8])
def test_disk_aperture_transforms_to_airy_power_beam(dl):
    """Inverse Hankel transform of A° is (2 J1(x)/x)^2, x = pi D_lambda rho."""
    for rho in [0.0, 0.3 / dl, 0.8 / dl, 1.7 / dl]:
        f = lambda q: aperture.aperture_disk(q, dl) * special.j0(2 * math.pi * q * rho) * q
        pb = 2 * math.pi * integrate.quad(f, 0.0, dl, limit=400, epsabs=1e-13, epsrel=1e-11)[0]
        ref = float(aperture.efp_disk(np.array([rho]), dl)[0]) ** 2
        assert abs(pb - ref) < 1e-8


def test_gauss_aperture_transforms_to_gauss_power_beam():
    alpha = 133.6
    for rho in [0.0, 0.002, 0.006, 0.01]:
        f = lambda q: aperture.aperture_gauss(q, alpha) * special.j0(2 * math.pi * q * rho) * q
        pb = 2 * math.pi * integrate.quad(f, 0.0, 20 * alpha / math.pi, limit=400, epsabs=1e-13)[0]
        assert abs(pb - math.exp(-2 * alpha ** 2 * rho ** 2)) < 1e-9


def test_alpha_constant_matches_airy_half_power():
    a = aperture.alpha_per_dlambda_disk()
    assert abs(a - I.ALPHA_PER_DLAMBDA_DISK) < 1e-9
    dl = 100.0
    x_h = aperture.airy_half_power_x()
    rho_h = x_h / (math.pi * dl)
    assert abs((2 * special.j1(x_h) / x_h) ** 2 - 0.5) < 1e-12
    assert abs(math.exp(-2 * (a * dl) ** 2 * rho_h ** 2) - 0.5) < 1e-9


def test_table_nodes_support_and_normalisation():
    dl, du, ov = 116.8, 8.4, 20
    tab = aperture.radial_table("disk", dl, 0.0, du, ov, 32)
    assert len(tab) == int(math.floor(ov * dl / du)) + 2
    assert tab[-1] == 0.0 and tab[-2] > 0.0
    n = np.arange(len(tab) - 1)
    assert np.allclose(tab[:-1], aperture.aperture_disk(n * du / ov, dl) * du * du, rtol=1e-14, atol=0)
    # sum of the kernel over a fine 2-D lattice ~ its integral, PB(0) = 1
    h = dl / 200
    q = (np.arange(-400, 401)) * h
    s = aperture.aperture_disk(np.hypot(q[:, None], q[None, :]), dl).sum() * h * h
    assert abs(s - 1.0) < 1e-4


def test_decorrelation_claim_of_the_paper():
    g = GOLDEN["decorrelation"]
    dl = 100.0
    alpha = I.ALPHA_PER_DLAMBDA_DISK * dl
    d = g["max_dl_fraction_of_beam"] / dl          # 2% of lambda/D
    assert 1.0 - math.exp(-(alpha * d) ** 2 / 2.0) < g["max_amplitude_error"]


def test_offset_fraction_of_beam():
    g = GOLDEN["offset_fraction_of_beam"]
    beam = 1.0 / float(aperture.d_lambda(g["diam_m"], g["freq_hz"]))
    frac = g["offset_arcsec"] * I.ARCSEC / beam
    assert abs(frac - g["fraction"]) < 0.25 * g["fraction"]


def test_signal_profile_null_and_peak():
    """|E dE/dl| (Sec. 5) vanishes at the centre and peaks near half power."""
    dl = 100.0
    rho = np.linspace(0.0, 0.9 / dl, 20001)
    e = aperture.efp_disk(rho, dl)
    h = 1e-4 / dl
    de = (aperture.efp_disk(rho + h, dl) - aperture.efp_disk(np.abs(rho - h), dl)) / (2 * h)
    prof = np.abs(e * de)
    assert prof[0] < 1e-6 * prof.max()
    r_peak = rho[np.argmax(prof)]
    r_half = aperture.airy_half_power_x() / (math.pi * dl)
    tol = GOLDEN["signal_profile"]["peak_over_half_power_radius_tolerance"]
    assert abs(r_peak / r_half - 1.0) < tol


# ------------------------------------------------------------------ degridding

@pytest.mark.parametrize("sigma", [0.0, 20.0, 120.0])
def test_gauss_prediction_matches_direct_sum(sigma):
    """Eq. AIJPOINTING is exact for the Gaussian pattern: only gridding error is left."""
    m, sky, lm, _ = cases.problem(cases.GAUSS_SMALL, sigma_arcsec=sigma)
    V, _ = psc.predict(m, lm, False)
    Vc = closed_form.visibilities(m.uvw_m, m.freq_hz, m.n_ant, sky, lm, "gauss", 25.0, m.alpha_per_dlambda)
    assert cases.rel_l2(V, Vc) < 1e-4


@pytest.mark.parametrize("sigma", [0.0, 20.0])
def test_disk_prediction_matches_direct_sum(sigma):
    """Uniform disk at the paper's offset scale: within 1e-3 of the direct sum."""
    m, sky, lm, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=sigma, freqs=(1.2e9, 1.4e9))
    V, _ = psc.predict(m, lm, False)
    Vc = closed_form.visibilities(m.uvw_m, m.freq_hz, m.n_ant, sky, lm, "disk", 25.0, m.alpha_per_dlambda)
    assert cases.rel_l2(V, Vc) < 1e-3


def test_sign_error_in_ramp_would_fail():
    """The ramp sign matters at these offsets: flipping it breaks the match."""
    m, sky, lm, _ = cases.problem(cases.GAUSS_SMALL, sigma_arcsec=120.0)
    V, _ = psc.predict(m, -lm, False)
    Vc = closed_form.visibilities(m.uvw_m, m.freq_hz, m.n_ant, sky, lm, "gauss", 25.0, m.alpha_per_dlambda)
    assert cases.rel_l2(V, Vc) > 1e-2


@pytest.mark.parametrize("decorrelation", [0, 1])
def test_derivatives_match_finite_differences(decorrelation):
    m, _, lm, _ = cases.problem(cases.DISK_SMALL, decorrelation=decorrelation, sigma_arcsec=60.0)
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
            for b, (i, j) in enumerate(ij):
                if i == a:
                    an[:, b] = dV[ax][:, b]
                elif j == a:
                    an[:, b] = dV[2 + ax][:, b]
            assert cases.rel_l2(an, fd) < 1e-6


def test_hermitian_symmetry():
    m, _, lm, _ = cases.problem(cases.DISK_SMALL)
    V, _ = psc.predict(m, lm, False)
    m2 = psc.Model(**{**m.__dict__, "uvw_m": -m.uvw_m})
    V2, _ = psc.predict(m2, lm, False)
    assert np.max(np.abs(V2 - np.conj(V))) < 1e-12 * np.max(np.abs(V))


def test_beam_centre_null():
    """A source at the pointing centre gives no pointing signal (Sec. 5)."""
    kind, N, cell_as, Ng = cases.DISK_SMALL
    uvw, freq = cases.geometry(n_ant=6)
    img = np.zeros((N, N))
    img[N // 2, N // 2] = 1.0
    m = psc.Model(uvw_m=uvw, freq_hz=freq, n_ant=6, grid=model_grid.grid_from_image(img, Ng),
                  cell_rad=cell_as * I.ARCSEC, support=32, oversample=20, ap_kind=kind, diam_m=25.0,
                  alpha_per_dlambda=I.ALPHA_PER_DLAMBDA_DISK, decorrelation=1)
    V, dV = psc.predict(m, np.zeros((6, 2)))
    scale = math.pi * float(aperture.d_lambda(25.0, freq[0])) * np.max(np.abs(V))
    assert np.max(np.abs(dV)) < 1e-4 * scale
    assert np.allclose(V, 1.0, atol=2e-4)


# ------------------------------------------------------------------ chi^2, gradient, normals

def _noisy(m, lm_true, sigma=1e-3, seed=7):
    V, _ = psc.predict(m, lm_true, False)
    noise = I.complex_noise(V.shape, sigma, seed)
    return V + noise, np.full(V.shape, 1.0 / sigma ** 2)


def test_gradient_matches_finite_differences_of_chi2():
    m, _, lmt, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=30.0)
    vobs, w = _noisy(m, lmt)
    lm = np.zeros_like(lmt)
    chi2, g, H, X = psc.chi2_grad_normal(m, lm, vobs, w)
    h = 1e-3 * I.ARCSEC
    for a in range(m.n_ant):
        for ax in (0, 1):
            lp, ln = lm.copy(), lm.copy()
            lp[a, ax] += h
            ln[a, ax] -= h
            fd = (psc.chi2_grad_normal(m, lp, vobs, w)[0] - psc.chi2_grad_normal(m, ln, vobs, w)[0]) / (2 * h)
            assert abs(fd - g[a, ax]) < 1e-6 * np.max(np.abs(g))


def test_normals_equal_hessian_at_exact_fit():
    """With noiseless data at the true offsets the Gauss-Newton matrix is the
    Hessian of chi^2; check it against second differences."""
    m, _, lmt, _ = cases.problem(cases.DISK_SMALL, n_ant=4, sigma_arcsec=30.0)
    vobs, _ = psc.predict(m, lmt, False)
    chi2, g, H, X = psc.chi2_grad_normal(m, lmt, vobs)
    _, A = psc.assemble_full(m.n_ant, g, H, X)
    h = 2e-2 * I.ARCSEC
    n = 2 * m.n_ant
    f = lambda p: psc.chi2_grad_normal(m, p.reshape(-1, 2), vobs)[0]
    p0 = lmt.reshape(-1)
    for a in range(n):
        for b in range(a, n):
            ea, eb = np.eye(n)[a] * h, np.eye(n)[b] * h
            fd = (f(p0 + ea + eb) - f(p0 + ea - eb) - f(p0 - ea + eb) + f(p0 - ea - eb)) / (4 * h * h)
            assert abs(fd - A[a, b]) < 1e-4 * np.max(np.abs(A))


def test_blocks_assemble_to_jacobian_normals():
    m, _, lmt, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=30.0)
    vobs, w = _noisy(m, lmt)
    chi2, g, H, X = psc.chi2_grad_normal(m, lmt * 0.5, vobs, w)
    G, A = psc.assemble_full(m.n_ant, g, H, X)
    chi2b, gb, Ab = psc.full_normal(m, lmt * 0.5, vobs, w)
    assert abs(chi2 - chi2b) < 1e-12 * chi2
    assert np.max(np.abs(G - gb)) < 1e-10 * np.max(np.abs(gb))
    assert np.max(np.abs(A - Ab)) < 1e-10 * np.max(np.abs(Ab))


def test_chi2_at_truth_is_thermal():
    m, _, lmt, _ = cases.problem(cases.DISK_SMALL, n_ant=10, n_time=12, sigma_arcsec=20.0)
    vobs, w = _noisy(m, lmt)
    chi2 = psc.chi2_grad_normal(m, lmt, vobs, w)[0]
    n2 = 2 * vobs.size
    assert abs(chi2 / n2 - 1.0) < 5.0 / math.sqrt(n2)


# ------------------------------------------------------------------ LM

def _full_eval(m, vobs, w=None):
    def ev(p):
        chi2, g, H, X = psc.chi2_grad_normal(m, p, vobs, w)
        G, A = psc.assemble_full(m.n_ant, g, H, X)
        return chi2, G, A
    return ev


@pytest.mark.parametrize("spec", [cases.GAUSS_SMALL, cases.DISK_SMALL])
def test_noiseless_recovery_is_exact(spec):
    m, _, lmt, _ = cases.problem(spec, n_src=8)
    vobs, _ = psc.predict(m, lmt, False)
    sol, rep = LM.solve_full(_full_eval(m, vobs), np.zeros_like(lmt))
    assert rep.reason in ("step", "chi2")
    assert np.max(np.abs(sol - lmt)) < 1e-5 * I.ARCSEC


def test_block_and_full_reach_the_same_minimum():
    m, _, lmt, _ = cases.problem(cases.DISK_SMALL, n_ant=6, n_src=8)
    vobs, w = _noisy(m, lmt)
    sf, rf = LM.solve_full(_full_eval(m, vobs, w), np.zeros_like(lmt))
    sb, rb = LM.solve_block(lambda p: psc.chi2_grad_normal(m, p, vobs, w), np.zeros_like(lmt),
                            LM.Options(max_iter=400))
    assert np.max(np.abs(sb - sf)) < 0.01 * I.ARCSEC
    assert rb.chi2 >= rf.chi2 * (1 - 1e-9)


def test_scatter_matches_fisher_information():
    """Scatter of the solutions over noise draws ~ sqrt(diag(2 H^-1))
    (the noise-limited behaviour of Sec. 5)."""
    m, _, lmt, _ = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=6, n_src=8)
    v0, _ = psc.predict(m, lmt, False)
    sigma = 3e-3
    w = np.full(v0.shape, 1.0 / sigma ** 2)
    sols = []
    for s in range(40):
        vobs = v0 + I.complex_noise(v0.shape, sigma, 1000 + s)
        sol, _ = LM.solve_full(_full_eval(m, vobs, w), lmt)
        sols.append(sol.reshape(-1))
    spread = np.std(np.asarray(sols), axis=0)
    chi2, g, H, X = psc.chi2_grad_normal(m, lmt, v0, w)
    _, A = psc.assemble_full(m.n_ant, g, H, X)
    pred = np.sqrt(np.diag(2.0 * np.linalg.inv(A)))
    ratio = spread / pred
    assert 0.7 < np.median(ratio) < 1.3


def test_predict_points_equals_predict():
    m, _, lm, _ = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=7, freqs=(1.3e9, 1.4e9), sigma_arcsec=40.0)
    V, dV = psc.predict(m, lm)
    rng = np.random.default_rng(0)
    t, b, c = rng.integers(0, 7, 30), rng.integers(0, 10, 30), rng.integers(0, 2, 30)
    Vp, dVp = psc.predict_points(m, lm, t, b, c)
    assert np.allclose(Vp, V[t, b, c], rtol=1e-13, atol=1e-15)
    assert np.allclose(dVp, dV[:, t, b, c], rtol=1e-13, atol=1e-12)


def test_lm_stops_on_a_rejected_step_below_ten_tolerances():
    """The rejected-step stop rule of the LM (Terminate() is left to the
    minimiser, Sec. 2.2).  chi^2 is a quadratic plus a bump within 1.5 step
    tolerances of its minimum (standing in for rounding noise there).  From a
    start 2 tolerances away, the Gauss-Newton trial lands next to the minimum,
    inside the bump, and is rejected; its step (about 2 tolerances) is above
    the plain step rule, so only the rejected-step rule can stop the solve:
    after one iteration, at the start, within 10 tolerances of the minimum.
    Without the bump the trial is accepted and the solve converges."""
    tol = LM.Options().step_tol
    H = np.array([[4.0, 1.0], [1.0, 3.0]])
    x_min = np.array([3e-5, -2e-5])

    def evaluate(bump):
        def f(p):
            d = np.ravel(p) - x_min
            chi2 = 0.5 * d @ H @ d               # about 8 tol^2 = 2e-18 at the start
            if bump and 0.0 < np.max(np.abs(d)) < 1.5 * tol:
                chi2 += 1e-15
            return chi2, H @ d, H
        return f

    start = x_min + np.array([2.0 * tol, 0.0])
    p, rep = LM.solve_full(evaluate(True), start)
    assert rep.reason == "step" and rep.n_iter == 1 and rep.n_eval == 2, rep
    assert np.array_equal(np.ravel(p), start)
    assert np.max(np.abs(np.ravel(p) - x_min)) < 10 * tol
    p0, rep0 = LM.solve_full(evaluate(False), start)
    assert rep0.reason in ("step", "chi2"), rep0
    assert np.max(np.abs(np.ravel(p0) - x_min)) < tol
