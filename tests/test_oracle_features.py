"""Pins of the oracle's learned-initialiser features (oracle/features.py)
against the core oracle and against cases with a known answer."""
import numpy as np
import pytest

from paper_1709_08681_gb300 import inputs as I
from oracle import features as F, psc

import cases

SIG = 30.0 * I.ARCSEC


def test_stencil_model_equals_predict_with_one_antenna_offset():
    m, _, _, _ = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=4, freqs=(1.3e9, 1.4e9))
    Vs = F.stencil_model(m, SIG)
    ij = m.antenna_pairs()
    for s in (0, 7, 24):
        a, b = F.STENCIL[s]
        for ant in (0, 3):          # first and second end of its baselines
            lm = np.zeros((m.n_ant, 2))
            lm[ant] = (a * SIG, b * SIG)
            V, _ = psc.predict(m, lm, False)
            for bl, (i, j) in enumerate(ij):
                if ant in (i, j):
                    assert np.allclose(Vs[s][:, bl], V[:, bl], rtol=1e-12, atol=1e-14)


def test_centre_point_is_unity_on_noiseless_zero_offset_data():
    m, _, _, _ = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=6)
    V, _ = psc.predict(m, np.zeros((5, 2)), False)
    f = F.features(m, V, None, SIG)
    c = F.STENCIL.index((0, 0))
    assert f.shape == (5, F.N_FEAT)
    assert np.allclose(f[:, 2 + c], 1.0, atol=1e-12)
    assert np.allclose(f[:, 27 + c], 0.0)
    assert np.all(f[:, 27:] >= -1e-12)          # zero offsets are the chi^2 minimum here
    assert np.max(np.abs(f[:, :2])) < 1e-9


def test_offset_on_the_stencil_is_found_exactly():
    m, _, _, _ = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=6)
    s = F.STENCIL.index((1, -1))
    lm = np.zeros((5, 2))
    lm[0] = (SIG, -SIG)
    V, _ = psc.predict(m, lm, False)
    f = F.features(m, V, None, SIG)
    # chi^2 at the true trial offset vanishes: C = -chi2(0) / sum w |V_0|^2 there
    V0, _ = psc.predict(m, np.zeros((5, 2)), False)
    ij = m.antenna_pairs()
    b0 = [k for k, (i, j) in enumerate(ij) if 0 in (i, j)]
    chi0 = np.sum(np.abs(V[:, b0] - V0[:, b0]) ** 2)
    y0 = np.sum(np.abs(V0[:, b0]) ** 2)
    assert abs(f[0, 27 + s] + chi0 / y0) < 1e-12
    assert abs(f[0, 2 + s] - 1.0) < 1e-12     # amplitude ratio is one there
    assert np.argmin(f[0, 27:]) == s


def test_time_stride_keeps_every_kth_step():
    m, _, lmt, _ = cases.problem(cases.DISK_SMALL, n_ant=4, n_time=9)
    V, _ = psc.predict(m, lmt, False)
    m3 = psc.Model(**{**m.__dict__, "uvw_m": m.uvw_m[::3]})
    f1 = F.features(m, V, None, SIG, time_stride=3)
    f2 = F.features(m3, V[::3], None, SIG, time_stride=1)
    assert np.allclose(f1[:, 2:], f2[:, 2:], rtol=1e-12)


def _chi2(m, lm, vobs):
    V, _ = psc.predict(m, lm, False)
    return float(np.sum(np.abs(vobs - V) ** 2))


def test_newton_step_columns_follow_the_offset_and_finite_differences():
    """Columns 0-1 are the block Newton step -H_ii^-1 g_i at zero offsets over
    sigma_prior.  With one antenna offset by a small delta (unequal l and m, so
    a swapped pair or a flipped sign shows) on noiseless data, the step of that
    antenna is delta to first order, and every antenna's step equals the one
    formed from a central finite-difference gradient and Hessian of chi^2
    (a route that never uses the analytic derivatives of Eq. DAIJPOINTING)."""
    m, _, _, _ = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=6, freqs=(1.3e9, 1.45e9))
    n = m.n_ant
    delta = np.array([3.0, -1.2]) * I.ARCSEC
    lm = np.zeros((n, 2))
    lm[2] = delta
    vobs, _ = psc.predict(m, lm, False)
    f = F.features(m, vobs, None, SIG)
    step = f[:, :2] * SIG
    # antenna 2: the offset itself, to first order in delta
    assert np.allclose(step[2], delta, rtol=0.03, atol=0.02 * I.ARCSEC)
    # every antenna: -H_ii^-1 g_i with g and H from finite differences of chi^2
    h = 0.05 * I.ARCSEC
    z = np.zeros((n, 2))
    for a in range(n):
        g = np.zeros(2)
        H = np.zeros((2, 2))
        for p in range(2):
            e = np.zeros((n, 2))
            e[a, p] = h
            g[p] = (_chi2(m, z + e, vobs) - _chi2(m, z - e, vobs)) / (2 * h)
            for q in range(2):
                d = np.zeros((n, 2))
                d[a, q] = h
                H[p, q] = (_chi2(m, z + e + d, vobs) - _chi2(m, z + e - d, vobs)
                           - _chi2(m, z - e + d, vobs) + _chi2(m, z - e - d, vobs)) / (4 * h * h)
        # the full Hessian at small residuals is the Gauss-Newton block to O(delta)
        s_fd = -np.linalg.solve(0.5 * (H + H.T), g)
        assert np.allclose(step[a], s_fd, rtol=0.05, atol=0.01 * np.linalg.norm(delta)), a
    # the antennas that share no term with antenna 2's offset see a smaller,
    # same-signed pull: baseline (i, 2) moves with l_i + l_2
    for a in (0, 1, 3, 4):
        assert np.dot(step[a], delta) > 0
        assert np.linalg.norm(step[a]) < np.linalg.norm(step[2])
