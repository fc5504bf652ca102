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
