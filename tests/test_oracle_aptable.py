"""Pins of the oracle's tabulated aperture (PSC_AP_TABLE): A° given on the
dish scale, T(x) = A°(x D_lambda) D_lambda^2 at x = k/(K-1), linear between
samples.  The uniform disk's samples must give the disk's own radial
tables and predictions; the blocked disk's autocorrelation samples must
integrate to PB(0) = 1, reduce to the disk without blockage, and give
predictions that match the direct sum of Eq. ME with the blocked disk's
closed-form voltage pattern."""
import math

import numpy as np
import pytest
from scipy import integrate, special

from oracle import aperture, closed_form, psc

import cases

EPS = 0.2          # blockage: a central obstruction of a fifth of the dish diameter


def _table_model(m, samples):
    return psc.Model(**{**m.__dict__, "ap_kind": "table", "ap_table": samples})


def test_disk_samples_give_the_disk_tables_and_predictions():
    m, _, lm, _ = cases.problem(cases.DISK_SMALL, freqs=(1.2e9, 1.4e9), sigma_arcsec=20.0)
    mt = _table_model(m, aperture.disk_table_samples(20001))
    for a, b in zip(m.tables(), mt.tables()):
        assert a.shape == b.shape
        assert np.max(np.abs(a - b)) < 1e-7 * np.max(a)
    V, dV = psc.predict(m, lm)
    Vt, dVt = psc.predict(mt, lm)
    assert cases.rel_l2(Vt, V) < 1e-6
    assert max(cases.rel_l2(dVt[p], dV[p]) for p in range(4)) < 1e-6


def test_blocked_disk_samples_normalise_and_reduce_to_the_disk():
    T = aperture.annulus_table_samples(4001, EPS)
    x = np.linspace(0.0, 1.0, T.size)
    pb0 = 2.0 * math.pi * integrate.simpson(T * x, x=x)
    assert abs(pb0 - 1.0) < 1e-5
    assert np.allclose(aperture.annulus_table_samples(513, 0.0), aperture.disk_table_samples(513), atol=1e-14)
    # the Hankel transform of the tabulated A° is the blocked disk's power beam
    # (on the dish scale, D_lambda = 1: PB(rho) = int A°(q) J0(2 pi q rho) 2 pi q dq)
    for rho in (0.3, 0.7, 1.3):
        f = lambda q: np.interp(q, x, T) * 2.0 * math.pi * q * special.j0(2.0 * math.pi * q * rho)
        pb, _ = integrate.quad(f, 0.0, 1.0, limit=400)
        e = aperture.efp_annulus(np.array([rho]), 1.0, EPS)[0]
        assert abs(pb - e * e) < 2e-5, rho


@pytest.mark.parametrize("sigma", [0.0, 20.0])
def test_blocked_disk_table_matches_the_direct_sum(sigma):
    m, sky, lm, _ = cases.problem(cases.DISK_SMALL, sigma_arcsec=sigma, freqs=(1.2e9, 1.4e9))
    mt = _table_model(m, aperture.annulus_table_samples(4001, EPS))
    V, _ = psc.predict(mt, lm, False)
    Vc = closed_form.visibilities(m.uvw_m, m.freq_hz, m.n_ant, sky, lm, "annulus", 25.0, m.alpha_per_dlambda,
                                  blockage=EPS)
    assert cases.rel_l2(V, Vc) < 1e-3
    # and the unblocked model misses it by more
    V0, _ = psc.predict(m, lm, False)
    assert cases.rel_l2(V0, Vc) > 3e-3
