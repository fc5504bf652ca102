"""Pins of the oracle's W-snapshot model (``oracle/wsnap``) against the
direct-sum visibilities with the w-term (Eq. ME without the co-planar
approximation, ``closed_form.visibilities(..., w_term=True)``).

* An east-west array's baselines lie in the plane w = -cot(dec) v at every
  hour angle (u = B cos H, v = B sin dec sin H, w = -B cos dec sin H), so the
  fit must return (0, -cot dec) and the snapshot model must reach the
  gridding error of the w-free case.
* A flat array at one instant is co-planar too.
* A Y array over a short interval is nearly co-planar: the snapshot model
  must remove most of the w error that the co-planar model leaves.
"""
import math

import numpy as np
import pytest

from paper_1709_08681_gb300 import inputs as I
from oracle import closed_form, model_grid, psc, wsnap

import cases

DEC = 30.0


def _problem(enu, span_h=1.0, n_time=8, freqs=(1.4e9,), seed=1):
    kind, N, cell_as, Ng = cases.DISK_SMALL
    ha = np.linspace(-span_h / 2, span_h / 2, n_time) * 15 * I.DEG if n_time > 1 else np.zeros(1)
    uvw = I.uvw_tracks(enu, 34 * I.DEG, DEC * I.DEG, ha)
    cell = cell_as * I.ARCSEC
    sky = I.sky_points(10, 12.0 * I.ARCMIN, N, cell, ("loguniform", 0.1, 1.0), seed)
    lm = I.true_offsets(enu.shape[0], 20.0 * I.ARCSEC, seed)
    return uvw, np.asarray(freqs), sky, lm, cell, Ng


def _predict(uvw, freq, n_ant, sky, lm, cell, Ng):
    grid = model_grid.grid_from_components(sky, Ng, 1.0 / (Ng * cell))
    m = psc.Model(uvw_m=uvw, freq_hz=freq, n_ant=n_ant, grid=grid, cell_rad=cell, support=32, oversample=20,
                  ap_kind="disk", diam_m=25.0, alpha_per_dlambda=I.ALPHA_PER_DLAMBDA_DISK, decorrelation=1)
    return psc.predict(m, lm, False)[0]


def _direct(uvw, freq, n_ant, sky, lm, w_term):
    return closed_form.visibilities(uvw, freq, n_ant, sky, lm, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, w_term=w_term)


def _ew(n=6, seed=0):
    rng = np.random.default_rng(seed)
    return np.stack([np.sort(rng.uniform(-300.0, 300.0, n)), np.zeros(n), np.zeros(n)], axis=1)


def test_plane_of_an_east_west_array():
    uvw, *_ = _problem(_ew())
    a, b = wsnap.plane_fit(uvw)
    assert abs(a) < 1e-12
    assert b == pytest.approx(-1.0 / math.tan(DEC * I.DEG), rel=1e-12)


def test_distortion_formula():
    src = np.array([[0.003, -0.002, 1.0], [0.0, 0.0, 2.0]])
    out = wsnap.distort(src, 0.5, -2.0)
    nm1 = math.sqrt(1 - 0.003 ** 2 - 0.002 ** 2) - 1
    assert out[0, 0] == pytest.approx(0.003 + 0.5 * nm1, rel=1e-15)
    assert out[0, 1] == pytest.approx(-0.002 - 2.0 * nm1, rel=1e-15)
    assert np.array_equal(out[1], src[1]) and np.array_equal(out[:, 2], src[:, 2])


def test_snapshot_model_is_exact_for_a_coplanar_array():
    enu = _ew()
    uvw, freq, sky, lm, cell, Ng = _problem(enu)
    a, b = wsnap.plane_fit(uvw)
    Vw = _direct(uvw, freq, enu.shape[0], sky, lm, True)
    floor = cases.rel_l2(_predict(uvw, freq, enu.shape[0], sky, lm, cell, Ng),
                                 _direct(uvw, freq, enu.shape[0], sky, lm, False))
    snap = wsnap.snapshot_sources(sky, a, b, "disk", freq[0], 25.0, I.ALPHA_PER_DLAMBDA_DISK)
    err_snap = cases.rel_l2(_predict(uvw, freq, enu.shape[0], snap, lm, cell, Ng), Vw)
    err_copl = cases.rel_l2(_predict(uvw, freq, enu.shape[0], sky, lm, cell, Ng), Vw)
    err_nopb = cases.rel_l2(_predict(uvw, freq, enu.shape[0], wsnap.distort(sky, a, b), lm, cell, Ng), Vw)
    assert err_snap < 1.2 * floor + 1e-5          # the w-free gridding error, 6e-5
    assert err_copl > 10 * err_snap               # 1.5e-3: what the co-planar model leaves
    assert err_nopb > 5 * err_snap                # 5e-4: the beam belongs at the true position


def test_flat_array_is_coplanar_at_one_instant():
    enu = I.y_layout(6, 300.0, 1)
    uvw, freq, sky, lm, cell, Ng = _problem(enu, n_time=1)
    a, b = wsnap.plane_fit(uvw)
    x = uvw.reshape(-1, 3)
    assert np.max(np.abs(x[:, 2] - a * x[:, 0] - b * x[:, 1])) < 1e-9 * np.max(np.abs(x))
    Vw = _direct(uvw, freq, enu.shape[0], sky, lm, True)
    snap = wsnap.snapshot_sources(sky, a, b, "disk", freq[0], 25.0, I.ALPHA_PER_DLAMBDA_DISK)
    assert cases.rel_l2(_predict(uvw, freq, enu.shape[0], snap, lm, cell, Ng), Vw) < 1e-4


def test_short_interval_removes_most_of_the_w_error():
    enu = I.y_layout(6, 300.0, 1)
    uvw, freq, sky, lm, cell, Ng = _problem(enu, span_h=0.3)
    a, b = wsnap.plane_fit(uvw)
    Vw = _direct(uvw, freq, enu.shape[0], sky, lm, True)
    snap = wsnap.snapshot_sources(sky, a, b, "disk", freq[0], 25.0, I.ALPHA_PER_DLAMBDA_DISK)
    err_snap = cases.rel_l2(_predict(uvw, freq, enu.shape[0], snap, lm, cell, Ng), Vw)
    err_copl = cases.rel_l2(_predict(uvw, freq, enu.shape[0], sky, lm, cell, Ng), Vw)
    assert err_snap < err_copl / 3               # 2e-4 vs 9e-4 over 18 minutes
