"""Pins of the oracle's residual-w stack (``oracle/wstack``).

* Against the direct sum with the w-term (Eq. ME without the co-planar
  approximation): over a 6-hour track of a Y array the stack reaches the
  gridding error of the w-free case, where the co-planar model and W-snapshots
  alone leave two orders of magnitude more.
* One source: every grid of the stack is a scalar multiple of the snapshot
  grid, so the stacked visibilities and derivatives are the snapshot-frame
  ones times the interpolated phasor (1 - f) e^{i t w_p} + f e^{i t w_{p+1}},
  t = 2 pi (n - 1), computed here in closed form per visibility.
* The interpolation error falls as dw^2 (linear interpolation of e^{i t w})
  and stays inside its bound (t dw)^2 / 8.
* Visibilities outside the stack are refused.
"""
import math

import numpy as np
import pytest

from paper_1709_08681_gb300 import inputs as I
from oracle import closed_form, model_grid, psc, wsnap, wstack

import cases

DEC = 30.0
F_C = 1.4e9


def _geometry(extent_m=300.0, span_h=6.0, n_time=10, freqs=(1.3e9, 1.4e9, 1.5e9)):
    enu = I.y_layout(6, extent_m, 1)
    ha = np.linspace(-span_h / 2, span_h / 2, n_time) * 15 * I.DEG
    return I.uvw_tracks(enu, 34 * I.DEG, DEC * I.DEG, ha), np.asarray(freqs)


def _model(uvw, freq, grid, cell):
    return psc.Model(uvw_m=uvw, freq_hz=freq, n_ant=6, grid=grid, cell_rad=cell, support=32, oversample=20,
                     ap_kind="disk", diam_m=25.0, alpha_per_dlambda=I.ALPHA_PER_DLAMBDA_DISK, decorrelation=1)


def _stack(uvw, freq, sky, dw):
    a, b = wsnap.plane_fit(uvw)
    wr = wstack.residual_w(uvw, freq, a, b)
    w0 = math.floor(wr.min() / dw) * dw
    n_planes = max(2, int(math.ceil((wr.max() - w0) / dw)) + 1)
    s4 = wstack.stack_sources(sky, a, b, "disk", F_C, 25.0, I.ALPHA_PER_DLAMBDA_DISK)
    return a, b, w0, n_planes, s4


def test_long_interval_reaches_the_gridding_floor():
    _, N, cell_as, Ng = cases.DISK_SMALL
    cell = cell_as * I.ARCSEC
    uvw, freq = _geometry(n_time=12, freqs=(1.4e9,))
    sky = I.sky_points(10, 12.0 * I.ARCMIN, N, cell, ("loguniform", 0.1, 1.0), 1)
    lm = I.true_offsets(6, 20.0 * I.ARCSEC, 1)
    du = 1.0 / (Ng * cell)
    Vw = closed_form.visibilities(uvw, freq, 6, sky, lm, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, w_term=True)
    Vn = closed_form.visibilities(uvw, freq, 6, sky, lm, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, w_term=False)
    g0 = model_grid.grid_from_components(sky, Ng, du)
    floor = cases.rel_l2(psc.predict(_model(uvw, freq, g0, cell), lm, False)[0], Vn)
    a, b, w0, P, s4 = _stack(uvw, freq, sky, 200.0)
    gs = model_grid.grid_from_components(s4[:, :3], Ng, du)
    m = _model(uvw, freq, gs, cell)
    err_snap = cases.rel_l2(psc.predict(m, lm, False)[0], Vw)
    planes = wstack.plane_grids(s4, Ng, du, w0, 200.0, P)
    err_stack = cases.rel_l2(wstack.predict(m, planes, w0, 200.0, a, b, lm, False)[0], Vw)
    err_copl = cases.rel_l2(psc.predict(_model(uvw, freq, g0, cell), lm, False)[0], Vw)
    assert P >= 8                                   # residual w spans ~1800 wavelengths
    assert err_stack < 1.05 * floor                 # 6.2e-5, the w-free gridding error
    assert err_snap > 50 * err_stack                # 4.8e-3
    assert err_copl > 50 * err_stack                # 5.0e-3


def _one_source(offset_arcmin=10.0):
    _, N, cell_as, Ng = cases.DISK_SMALL
    cell = cell_as * I.ARCSEC
    uvw, freq = _geometry()
    k = round(offset_arcmin * I.ARCMIN / cell)
    sky = np.array([[k * cell, -0.5 * k * cell, 0.7]])
    return uvw, freq, sky, cell, Ng


@pytest.mark.parametrize("dw", [150.0, 400.0])
def test_one_source_is_the_snapshot_times_the_interpolated_phasor(dw):
    uvw, freq, sky, cell, Ng = _one_source()
    du = 1.0 / (Ng * cell)
    lm = I.true_offsets(6, 20.0 * I.ARCSEC, 2)
    a, b, w0, P, s4 = _stack(uvw, freq, sky, dw)
    m = _model(uvw, freq, model_grid.grid_from_components(s4[:, :3], Ng, du), cell)
    V0, dV0 = psc.predict(m, lm)
    V, dV = wstack.predict(m, wstack.plane_grids(s4, Ng, du, w0, dw, P), w0, dw, a, b, lm)
    t = 2.0 * math.pi * s4[0, 3]
    q = (wstack.residual_w(uvw, freq, a, b) - w0) / dw
    p = np.minimum(np.floor(q), P - 2)
    f = q - p
    phasor = (1.0 - f) * np.exp(1j * t * (w0 + p * dw)) + f * np.exp(1j * t * (w0 + (p + 1) * dw))
    scale = np.max(np.abs(V0))
    assert np.max(np.abs(V - phasor * V0)) < 1e-12 * scale
    assert np.max(np.abs(dV - phasor[None] * dV0)) < 1e-12 * np.max(np.abs(dV0))
    assert np.max(np.abs(np.angle(phasor))) > 0.02          # 0.034 rad: far above the tolerance


def test_interpolation_error_is_second_order_in_dw():
    uvw, freq, sky, cell, Ng = _one_source(offset_arcmin=12.0)
    du = 1.0 / (Ng * cell)
    lm = np.zeros((6, 2))
    out = {}
    for dw in (400.0, 200.0, 100.0, 12.5):
        a, b, w0, P, s4 = _stack(uvw, freq, sky, dw)
        m = _model(uvw, freq, model_grid.grid_from_components(s4[:, :3], Ng, du), cell)
        out[dw] = wstack.predict(m, wstack.plane_grids(s4, Ng, du, w0, dw, P), w0, dw, a, b, lm, False)[0]
        V0 = psc.predict(m, lm, False)[0]
    t = 2.0 * math.pi * abs(s4[0, 3])
    ref = out[12.5]
    err = {dw: np.max(np.abs(out[dw] - ref) / np.abs(V0)) for dw in (400.0, 200.0, 100.0)}
    for dw in (400.0, 200.0, 100.0):
        assert err[dw] <= (t * dw) ** 2 / 8 * 1.01
    assert 3.3 < err[400.0] / err[200.0] < 4.7
    assert 3.3 < err[200.0] / err[100.0] < 4.7


def test_uncovered_visibilities_are_refused():
    uvw, freq, sky, cell, Ng = _one_source()
    a, b, w0, P, s4 = _stack(uvw, freq, sky, 300.0)
    wr = wstack.residual_w(uvw, freq, a, b)
    with pytest.raises(ValueError):
        wstack.plane_weights(wr, w0 + 300.0, 300.0, P)
    assert P >= 3
    with pytest.raises(ValueError):
        wstack.plane_weights(wr, w0, 150.0, P)           # covers (P - 1) 150 < (P - 2) 300
    with pytest.raises(ValueError):
        wstack.plane_weights(wr, w0, 300.0, 1)
    p, f = wstack.plane_weights(np.array([w0, w0 + (P - 1) * 300.0]), w0, 300.0, P)
    assert list(p) == [0, P - 2] and list(f) == [0.0, 1.0]


def test_derivatives_match_finite_differences():
    uvw, freq, sky, cell, Ng = _one_source()
    uvw = uvw[::3]
    du = 1.0 / (Ng * cell)
    sky = np.concatenate([sky, [[-6 * cell, 9 * cell, 0.4]]])
    lm = I.true_offsets(6, 30.0 * I.ARCSEC, 3)
    a, b, w0, P, s4 = _stack(uvw, freq, sky, 250.0)
    m = _model(uvw, freq, model_grid.grid_from_components(s4[:, :3], Ng, du), cell)
    planes = wstack.plane_grids(s4, Ng, du, w0, 250.0, P)
    _, dV = wstack.predict(m, planes, w0, 250.0, a, b, lm)
    h = 1e-3 * I.ARCSEC
    ij = m.antenna_pairs()
    for ant, axis in ((1, 0), (4, 1)):
        lp, lq = lm.copy(), lm.copy()
        lp[ant, axis] += h
        lq[ant, axis] -= h
        fd = (wstack.predict(m, planes, w0, 250.0, a, b, lp, False)[0]
              - wstack.predict(m, planes, w0, 250.0, a, b, lq, False)[0]) / (2 * h)
        an = np.zeros_like(fd)
        for bl, (i, j) in enumerate(ij):
            if i == ant:
                an[:, bl] = dV[axis, :, bl]
            elif j == ant:
                an[:, bl] = dV[2 + axis, :, bl]
        assert np.max(np.abs(fd - an)) < 1e-6 * np.max(np.abs(an))
