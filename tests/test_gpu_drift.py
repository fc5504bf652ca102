"""Drifting pointing solved interval by interval (reduced size: 27 antennas in
a 1 km disk, 8 channels over 0.95-1.76 GHz, 4 intervals of 60 x 1 s, a 256^2
image at 6" padded to 1024^2).  The prediction is checked against the FP64
oracle on sampled visibilities; warm-started sequential solves must reach
the same minimiser as cold batched solves, in no more iterations, and both
must recover the drifting offsets."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import drift, inputs as I
from paper_1709_08681_gb300.session import Session
from oracle import model_grid, psc

import cases

SMALL = dict(n_ant=27, extent_m=1000.0, n_time=240, n_chan=8, n_interval=4, n_img=256, cell_arcsec=6.0, pad=4,
             n_src=100, src_radius_arcmin=10.0)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_drift_prediction_matches_oracle_on_samples():
    wl = I.make_workload("drift197_l128ch", seed=1, **SMALL)
    s = Session(wl)
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    rng = np.random.default_rng(3)
    for k in (0, 3):
        t0, nt = wl.intervals[k]
        m = psc.Model(uvw_m=wl.uvw_m[t0:t0 + nt], freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=grid,
                      cell_rad=wl.cell_rad, support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind,
                      diam_m=wl.diam_m, alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)
        n = 300
        ti, bi, ci = rng.integers(0, nt, n), rng.integers(0, wl.n_bl, n), rng.integers(0, wl.n_chan, n)
        Vo, dVo = psc.predict_points(m, wl.lm_true[k], ti, bi, ci)
        vg = torch.empty((nt, wl.n_bl, wl.n_chan), dtype=torch.complex64, device="cuda")
        dg = torch.empty((4, nt, wl.n_bl, wl.n_chan), dtype=torch.complex64, device="cuda")
        s.ctxs[k].psc_predict(wl.lm_true[k], vg, dg)
        assert cases.rel_l2(vg.cpu().numpy()[ti, bi, ci], Vo) < 1e-5
        dVg = dg.cpu().numpy()[:, ti, bi, ci]
        for p in range(4):
            assert cases.rel_l2(dVg[p], dVo[p]) < 1e-5
    s.close()


def test_warm_start_reaches_the_cold_minimum_in_fewer_iterations():
    rep = drift.run("drift197_l128ch", seed=1, **SMALL)
    assert rep["warm_vs_cold_max_arcsec"] < 0.01
    assert rep["warm_mean_lm_iters"] <= rep["cold_mean_lm_iters"]
    assert rep["rms_err_arcsec_cold"] < 1.0 and rep["rms_err_arcsec_warm"] < 1.0
    assert rep["gvis_per_s_iteration"] > 0
