"""Two parallel-hand polarisations solved separately (beam squint).

The R and L data of the 27-antenna single-channel workload are simulated by
the FP64 oracle at the mechanical offset plus and minus half a squint vector
(60 arcsec) with independent noise; the GPU solves both polarisations as one
batch.  Each polarisation's offsets must match the oracle's solution of the
same data within 0.1 arcsec, and the half-sum and difference must recover the
mechanical offsets and the squint."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I, squint
from paper_1709_08681_gb300.session import Session
from oracle import lm as LM, model_grid, psc


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_two_polarisations_match_the_oracle_and_give_the_squint():
    wl = I.make_workload("vla27_l1ch", seed=2)
    mech, sq, lm_r, lm_l = I.squinted_offsets(wl.n_ant, 20.0 * I.ARCSEC, 60.0 * I.ARCSEC, 2)
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    m = psc.Model(uvw_m=wl.uvw_m, freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=grid, cell_rad=wl.cell_rad,
                  support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind, diam_m=wl.diam_m,
                  alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)
    w_scale = 1.0 / wl.sigma_noise ** 2
    data, ref = [], []
    for pol, lm in enumerate((lm_r, lm_l)):
        V, _ = psc.predict(m, lm, False)
        vobs = (V + wl.noise(20 + pol)).astype(np.complex64)
        data.append(vobs)

        def ev(p, vobs=vobs):
            c, g_, H_, X_ = psc.chi2_grad_normal(m, p, vobs, None)
            G, A = psc.assemble_full(m.n_ant, g_ * w_scale, H_ * w_scale, X_ * w_scale)
            return c * w_scale, G, A
        ref.append(LM.solve_full(ev, np.zeros_like(lm))[0])
    s_r = Session(wl)
    s_l = Session(wl, grid=s_r.grid)
    dv = [torch.from_numpy(d).cuda() for d in data]
    sols, reps = _abi.psc_solve_batch(s_r.ctxs + s_l.ctxs, dv, None, w_scale=[w_scale, w_scale])
    for pol in range(2):
        assert np.max(np.abs(sols[pol] - ref[pol])) < 0.1 * I.ARCSEC, pol
    mech_hat = 0.5 * (sols[0] + sols[1])
    sq_hat = sols[0] - sols[1]
    assert np.sqrt(np.mean((mech_hat - mech) ** 2)) / I.ARCSEC < 1.0
    assert np.sqrt(np.mean((sq_hat - sq) ** 2)) / I.ARCSEC < 2.0
    s_r.close()
    s_l.close()


def test_squint_driver_recovers_squint_on_the_64_channel_workload():
    rep, _, _ = squint.run("vla27_l64ch", seed=1)
    assert rep["squint_rms_err_arcsec"] < 0.1 and rep["mechanical_rms_err_arcsec"] < 0.1
