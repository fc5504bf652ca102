"""Parity of the exact disk kernel (psc_set_kernel_model(PSC_KERNEL_EXACT_DISK))
with the oracle's exact kernel (``oracle/exact``), through the C ABI.

Tolerances as in the Gaussian-model parity tests: visibilities and their
derivatives within 1e-5 relative L2 (FP32 against FP64; the GPU's Taylor
series of the lens integral is truncated below 1e-7 at these offsets), chi^2,
gradient and normal blocks to the same level, solved offsets within
0.1 arcsec of the oracle's solution.  The offsets go up to 120 arcsec, where
the Gaussian model of Eq. AIJPOINTING biases the solution by arcseconds.
"""
import dataclasses

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from paper_1709_08681_gb300.session import Session
from oracle import lm as LM, model_grid, psc

import cases
from gpu_cases import GpuProblem

TOL_V = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _exact(m):
    return dataclasses.replace(m, kernel="exact")


def _gpu(m, img, **kw):
    gp = GpuProblem(m, img, **kw)
    gp.ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)
    return gp


# (n_ant, n_time, freqs, t_tile, c_group, sigma arcsec): several tiles, ragged
# tails, idle lanes, a single visibility
EXACT_CASES = [
    (7, 40, (1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), 32, 4, 60.0),
    (6, 31, (1.2e9, 1.3e9, 1.4e9), 25, 3, 120.0),
    (5, 9, (1.4e9,), 8, 4, 120.0),
    (2, 1, (1.4e9,), 32, 4, 20.0),
]


@pytest.mark.parametrize("case", EXACT_CASES)
@pytest.mark.parametrize("staging", [_abi.PSC_STAGE_AUTO, _abi.PSC_STAGE_NEVER])
def test_exact_predict_matches_oracle(case, staging):
    n_ant, nt, freqs, tt, cg, sigma = case
    m, _, lm, img = cases.problem(cases.DISK_SMALL, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=sigma)
    V, dV = psc.predict(_exact(m), lm)
    gp = _gpu(m, img, t_tile=tt, c_group=cg)
    gp.ctx.psc_set_staging(staging)
    Vg, dVg = gp.predict(lm)
    assert cases.rel_l2(Vg, V) < TOL_V
    for p in range(4):
        assert cases.rel_l2(dVg[p], dV[p]) < TOL_V, p


@pytest.mark.parametrize("case", [(6, 37, (1.2e9, 1.3e9, 1.4e9, 1.5e9), 64, 120.0),
                                  (5, 150, (1.3e9, 1.4e9, 1.5e9), 256, 60.0),
                                  (7, 40, (1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), 128, 60.0)])
def test_exact_flat_bricks_match_oracle(case):
    """Flat bricks (blocks straddling channels) with the exact kernel."""
    n_ant, nt, freqs, items, sigma = case
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=sigma)
    me = _exact(m)
    V, dV = psc.predict(me, lmt)
    gp = _gpu(m, img)
    gp.ctx.psc_set_flat_tiling(items, 1)
    Vg, dVg = gp.predict(lmt)
    assert cases.rel_l2(Vg, V) < TOL_V
    for p in range(4):
        assert cases.rel_l2(dVg[p], dV[p]) < TOL_V, p
    vobs, w = _obs(m, lmt)
    lm = 0.5 * lmt
    chi2, g, H, X = psc.chi2_grad_normal(me, lm, vobs, w)
    chi2g, gg, Hg, Xg = gp.ctx.psc_residual_grad(lm, gp.upload(vobs), gp.upload(w, torch.float32), 1.0, cross=True)
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_flat_tiling(items, 2)                  # one visibility per thread


def test_exact_equals_gauss_kernel_without_offsets():
    """At l_i = l_j the exact kernel is A° times the ramp (decorrelation 1)."""
    m, _, lm, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=12, freqs=(1.3e9, 1.5e9), sigma_arcsec=0.0)
    lm = np.tile(np.array([[30.0, -20.0]]) * I.ARCSEC, (m.n_ant, 1))     # common offset: dl = 0
    gp = GpuProblem(m, img)
    Vg, dVg = gp.predict(lm)
    gp.ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)
    Ve, dVe = gp.predict(lm)
    assert cases.rel_l2(Ve, Vg) < 1e-6
    assert cases.rel_l2(dVe, dVg) < 1e-6


def _obs(m, lmt, sigma=1e-4, seed=7):
    V, _ = psc.predict(_exact(m), lmt, False)
    vobs = (V + I.complex_noise(V.shape, sigma, seed)).astype(np.complex64)
    w = np.full(V.shape, 1.0 / sigma ** 2, dtype=np.float32)
    return vobs, w


@pytest.mark.parametrize("case", EXACT_CASES[:3])
def test_exact_residual_grad_matches_oracle(case):
    n_ant, nt, freqs, tt, cg, sigma = case
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=sigma)
    me = _exact(m)
    vobs, w = _obs(m, lmt)
    lm = 0.5 * lmt
    chi2, g, H, X = psc.chi2_grad_normal(me, lm, vobs, w)
    gp = _gpu(m, img, t_tile=tt, c_group=cg)
    chi2g, gg, Hg, Xg = gp.ctx.psc_residual_grad(lm, gp.upload(vobs), gp.upload(w, torch.float32), 1.0, cross=True)
    V, dV = psc.predict(me, lm)
    chi2_scale = float(np.sum(w * np.abs(vobs - V) ** 2) + 2.0 * np.sum(w * np.abs(vobs - V) * np.abs(V)))
    assert abs(chi2g - chi2) < TOL_V * chi2_scale
    gscale = 2.0 * np.sum(w[None] * np.abs(vobs - V)[None] * np.abs(dV))
    assert np.max(np.abs(gg - g)) < TOL_V * gscale
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))
    assert np.max(np.abs(Xg - X)) < TOL_V * np.max(np.abs(H))


def test_exact_solve_matches_oracle_and_removes_the_gaussian_bias():
    """Data from the exact kernel at 120" offsets: the exact-model solve equals
    the oracle's and recovers the offsets to the noise level; the Gaussian
    model's solve on the same data is off by arcseconds."""
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=10, n_src=8, sigma_arcsec=120.0,
                                   freqs=(1.2e9, 1.4e9))
    me = _exact(m)
    vobs, w = _obs(m, lmt)

    def ev(p):
        c, g, H, X = psc.chi2_grad_normal(me, p, vobs, w)
        G, A = psc.assemble_full(me.n_ant, g, H, X)
        return c, G, A
    sol_o, rep_o = LM.solve_full(ev, np.zeros_like(lmt))
    gp = _gpu(m, img)
    sol_e, rep_e = gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(w, torch.float32), 1.0)
    assert _abi.STOP_REASONS[rep_e.reason] in ("step", "chi2")
    assert np.max(np.abs(sol_e - sol_o)) < 0.1 * I.ARCSEC
    assert np.max(np.abs(sol_e - lmt)) < 0.5 * I.ARCSEC
    gp.ctx.psc_set_kernel_model(_abi.PSC_KERNEL_GAUSS)
    sol_g, _ = gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(w, torch.float32), 1.0)
    assert np.max(np.abs(sol_g - lmt)) > 1.0 * I.ARCSEC


def test_exact_on_the_64_channel_workload_sampled():
    """27 antennas, 64 channels 1-2 GHz, 2048^2 grid, first interval, true
    offsets (sigma 20"): 400 sampled visibilities against the oracle."""
    wl = I.make_workload("vla27_l64ch")
    s = Session(wl)
    ctx = s.ctxs[0]
    ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)
    t0, nt = wl.intervals[0]
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    m = psc.Model(uvw_m=wl.uvw_m[t0:t0 + nt], freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=grid, cell_rad=wl.cell_rad,
                  support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind, diam_m=wl.diam_m,
                  alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation, kernel="exact")
    rng = np.random.default_rng(11)
    n = 400
    ti, bi, ci = rng.integers(0, nt, n), rng.integers(0, wl.n_bl, n), rng.integers(0, wl.n_chan, n)
    Vo, dVo = psc.predict_points(m, wl.lm_true[0], ti, bi, ci)
    vg = torch.empty((nt, wl.n_bl, wl.n_chan), dtype=torch.complex64, device="cuda")
    dg = torch.empty((4, nt, wl.n_bl, wl.n_chan), dtype=torch.complex64, device="cuda")
    ctx.psc_predict(wl.lm_true[0], vg, dg)
    assert cases.rel_l2(vg.cpu().numpy()[ti, bi, ci], Vo) < TOL_V
    dVg = dg.cpu().numpy()[:, ti, bi, ci]
    for p in range(4):
        assert cases.rel_l2(dVg[p], dVo[p]) < TOL_V, p
    s.close()


def test_exact_mode_arguments():
    m, _, lm, img = cases.problem(cases.DISK_SMALL, n_ant=4, n_time=4)
    gp = _gpu(m, img)
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_tiling(16, 2, 2)                 # one visibility per thread only
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_kernel_model(7)
    vis = [gp.upload(np.zeros(gp.shape, np.complex64))]
    with pytest.raises(_abi.PscError):
        _abi.Batch([gp.ctx], vis, None)                 # batches take the Gaussian model only
    mg, _, _, img_g = cases.problem(cases.GAUSS_SMALL, n_ant=4, n_time=4)
    gg = GpuProblem(mg, img_g)
    with pytest.raises(_abi.PscError):
        gg.ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)   # uniform disks only
