"""Parity at the full sizes of the two plain-method workloads.

vla27_l1ch (27 antennas, 1 channel, 60 times, 256^2 image padded to 4096^2)
is small enough for the oracle everywhere: predict, derivatives, the fused
reductions and the solve are compared in full.  vla27_l64ch (13,478,400
visibilities, the benchmark's workload, in the benchmark's launch shape:
autotuned tiles, one persistent batched launch) is compared on sampled
visibilities that the oracle computes one by one, and its fused chi^2 /
gradient / normal sums against FP64 reductions of the GPU's own predicted
visibilities and derivatives (a property that holds at any size)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from paper_1709_08681_gb300.session import Session
from oracle import lm as LM, model_grid, psc

import cases


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_model(wl, grid, t0=0, nt=None):
    nt = wl.n_time if nt is None else nt
    return psc.Model(uvw_m=wl.uvw_m[t0:t0 + nt], freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=grid,
                     cell_rad=wl.cell_rad, support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind,
                     diam_m=wl.diam_m, alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)


def test_vla27_l1ch_full_parity_and_solve():
    wl = I.make_workload("vla27_l1ch")
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    m = oracle_model(wl, grid)
    lmt = wl.lm_true[0]
    s = Session(wl)
    assert cases.rel_l2(s.grid.cpu().numpy(), grid) < 1e-5
    V, dV = psc.predict(m, lmt)
    vg = s.empty_vis()
    dg = torch.empty((4,) + tuple(vg.shape), dtype=torch.complex64, device="cuda")
    s.ctxs[0].psc_predict(lmt, vg, dg)
    assert cases.rel_l2(vg.cpu().numpy(), V) < 1e-5
    for p in range(4):
        assert cases.rel_l2(dg[p].cpu().numpy(), dV[p]) < 1e-5
    vobs = (V + wl.noise()).astype(np.complex64)
    w_scale = 1.0 / wl.sigma_noise ** 2
    chi2, g, H, X = psc.chi2_grad_normal(m, 0.5 * lmt, vobs, None)
    dv = torch.from_numpy(vobs).cuda()
    c2, gg, Hg, Xg = s.ctxs[0].psc_residual_grad(0.5 * lmt, dv, None, 1.0, cross=True)
    assert abs(c2 - chi2) < 1e-5 * chi2
    assert np.max(np.abs(Hg - H)) < 1e-5 * np.max(np.abs(H))

    def ev(p):
        c, g_, H_, X_ = psc.chi2_grad_normal(m, p, vobs, np.full(vobs.shape, w_scale))
        G, A = psc.assemble_full(m.n_ant, g_, H_, X_)
        return c, G, A
    so, _ = LM.solve_full(ev, np.zeros_like(lmt))
    sg, rep = s.ctxs[0].psc_solve_offsets(dv, None, w_scale)
    assert np.max(np.abs(sg - so)) < 0.1 * I.ARCSEC
    assert np.sqrt(np.mean((sg - lmt) ** 2)) < 1.0 * I.ARCSEC


def test_vla27_l64ch_sampled_parity_in_the_bench_launch_shape():
    wl = I.make_workload("vla27_l64ch")
    s = Session(wl)
    vis = s.simulate()
    w = torch.full(vis.shape, 1.0 / wl.sigma_noise ** 2, dtype=torch.float32, device="cuda")
    vk = [s.vis_slice(vis, k) for k in range(4)]
    wk = [s.vis_slice(w, k) for k in range(4)]
    batch = _abi.Batch(s.ctxs, vk, wk)
    batch.psc_batch_autotune()                        # the benchmark's tiles
    lm_eval = [0.5 * wl.lm_true[k] for k in range(4)]
    batch.psc_batch_begin(lm_eval)
    batch.psc_batch_iterate(1)                        # one fused evaluation at lm_eval per interval
    _, reps = batch.psc_batch_end()
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    rng = np.random.default_rng(11)
    for k, (t0, nt) in enumerate(wl.intervals):
        ctx = s.ctxs[k]
        vg = torch.empty_like(vk[k])
        dg = torch.empty((4,) + tuple(vg.shape), dtype=torch.complex64, device="cuda")
        ctx.psc_predict(lm_eval[k], vg, dg)
        # sampled visibilities against the oracle, one by one
        n = 150
        ti, bi, ci = rng.integers(0, nt, n), rng.integers(0, wl.n_bl, n), rng.integers(0, wl.n_chan, n)
        Vo, dVo = psc.predict_points(oracle_model(wl, grid, t0, nt), lm_eval[k], ti, bi, ci)
        V = vg.cpu().numpy()
        dV = dg.cpu().numpy()
        assert cases.rel_l2(V[ti, bi, ci], Vo) < 1e-5
        for p in range(4):
            assert cases.rel_l2(dV[p][ti, bi, ci], dVo[p]) < 1e-5
        # fused chi^2 of the batched launch = FP64 sum over the GPU's predicted V
        vo = vk[k].cpu().numpy().astype(np.complex128)
        ww = wk[k].cpu().numpy().astype(np.float64)
        R = vo - V
        chi2 = float(np.sum(ww * np.abs(R) ** 2))
        assert abs(reps[k].chi2 - chi2) < 1e-5 * chi2
        # fused gradient and normal blocks (single-interval launch, same tiles)
        c2, gg, Hg = ctx.psc_residual_grad(lm_eval[k], vk[k], wk[k], 1.0)
        ij = np.asarray([(i, j) for i in range(wl.n_ant) for j in range(i + 1, wl.n_ant)])
        gp = -2.0 * np.sum(ww[None] * np.real(np.conj(R)[None] * dV), axis=(1, 3))
        g = np.zeros((wl.n_ant, 2))
        for b, (i, j) in enumerate(ij):
            g[i] += gp[0, b], gp[1, b]
            g[j] += gp[2, b], gp[3, b]
        gscale = 2.0 * np.sum(ww[None] * np.abs(R)[None] * np.abs(dV))
        assert np.max(np.abs(gg - g)) < 1e-5 * gscale
        # H_ll of antenna i: d/dl_i of its baselines as first (plane 0) and second (plane 2) antenna
        hli = 2.0 * np.sum(ww * np.abs(dV[0]) ** 2, axis=(0, 2))
        hlj = 2.0 * np.sum(ww * np.abs(dV[2]) ** 2, axis=(0, 2))
        H0 = np.zeros(wl.n_ant)
        for b, (i, j) in enumerate(ij):
            H0[i] += hli[b]
            H0[j] += hlj[b]
        assert np.max(np.abs(Hg[:, 0] - H0)) < 1e-5 * np.max(H0)
    batch.close()
