"""The track kernel (psc_set_track_tiling: one warp per baseline and chunk of
32 lanes x kv time steps, looping over channels, grid boxes and tables staged
by TMA) against the FP64 oracle.

The small-aperture grid (a 512^2 image at 5" padded to 1024^2: du = 40
wavelengths, so a 25 m disk reaches 2.5-3.5 cells) gives boxes that the
warp stages; longer baselines and the large-aperture grid give boxes beyond
the 32-cell / 512-cell tile, which read the grid from global memory instead.
Cases cover one and several time chunks, ragged last chunks and lanes, one
visibility, both visibilities per lane, batches (persistent launch) and the
full-scale workload's interval in the benchmark's launch configuration.
Tolerances are those of test_gpu_parity: chi^2, H and the cross blocks to
1e-5 relative, the gradient to 1e-5 of the sum of its terms' magnitudes,
offsets within 0.1 arcsec of the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import lm as LM, model_grid, psc

import cases
from gpu_cases import GpuProblem

TOL = 1e-5
SMALL_AP = ("disk", 512, 5.0, 1024)


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _obs(m, lmt, sigma=1e-3, seed=7):
    V, _ = psc.predict(m, lmt, False)
    vobs = (V + I.complex_noise(V.shape, sigma, seed)).astype(np.complex64)
    w = np.full(V.shape, 1.0 / sigma ** 2, dtype=np.float32)
    return vobs, w


def _check_sums(m, lm, vobs, w, got):
    chi2, g, H, X = psc.chi2_grad_normal(m, lm, vobs, w)
    V, dV = psc.predict(m, lm)
    R = vobs - V
    chi_scale = float(np.sum(w * np.abs(R) ** 2) + 2.0 * np.sum(w * np.abs(R) * np.abs(V)))
    assert abs(got[0] - chi2) < TOL * chi_scale
    if chi2 > 0.1 * chi_scale:                    # residuals not small against V: plain relative accuracy too
        assert abs(got[0] - chi2) < TOL * chi2
    gscale = 2.0 * np.sum(w[None] * np.abs(R)[None] * np.abs(dV))
    assert np.max(np.abs(got[1] - g)) < TOL * gscale
    assert np.max(np.abs(got[2] - H)) < TOL * np.max(np.abs(H))
    assert np.max(np.abs(got[3] - X)) < TOL * np.max(np.abs(H))


# (grid spec, n_ant, n_time, freqs, vis_per_lane, array extent in m)
TRACK_CASES = [
    (SMALL_AP, 7, 40, (1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), 1, 300.0),   # chunks of 32 + 8 steps
    (SMALL_AP, 6, 37, (1.3e9, 1.35e9, 1.4e9, 1.45e9), 2, 300.0),        # one chunk, last lane half full
    (SMALL_AP, 5, 130, (1.4e9,), 2, 300.0),                             # chunks of 64 + 64 + 2
    (SMALL_AP, 6, 24, (1.0e9, 1.3e9, 1.6e9, 1.9e9), 1, 1200.0),         # long tracks: boxes past the tile
    (SMALL_AP, 2, 1, (1.4e9,), 1, 300.0),                               # a single visibility
    (cases.DISK_SMALL, 5, 20, (1.3e9, 1.4e9), 1, 300.0),                # 14-cell aperture: global reads
]


@pytest.mark.parametrize("case", TRACK_CASES)
def test_track_kernel_matches_oracle_and_brick_kernel(case):
    spec, n_ant, nt, freqs, kv, extent = case
    m, _, lmt, img = cases.problem(spec, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=30.0, extent_m=extent)
    vobs, w = _obs(m, lmt)
    gp = GpuProblem(m, img)
    dv, dw = gp.upload(vobs), gp.upload(w, torch.float32)
    lm = 0.5 * lmt
    brick = gp.ctx.psc_residual_grad(lm, dv, dw, 1.0, cross=True)
    gp.ctx.psc_set_track_tiling(kv)
    got = gp.ctx.psc_residual_grad(lm, dv, dw, 1.0, cross=True)
    _check_sums(m, lm, vobs, w, got)
    # the brick kernel computes the same sums in another order, to the same bar
    _check_sums(m, lm, vobs, w, brick)
    assert np.max(np.abs(got[2] - brick[2])) < TOL * np.max(np.abs(brick[2]))
    # predictions keep the brick kernel; switching back restores it bit for bit
    gp.ctx.psc_set_track_tiling(0)
    again = gp.ctx.psc_residual_grad(lm, dv, dw, 1.0, cross=True)
    assert again[0] == brick[0] and all(np.array_equal(a, b) for a, b in zip(again[1:], brick[1:]))


def test_track_kernel_with_scalar_weights_and_zero_offsets():
    m, _, lmt, img = cases.problem(SMALL_AP, n_ant=6, n_time=50, freqs=(1.3e9, 1.4e9, 1.5e9), sigma_arcsec=30.0)
    vobs, w = _obs(m, lmt)
    gp = GpuProblem(m, img)
    gp.ctx.psc_set_track_tiling(2)
    got = gp.ctx.psc_residual_grad(np.zeros_like(lmt), gp.upload(vobs), None, 1e6, cross=True)
    _check_sums(m, np.zeros_like(lmt), vobs, w, got)


def _oracle_solve(m, vobs, w):
    def ev(p):
        c, g, H, X = psc.chi2_grad_normal(m, p, vobs, w)
        G, A = psc.assemble_full(m.n_ant, g, H, X)
        return c, G, A
    return LM.solve_full(ev, np.zeros((m.n_ant, 2)))


@pytest.mark.parametrize("kv", [1, 2])
def test_track_solve_matches_oracle(kv):
    m, _, lmt, img = cases.problem(SMALL_AP, n_ant=7, n_time=45, freqs=(1.3e9, 1.4e9, 1.5e9), n_src=8)
    vobs, w = _obs(m, lmt)
    sol_o, rep_o = _oracle_solve(m, vobs, w)
    gp = GpuProblem(m, img)
    gp.ctx.psc_set_track_tiling(kv)
    sol_g, rep_g = gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(w, torch.float32), 1.0)
    assert _abi.STOP_REASONS[rep_g.reason] in ("step", "chi2")
    assert np.max(np.abs(sol_g - sol_o)) < 0.1 * I.ARCSEC
    assert abs(rep_g.chi2 - rep_o.chi2) < 1e-4 * rep_o.chi2


def test_track_batch_equals_single_solves_and_launch_order_is_irrelevant():
    """A batch of track contexts runs one persistent track launch per LM
    iteration (items pulled from a queue); every item writes its own record,
    so solves equal the single-context solves (static item assignment) bit
    for bit, and so does the locality launch order of baselines."""
    ivs = []
    for seed, (nt, freqs) in enumerate([(33, (1.4e9,)), (70, (1.3e9, 1.45e9)), (64, (1.2e9, 1.3e9, 1.4e9))]):
        m, _, lmt, img = cases.problem(SMALL_AP, n_ant=6, n_time=nt, freqs=freqs, n_src=8, seed=seed + 1)
        vobs, w = _obs(m, lmt, seed=seed + 20)
        gp = GpuProblem(m, img)
        gp.ctx.psc_set_track_tiling(2)
        ivs.append((m, gp, gp.upload(vobs), gp.upload(w, torch.float32)))
    single = [gp.ctx.psc_solve_offsets(dv, dw, 1.0) for _, gp, dv, dw in ivs]
    ctxs = [gp.ctx for _, gp, _, _ in ivs]
    sols, reps = _abi.psc_solve_batch(ctxs, [x[2] for x in ivs], [x[3] for x in ivs])
    for k in range(len(ivs)):
        assert np.array_equal(sols[k], single[k][0]), k
        assert reps[k].n_iter == single[k][1].n_iter
    b = _abi.Batch(ctxs, [x[2] for x in ivs], [x[3] for x in ivs])
    assert b.psc_batch_kernel() == "track_kernel<2>"
    b.close()
    m, gp, dv, dw = ivs[2]
    a = gp.ctx.psc_residual_grad(0.3 * single[2][0], dv, dw, 1.0, cross=True)
    gp.ctx.psc_set_brick_order(_abi.PSC_ORDER_UV)
    c = gp.ctx.psc_residual_grad(0.3 * single[2][0], dv, dw, 1.0, cross=True)
    assert a[0] == c[0] and all(np.array_equal(x, y) for x, y in zip(a[1:], c[1:]))


def test_batch_refuses_mixed_kernels_and_autotune_may_pick_the_track_kernel():
    m, _, lmt, img = cases.problem(SMALL_AP, n_ant=6, n_time=64, freqs=(1.3e9, 1.4e9), n_src=8)
    vobs, w = _obs(m, lmt)
    g1, g2 = GpuProblem(m, img), GpuProblem(m, img)
    dv, dw = g1.upload(vobs), g1.upload(w, torch.float32)
    g1.ctx.psc_set_track_tiling(1)
    with pytest.raises(_abi.PscError) as e:
        _abi.Batch([g1.ctx, g2.ctx], [dv, dv], [dw, dw])
    assert e.value.status == _abi.PSC_ERR_ARG
    g1.ctx.psc_set_track_tiling(0)
    b = _abi.Batch([g1.ctx, g2.ctx], [dv, dv], [dw, dw])
    tiles = b.psc_batch_autotune()
    kern = b.psc_batch_kernel()
    assert kern.startswith("track_kernel") == (tiles[0][0] == -1)
    b.psc_batch_begin([np.zeros((m.n_ant, 2))] * 2)
    b.psc_batch_iterate(60)
    sols, reps = b.psc_batch_end()
    b.close()
    so, _ = _oracle_solve(m, vobs, w)
    for s in sols:
        assert np.max(np.abs(s - so)) < 0.1 * I.ARCSEC


def test_track_tiling_refusals():
    mg, _, _, imgg = cases.problem(cases.GAUSS_SMALL, n_ant=4, n_time=6)
    gg = GpuProblem(mg, imgg)
    with pytest.raises(_abi.PscError) as e:                       # Gaussian table past the S x S window
        gg.ctx.psc_set_track_tiling(1)
    assert e.value.status == _abi.PSC_ERR_ARG
    m, _, _, img = cases.problem(SMALL_AP, n_ant=4, n_time=6)
    gp = GpuProblem(m, img)
    for bad in (3, -1):
        with pytest.raises(_abi.PscError):
            gp.ctx.psc_set_track_tiling(bad)
    gp.ctx.psc_set_grid_precision(_abi.PSC_GRID_BF16)
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_track_tiling(1)
    gp.ctx.psc_set_grid_precision(_abi.PSC_GRID_F32)
    gp.ctx.psc_set_track_tiling(1)
    gp.ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)        # switches the track tiling off
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_track_tiling(1)


def test_full_scale_interval_in_the_benchmark_configuration():
    """Interval 0 of the full-scale workload (197 antennas, 128 channels,
    60 x 1 s: 148,262,400 visibilities, 8192^2 grid) with the track tiling of
    two visibilities per lane.  The per-baseline cross blocks do not depend on
    the data, so sampled baselines are checked against the oracle visibility by
    visibility; chi^2, the gradient and the antenna blocks against the brick
    kernel on the same data (both FP32; the brick kernel is itself checked
    against the oracle above)."""
    from paper_1709_08681_gb300.session import Session
    wl = I.make_workload("drift197_l128ch", seed=0, n_time=60, n_interval=1)
    s = Session(wl)
    vis = s.simulate()
    ctx = s.ctxs[0]
    lm = 0.5 * wl.lm_true[0]
    w_scale = 1.0 / wl.sigma_noise ** 2
    brick = ctx.psc_residual_grad(lm, vis, None, w_scale, cross=True)
    ctx.psc_set_track_tiling(2)
    got = ctx.psc_residual_grad(lm, vis, None, w_scale, cross=True)
    assert abs(got[0] - brick[0]) < TOL * brick[0]
    assert np.max(np.abs(got[2] - brick[2])) < TOL * np.max(np.abs(brick[2]))
    # |g_p| <= 2 sqrt(chi^2 H_pp) (Cauchy-Schwarz on the sum of its terms): the gradient's scale
    gscale = 2.0 * np.sqrt(brick[0] * np.maximum(brick[2][:, [0]], brick[2][:, [2]]))
    assert np.all(np.abs(got[1] - brick[1]) < TOL * gscale)
    grid = model_grid.grid_from_image(wl.image, wl.n_grid)
    m = psc.Model(uvw_m=wl.uvw_m[:60], freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=grid, cell_rad=wl.cell_rad,
                  support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind, diam_m=wl.diam_m,
                  alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)
    rng = np.random.default_rng(11)
    bls = rng.choice(wl.n_bl, 12, replace=False)
    tt, cc = np.meshgrid(np.arange(60), np.arange(wl.n_chan), indexing="ij")
    for bl in bls:
        _, dV = psc.predict_points(m, lm, tt.ravel(), np.full(tt.size, bl), cc.ravel())
        X = [2 * w_scale * np.sum(np.real(np.conj(dV[p]) * dV[q])) for p, q in ((0, 2), (0, 3), (1, 2), (1, 3))]
        scale = 2 * w_scale * np.sum(np.abs(dV[0]) ** 2 + np.abs(dV[1]) ** 2)
        assert np.max(np.abs(got[3][bl] - np.asarray(X))) < TOL * scale, bl
    s.close()


def test_a_wait_that_runs_out_reports_a_timeout_and_the_context_recovers():
    """Fault path without a fault: with a wait limit of 0 polls every mbarrier
    wait of the track kernel gives up at once.  Each warp then records the
    flag, waits (with its fixed larger bound) for its own TMA copies still in
    flight and stops; the call reports PSC_ERR_TIMEOUT.  With the default
    limit back, the same context gives the earlier results bit for bit."""
    m, _, lmt, img = cases.problem(SMALL_AP, n_ant=6, n_time=40, freqs=(1.3e9, 1.4e9), sigma_arcsec=30.0)
    vobs, w = _obs(m, lmt)
    gp = GpuProblem(m, img)
    gp.ctx.psc_set_track_tiling(2)
    dv, dw = gp.upload(vobs), gp.upload(w, torch.float32)
    ref = gp.ctx.psc_residual_grad(0.5 * lmt, dv, dw, 1.0, cross=True)
    try:
        _abi.psc_set_wait_limit(0)
        assert _abi.psc_get_wait_limit() == 0
        with pytest.raises(_abi.PscError) as e:
            gp.ctx.psc_residual_grad(0.5 * lmt, dv, dw, 1.0, cross=True)
        assert e.value.status == _abi.PSC_ERR_TIMEOUT
        with pytest.raises(_abi.PscError) as e:
            gp.ctx.psc_solve_offsets(dv, dw, 1.0)
        assert e.value.status == _abi.PSC_ERR_TIMEOUT
    finally:
        _abi.psc_set_wait_limit(-1)
    assert _abi.psc_get_wait_limit() == 1 << 24
    again = gp.ctx.psc_residual_grad(0.5 * lmt, dv, dw, 1.0, cross=True)
    assert again[0] == ref[0] and all(np.array_equal(x, y) for x, y in zip(again[1:], ref[1:]))
    sol, rep = gp.ctx.psc_solve_offsets(dv, dw, 1.0)
    assert _abi.STOP_REASONS[rep.reason] in ("step", "chi2")
