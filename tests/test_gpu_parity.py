"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Tolerances: visibilities and their derivatives within a relative L2 error of
1e-5 (FP32 complex against FP64), and every single visibility within 2e-5 of
the array's largest magnitude (so that a few wrong visibilities cannot hide
under the norm); chi^2 and the normal blocks to the same relative level; the
gradient, which is a sum of terms of both signs, to 1e-5 of the sum of the
magnitudes of its terms; solved offsets within 0.1 arcsec of the oracle's
solution.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import lm as LM, psc

import cases
from gpu_cases import GpuProblem

TOL_V = 1e-5
TOL_PT = 2e-5      # per visibility, relative to the largest |V| of the array


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return cases.rel_l2(a, b)


def _assert_vis(got, ref):
    """Relative L2 within TOL_V and every element within TOL_PT of max |ref|."""
    assert _rel(got, ref) < TOL_V
    assert np.max(np.abs(np.asarray(got) - ref)) <= TOL_PT * np.max(np.abs(ref))


@pytest.mark.parametrize("spec", [cases.GAUSS_SMALL, cases.DISK_SMALL])
def test_model_grid_matches_oracle(spec):
    m, _, _, img = cases.problem(spec)
    gp = GpuProblem(m, img)
    G = gp.grid.cpu().numpy()
    assert _rel(G, m.grid) < 1e-6


@pytest.mark.parametrize("N,Ng", [(72, 200), (256, 520), (62, 130)])
def test_model_grid_dense_random_image(N, Ng):
    """A dense image with both signs, ragged against the GEMM tiles: N % 8 == 0
    takes the split-bfloat16 tensor-core path (128 x 128 tiles, 32-deep K
    chunks), N = 62 the FP32 SIMT path."""
    from oracle import model_grid
    rng = np.random.default_rng(5)
    img = rng.normal(size=(N, N)).astype(np.float32)
    ref = model_grid.grid_from_image(img.astype(np.float64), Ng)
    out = torch.empty((Ng, Ng), dtype=torch.complex64, device="cuda:0")
    _abi.psc_model_grid(N, Ng, 1e-4, 32, 20, torch.from_numpy(img).cuda(), out)
    assert _rel(out.cpu().numpy(), ref) < 1e-6


# (spec, n_ant, n_time, freqs, t_tile, c_group): several tiles and ragged tails
PREDICT_CASES = [
    (cases.DISK_SMALL, 7, 40, (1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), 32, 4),
    (cases.DISK_SMALL, 6, 31, (1.2e9, 1.3e9, 1.4e9), 25, 3),                # 75 threads: idle lanes
    (cases.DISK_SMALL, 5, 9, (1.4e9,), 8, 4),
    (cases.GAUSS_SMALL, 6, 20, (1.3e9, 1.4e9, 1.45e9), 16, 2),
    (cases.DISK_SMALL, 2, 1, (1.4e9,), 32, 4),
]


@pytest.mark.parametrize("case", PREDICT_CASES)
def test_predict_matches_oracle(case):
    spec, n_ant, nt, freqs, tt, cg = case
    m, _, lm, img = cases.problem(spec, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=30.0)
    V, dV = psc.predict(m, lm)
    gp = GpuProblem(m, img, t_tile=tt, c_group=cg)
    Vg, dVg = gp.predict(lm)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])


# Two visibilities per thread (consecutive times share the staged cells):
# (n_ant, n_time, freqs, t_tile, c_group) with ragged time tails (odd n_time,
# a last thread holding one visibility) and channel groups.  Frequencies stay
# below 1.45 GHz so that the disk aperture fits inside the 32 x 32 window.
KV2_CASES = [
    (7, 37, (1.3e9, 1.35e9, 1.4e9), 8, 4),
    (5, 64, (1.4e9,), 32, 1),
    (6, 13, (1.25e9, 1.3e9, 1.35e9, 1.4e9, 1.42e9), 16, 2),
    (2, 1, (1.4e9,), 32, 4),
    (6, 23, (1.3e9, 1.33e9, 1.36e9, 1.39e9, 1.41e9, 1.43e9), 5, 5),     # warps straddle channels
]


@pytest.mark.parametrize("case", KV2_CASES)
def test_two_visibilities_per_thread_match_oracle(case):
    n_ant, nt, freqs, tt, cg = case
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=30.0)
    V, dV = psc.predict(m, lmt)
    gp = GpuProblem(m, img, t_tile=tt, c_group=cg, kv=2)
    Vg, dVg = gp.predict(lmt)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])
    vobs, w = _obs(m, lmt)
    lm = 0.5 * lmt
    chi2, g, H, X = psc.chi2_grad_normal(m, lm, vobs, w)
    chi2g, gg, Hg, Xg = gp.ctx.psc_residual_grad(lm, gp.upload(vobs), gp.upload(w, torch.float32), 1.0, cross=True)
    assert abs(chi2g - chi2) < TOL_V * _chi2_scale(m, lm, vobs, w)
    Vl, dVl = psc.predict(m, lm)
    gscale = 2.0 * np.sum(w[None] * np.abs(vobs - Vl)[None] * np.abs(dVl))
    assert np.max(np.abs(gg - g)) < TOL_V * gscale
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))
    assert np.max(np.abs(Xg - X)) < TOL_V * np.max(np.abs(H))


def test_two_visibilities_per_thread_refused_when_the_aperture_leaves_the_window():
    """The Gaussian table reaches S/sqrt(2) cells, beyond the window's half-width."""
    m, _, _, img = cases.problem(cases.GAUSS_SMALL, n_ant=4, n_time=6)
    gp = GpuProblem(m, img)
    with pytest.raises(_abi.PscError) as e:
        gp.ctx.psc_set_tiling(0, 0, 2)
    assert e.value.status == _abi.PSC_ERR_ARG
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_tiling(0, 0, 3)


def test_predict_with_the_oracle_grid():
    """Isolates the degridder: same grid values on both sides (rounded to complex64)."""
    m, _, lm, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=12, freqs=(1.3e9, 1.4e9))
    gp = GpuProblem(m, img, use_oracle_grid=True)
    V, dV = psc.predict(m, lm)
    Vg, dVg = gp.predict(lm)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])


def test_unstaged_fallback_matches_oracle():
    """Channels far apart in one block overflow the staging tile, so the
    block reads the grid from global memory; results must not change."""
    m, _, lm, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=8, freqs=(1.0e9, 1.3e9, 1.6e9, 1.9e9),
                                  sigma_arcsec=30.0, extent_m=600.0)
    V, dV = psc.predict(m, lm)
    gp = GpuProblem(m, img, t_tile=8, c_group=4)
    Vg, dVg = gp.predict(lm)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])


# Flat bricks (psc_set_flat_tiling): (n_ant, n_time, freqs, items, kv) with
# blocks that straddle channel boundaries, a baseline's last block ragged,
# blocks wider than a channel's items, and a single visibility
FLAT_CASES = [
    (6, 37, (1.3e9, 1.35e9, 1.4e9, 1.45e9), 64, 2),      # 19 groups per channel: 4 channels per block
    (7, 40, (1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), 128, 1),
    (5, 150, (1.3e9, 1.4e9, 1.5e9), 256, 2),             # 75 groups per channel: 5 channels per block
    (6, 13, (1.25e9, 1.3e9, 1.35e9, 1.4e9, 1.42e9), 32, 1),
    (2, 1, (1.4e9,), 32, 2),
]


@pytest.mark.parametrize("case", FLAT_CASES)
def test_flat_bricks_match_oracle(case):
    n_ant, nt, freqs, items, kv = case
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=30.0)
    V, dV = psc.predict(m, lmt)
    gp = GpuProblem(m, img)
    gp.ctx.psc_set_flat_tiling(items, kv)
    Vg, dVg = gp.predict(lmt)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])
    vobs, w = _obs(m, lmt)
    lm = 0.5 * lmt
    chi2, g, H, X = psc.chi2_grad_normal(m, lm, vobs, w)
    chi2g, gg, Hg, Xg = gp.ctx.psc_residual_grad(lm, gp.upload(vobs), gp.upload(w, torch.float32), 1.0, cross=True)
    assert abs(chi2g - chi2) < TOL_V * _chi2_scale(m, lm, vobs, w)
    Vh, dVh = psc.predict(m, lm)
    gscale = 2.0 * np.sum(w[None] * np.abs(vobs - Vh)[None] * np.abs(dVh))
    assert np.max(np.abs(gg - g)) < TOL_V * gscale
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))
    assert np.max(np.abs(Xg - X)) < TOL_V * np.max(np.abs(H))


def test_flat_tiling_arguments():
    m, _, _, img = cases.problem(cases.DISK_SMALL, n_ant=4, n_time=3, freqs=(1.3e9, 1.4e9))
    gp = GpuProblem(m, img)
    for items, kv in ((48, 1), (0, 1), (512, 1), (64, 3)):
        with pytest.raises(_abi.PscError):
            gp.ctx.psc_set_flat_tiling(items, kv)
    m9, _, _, img9 = cases.problem(cases.DISK_SMALL, n_ant=4, n_time=3, freqs=tuple(1.3e9 + 1e7 * k for k in range(12)))
    g9 = GpuProblem(m9, img9)
    with pytest.raises(_abi.PscError):
        g9.ctx.psc_set_flat_tiling(256, 1)                 # 3 items per channel: 86 channels per block


@pytest.mark.parametrize("kv", [1, 2])
def test_never_staged_matches_oracle(kv):
    """PSC_STAGE_NEVER: every tap reads the grid from global memory, with the
    cell half of the ramp from the block's tables; includes visibilities whose
    windows reach past the grid edge (cells outside contribute nothing)."""
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=41, freqs=(1.3e9, 1.4e9), sigma_arcsec=30.0,
                                   extent_m=1200.0)
    V, dV = psc.predict(m, lmt)
    gp = GpuProblem(m, img, t_tile=16, c_group=2, kv=kv)
    gp.ctx.psc_set_staging(_abi.PSC_STAGE_NEVER)
    Vg, dVg = gp.predict(lmt)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])
    vobs, w = _obs(m, lmt)
    chi2, g, H, X = psc.chi2_grad_normal(m, 0.5 * lmt, vobs, w)
    chi2g, gg, Hg, Xg = gp.ctx.psc_residual_grad(0.5 * lmt, gp.upload(vobs), gp.upload(w, torch.float32), 1.0,
                                                 cross=True)
    assert abs(chi2g - chi2) < TOL_V * _chi2_scale(m, 0.5 * lmt, vobs, w)
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_staging(2)


def test_zero_offset_invariant_bitwise():
    """At zero offsets the decorrelation factor is one: both settings agree bit for bit."""
    m, _, _, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=12)
    z = np.zeros((m.n_ant, 2))
    a = GpuProblem(m, img).predict(z)
    m0 = psc.Model(**{**m.__dict__, "decorrelation": 0})
    b = GpuProblem(m0, img).predict(z)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def _obs(m, lmt, sigma=1e-3, seed=7):
    V, _ = psc.predict(m, lmt, False)
    vobs = (V + I.complex_noise(V.shape, sigma, seed)).astype(np.complex64)
    w = np.full(V.shape, 1.0 / sigma ** 2, dtype=np.float32)
    return vobs, w


def _chi2_scale(m, lm, vobs, w):
    """Error scale of chi^2 = sum w |R|^2 for visibilities within TOL_V of the
    oracle: chi^2 itself plus its first-order sensitivity sum 2 w |R| |V|
    (when |R| << |V|, as for a single visibility near the fit, the relative
    error of chi^2 exceeds that of V by |V| / |R|)."""
    V, _ = psc.predict(m, lm, False)
    return float(np.sum(w * np.abs(vobs - V) ** 2) + 2.0 * np.sum(w * np.abs(vobs - V) * np.abs(V)))


@pytest.mark.parametrize("case", PREDICT_CASES[:4])
def test_residual_grad_matches_oracle(case):
    spec, n_ant, nt, freqs, tt, cg = case
    m, _, lmt, img = cases.problem(spec, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=30.0)
    vobs, w = _obs(m, lmt)
    lm = 0.5 * lmt
    chi2, g, H, X = psc.chi2_grad_normal(m, lm, vobs, w)
    gp = GpuProblem(m, img, t_tile=tt, c_group=cg)
    chi2g, gg, Hg, Xg = gp.ctx.psc_residual_grad(lm, gp.upload(vobs), gp.upload(w, torch.float32), 1.0, cross=True)
    assert abs(chi2g - chi2) < TOL_V * _chi2_scale(m, lm, vobs, w)
    # at half the true offsets the residuals are not small against V, so chi^2
    # also holds plain relative accuracy
    assert abs(chi2g - chi2) < TOL_V * chi2
    # gradient scale: sum over visibilities of |2 w R dV|
    V, dV = psc.predict(m, lm)
    gscale = 2.0 * np.sum(w[None] * np.abs(vobs - V)[None] * np.abs(dV))
    assert np.max(np.abs(gg - g)) < TOL_V * gscale
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))
    assert np.max(np.abs(Xg - X)) < TOL_V * np.max(np.abs(H))


def test_weight_scale_and_null_weights():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=10)
    vobs, _ = _obs(m, lmt)
    gp = GpuProblem(m, img)
    a = gp.ctx.psc_residual_grad(0 * lmt, gp.upload(vobs), None, 4.0)
    b = gp.ctx.psc_residual_grad(0 * lmt, gp.upload(vobs), gp.upload(np.ones(vobs.shape), torch.float32), 1.0)
    assert abs(a[0] - 4.0 * b[0]) < 1e-6 * a[0]
    assert np.allclose(a[1], 4.0 * b[1], rtol=1e-6, atol=0)


def _oracle_solve(m, vobs, w, mode="full"):
    def ev(p):
        c, g, H, X = psc.chi2_grad_normal(m, p, vobs, w)
        if mode == "block":
            return c, g, H
        G, A = psc.assemble_full(m.n_ant, g, H, X)
        return c, G, A
    if mode == "block":
        return LM.solve_block(ev, np.zeros((m.n_ant, 2)), LM.Options(max_iter=200))
    return LM.solve_full(ev, np.zeros((m.n_ant, 2)))


# the 40-antenna case factors its 80 x 80 system in global memory (block-wide
# Cholesky); the smaller ones in shared memory (one warp)
@pytest.mark.parametrize("spec,n_ant,n_time,freqs", [
    (cases.DISK_SMALL, 7, 12, (1.3e9, 1.4e9)),
    (cases.GAUSS_SMALL, 7, 12, (1.3e9, 1.4e9)),
    (cases.DISK_SMALL, 40, 3, (1.4e9,)),
])
def test_solve_matches_oracle(spec, n_ant, n_time, freqs):
    m, _, lmt, img = cases.problem(spec, n_ant=n_ant, n_time=n_time, freqs=freqs, n_src=8)
    vobs, w = _obs(m, lmt)
    sol_o, rep_o = _oracle_solve(m, vobs, w)
    gp = GpuProblem(m, img)
    sol_g, rep_g = gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(w, torch.float32), 1.0)
    assert _abi.STOP_REASONS[rep_g.reason] in ("step", "chi2")
    assert np.max(np.abs(sol_g - sol_o)) < 0.1 * I.ARCSEC
    assert abs(rep_g.chi2 - rep_o.chi2) < 1e-4 * rep_o.chi2


def test_noiseless_recovery_on_gpu():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=10, n_src=8)
    V, _ = psc.predict(m, lmt, False)
    gp = GpuProblem(m, img)
    sol, rep = gp.ctx.psc_solve_offsets(gp.upload(V.astype(np.complex64)), None, 1e6)
    assert np.max(np.abs(sol - lmt)) < 0.1 * I.ARCSEC


def test_block_mode_matches_oracle():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=10, n_src=8)
    vobs, w = _obs(m, lmt)
    sol_o, rep_o = _oracle_solve(m, vobs, w, "block")
    gp = GpuProblem(m, img)
    o = _abi.psc_solve_opts_default()
    o.mode = _abi.PSC_LM_BLOCK
    o.max_iter = 200
    sol_g, rep_g = gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(w, torch.float32), 1.0, opts=o)
    assert np.max(np.abs(sol_g - sol_o)) < 0.1 * I.ARCSEC


def test_lm_split_calls_equal_solve():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=10, n_src=8)
    vobs, w = _obs(m, lmt)
    gp = GpuProblem(m, img)
    dv, dw = gp.upload(vobs), gp.upload(w, torch.float32)
    sol_a, rep_a = gp.ctx.psc_solve_offsets(dv, dw, 1.0)
    gp.ctx.psc_lm_begin(np.zeros((m.n_ant, 2)))
    gp.ctx.psc_lm_iterate(dv, dw, 1.0, 60)
    sol_b, rep_b = gp.ctx.psc_lm_end()
    assert np.array_equal(sol_a, sol_b)
    assert rep_a.n_iter == rep_b.n_iter and rep_a.reason == rep_b.reason


def test_argument_errors_are_reported():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=4, n_time=4)
    gp = GpuProblem(m, img)
    with pytest.raises(_abi.PscError) as e:
        gp.ctx.psc_set_tiling(257, 1)
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_tiling(64, 8)
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_tiling(32, 9)
    assert e.value.status == _abi.PSC_ERR_ARG
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_residual_grad(lmt, gp.upload(np.zeros(gp.shape, np.complex64)), None, -1.0)


def test_visibilities_on_and_near_grid_nodes():
    """Taps at tiny radius (a visibility within 1e-4..0.5 cells of a grid
    node) exercise the table lookup at t = rho * ov < 0.5."""
    m, _, lm, img = cases.problem(cases.DISK_SMALL, n_ant=4, n_time=8)
    ng, du = m.grid.shape[0], m.du
    f = m.freq_hz[0]
    fr = np.array([0.0, 1e-4, 0.004, 0.02, 0.4999, 0.5, 0.9996, 0.99999])
    uvw = np.array(m.uvw_m)
    for t in range(uvw.shape[0]):
        for b in range(uvw.shape[1]):
            for ax in (0, 1):
                x = uvw[t, b, ax] * f / 299_792_458.0 / du
                xs = np.floor(x) + fr[(t + b + ax) % len(fr)]
                uvw[t, b, ax] = xs * du * 299_792_458.0 / f
    m2 = psc.Model(**{**m.__dict__, "uvw_m": uvw})
    V, dV = psc.predict(m2, lm)
    Vg, dVg = GpuProblem(m2, img).predict(lm)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])


def test_brick_order_keeps_results_bitwise():
    """PSC_ORDER_UV permutes the launch order of baseline groups; every brick's
    partial sums keep their place, so the results are identical."""
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=9, n_time=37, freqs=(1.3e9, 1.4e9, 1.5e9),
                                   sigma_arcsec=30.0, extent_m=800.0)
    vobs, w = _obs(m, lmt)
    gp = GpuProblem(m, img)
    vd, wd = gp.upload(vobs), gp.upload(w, torch.float32)
    for flat in (False, True):
        if flat:
            gp.ctx.psc_set_flat_tiling(128, 2)
        gp.ctx.psc_set_brick_order(_abi.PSC_ORDER_BASELINE)
        a = gp.ctx.psc_residual_grad(0.5 * lmt, vd, wd, 1.0, cross=True)
        gp.ctx.psc_set_brick_order(_abi.PSC_ORDER_UV)
        b = gp.ctx.psc_residual_grad(0.5 * lmt, vd, wd, 1.0, cross=True)
        assert a[0] == b[0]
        for x, y in zip(a[1:], b[1:]):
            assert np.array_equal(x, y)
        sol, rep = gp.ctx.psc_solve_offsets(vd, wd, 1.0)
        gp.ctx.psc_set_brick_order(_abi.PSC_ORDER_BASELINE)
        sol0, rep0 = gp.ctx.psc_solve_offsets(vd, wd, 1.0)
        assert np.array_equal(sol, sol0) and rep.n_iter == rep0.n_iter
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_brick_order(5)


# Support and oversampling at the ends of their ranges: a window narrower than
# the disk (S = 8, taps clipped to it), the widest window (S = 64, boxes past
# the staging tile for the Gaussian pattern), and a coarse table (ov = 4).
SUPPORT_CASES = [
    (cases.DISK_SMALL, 8, 20),
    (cases.DISK_SMALL, 16, 4),
    (cases.DISK_SMALL, 64, 20),
    (cases.GAUSS_SMALL, 64, 8),
]


@pytest.mark.parametrize("spec,support,ov", SUPPORT_CASES)
def test_support_and_oversampling_extremes_match_oracle(spec, support, ov):
    import dataclasses
    m, _, lmt, img = cases.problem(spec, n_ant=6, n_time=17, freqs=(1.3e9, 1.45e9), sigma_arcsec=40.0,
                                   support=support)
    m = dataclasses.replace(m, oversample=ov)
    V, dV = psc.predict(m, lmt)
    gp = GpuProblem(m, img)
    Vg, dVg = gp.predict(lmt)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])
    vobs, w = _obs(m, lmt)
    chi2, g, H, X = psc.chi2_grad_normal(m, 0.5 * lmt, vobs, w)
    chi2g, gg, Hg, Xg = gp.ctx.psc_residual_grad(0.5 * lmt, gp.upload(vobs), gp.upload(w, torch.float32), 1.0,
                                                 cross=True)
    assert abs(chi2g - chi2) < TOL_V * _chi2_scale(m, 0.5 * lmt, vobs, w)
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))


def test_blank_sky_predicts_exact_zeros():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=9)
    gp = GpuProblem(m, np.zeros_like(img))
    Vg, dVg = gp.predict(lmt)
    assert not np.any(Vg) and not np.any(dVg)


@pytest.mark.parametrize("kv", [1, 2])
def test_flat_bricks_never_staged_and_bf16_grid(kv):
    """Flat bricks with every tap read from global memory, and with the BF16
    grid copy (bound: bfloat16's unit roundoff on the grid, 2^-9).  Two
    visibilities per thread need consecutive time steps within 4 cells, which
    the 300 m array keeps and the 1200 m one does not."""
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=29, freqs=(1.3e9, 1.4e9, 1.5e9),
                                   sigma_arcsec=30.0, extent_m=1200.0 if kv == 1 else 300.0)
    V, dV = psc.predict(m, lmt)
    gp = GpuProblem(m, img)
    gp.ctx.psc_set_flat_tiling(64, kv)
    gp.ctx.psc_set_staging(_abi.PSC_STAGE_NEVER)
    Vg, dVg = gp.predict(lmt)
    _assert_vis(Vg, V)
    for p in range(4):
        _assert_vis(dVg[p], dV[p])
    gp.ctx.psc_set_staging(_abi.PSC_STAGE_AUTO)
    gp.ctx.psc_set_grid_precision(_abi.PSC_GRID_BF16)
    Vb, dVb = gp.predict(lmt)
    assert _rel(Vb, V) < 2.0 ** -9
    assert max(_rel(dVb[p], dV[p]) for p in range(4)) < 2.0 ** -9
    gp.ctx.psc_set_grid_precision(_abi.PSC_GRID_F32)


def test_nan_weight_stops_the_solver_with_a_numeric_error():
    """One NaN weight (set on the host) makes chi^2 non-finite at the first
    evaluation: the solver stops and the synchronising call reports
    PSC_ERR_NUMERIC; the context then solves clean data as before."""
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=5, n_time=8)
    vobs, w = _obs(m, lmt)
    gp = GpuProblem(m, img)
    bad = w.copy()
    bad[3, 2, 0] = np.nan
    with pytest.raises(_abi.PscError) as e:
        gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(bad, torch.float32), 1.0)
    assert e.value.status == _abi.PSC_ERR_NUMERIC
    sol, rep = gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(w, torch.float32), 1.0)
    assert np.all(np.isfinite(sol)) and _abi.STOP_REASONS[rep.reason] in ("step", "chi2")


def test_solve_197_antennas_matches_oracle():
    """The 394 x 394 damped system of a 197-antenna interval (the arrays of the
    batched and full-scale workloads) is factored in global memory with FP32
    Cholesky and FP64 refinement; the offsets must match the oracle's full LM
    solve within 0.1 arcsec."""
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=197, n_time=3, freqs=(1.3e9, 1.4e9), n_src=8)
    vobs, w = _obs(m, lmt)
    sol_o, rep_o = _oracle_solve(m, vobs, w)
    gp = GpuProblem(m, img)
    sol_g, rep_g = gp.ctx.psc_solve_offsets(gp.upload(vobs), gp.upload(w, torch.float32), 1.0)
    assert _abi.STOP_REASONS[rep_g.reason] in ("step", "chi2")
    assert np.max(np.abs(sol_g - sol_o)) < 0.1 * I.ARCSEC
    assert abs(rep_g.chi2 - rep_o.chi2) < 1e-4 * rep_o.chi2
