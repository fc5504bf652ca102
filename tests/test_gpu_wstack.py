"""GPU parity of the residual-w stack (psc_wstack_range, psc_wstack_components,
psc_model_grid_wstack, psc_set_wstack) with the oracle's ``wstack``, through
the C ABI.

The problem is a 6-antenna Y array tracked for 6 hours: after the plane fit
the residual w spans about 2000 wavelengths, and the W-snapshot model alone
is 5e-3 off the direct sum with the w-term.  Tolerances as in the co-planar
parity tests: V and dV within 1e-5 relative L2 of the oracle (FP32 against
FP64; the interpolation weight is rounded to FP32, an extra 6e-8 relative),
plane grids within 1e-6 (as psc_model_grid_components), the residual-w range
to 1e-12.
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import closed_form, lm as LM, model_grid, psc, wsnap, wstack

import cases

TOL_V = 1e-5
DW = 200.0
F_C = 1.4e9


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _problem(span_h=6.0, n_time=24, freqs=(1.3e9, 1.4e9, 1.5e9), n_ant=6, seed=1):
    _, N, cell_as, Ng = cases.DISK_SMALL
    enu = I.y_layout(n_ant, 300.0, seed)
    ha = np.linspace(-span_h / 2, span_h / 2, n_time) * 15 * I.DEG
    uvw = I.uvw_tracks(enu, 34 * I.DEG, 30 * I.DEG, ha)
    cell = cell_as * I.ARCSEC
    sky = I.sky_points(10, 12.0 * I.ARCMIN, N, cell, ("loguniform", 0.1, 1.0), seed)
    lmt = I.true_offsets(n_ant, 20.0 * I.ARCSEC, seed)
    return uvw, np.asarray(freqs), cell, Ng, sky, lmt


def _oracle_stack(uvw, freq, cell, Ng, sky, dw=DW):
    """Plane, stack extent (from the oracle's own residual w) and oracle model."""
    a, b = wsnap.plane_fit(uvw)
    wr = wstack.residual_w(uvw, freq, a, b)
    w0 = math.floor(wr.min() / dw) * dw
    P = max(2, int(math.ceil((wr.max() - w0) / dw)) + 1)
    s4 = wstack.stack_sources(sky, a, b, "disk", F_C, 25.0, I.ALPHA_PER_DLAMBDA_DISK)
    du = 1.0 / (Ng * cell)
    m = psc.Model(uvw_m=uvw, freq_hz=freq, n_ant=_n_ant(uvw), grid=model_grid.grid_from_components(s4[:, :3], Ng, du),
                  cell_rad=cell, support=32, oversample=20, ap_kind="disk", diam_m=25.0,
                  alpha_per_dlambda=I.ALPHA_PER_DLAMBDA_DISK, decorrelation=1)
    return (a, b, w0, P), m, wstack.plane_grids(s4, Ng, du, w0, dw, P)


def _n_ant(uvw):
    n_bl = uvw.shape[1]
    return int(round((1 + math.sqrt(1 + 8 * n_bl)) / 2))


class GpuStack:
    """plane -> stack components -> planes and snapshot grid -> context, all through the ABI."""

    def __init__(self, uvw, freq, cell, Ng, sky, w0, P, dw=DW):
        self.uvw = torch.from_numpy(np.ascontiguousarray(uvw)).cuda()
        rows = uvw.shape[0] * uvw.shape[1]
        self.a, self.b = _abi.psc_snapshot_plane(self.uvw, rows)
        self.range_m = _abi.psc_wstack_range(self.uvw, rows, self.a, self.b)
        comp = _abi.psc_wstack_components(sky, self.a, self.b, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, F_C)
        self.planes = torch.empty((P, Ng, Ng), dtype=torch.complex64, device="cuda")
        _abi.psc_model_grid_wstack(comp, Ng, cell, P, w0, dw, self.planes)
        self.grid = torch.empty((Ng, Ng), dtype=torch.complex64, device="cuda")
        _abi.psc_model_grid_components(comp[:, :3], Ng, cell, self.grid)
        self.n_ant = _n_ant(uvw)
        self.shape = (uvw.shape[0], uvw.shape[1], len(freq))
        self.ctx = _abi.Context(self.n_ant, uvw.shape[0], len(freq), self.uvw, freq, "disk", 25.0,
                                I.ALPHA_PER_DLAMBDA_DISK, 1, 64, Ng, cell, 32, 20, self.grid)
        self.ctx.psc_set_wstack(self.planes, P, w0, dw, self.a, self.b)

    def predict(self, lm):
        return _predict(self.ctx, self.shape, lm)

    def close(self):
        self.ctx.close()


def _predict(ctx, shape, lm):
    v = torch.empty(shape, dtype=torch.complex64, device="cuda")
    d = torch.empty((4,) + shape, dtype=torch.complex64, device="cuda")
    ctx.psc_predict(lm, v, d)
    return v.cpu().numpy(), d.cpu().numpy()


def test_range_and_plane_grids_match_oracle():
    uvw, freq, cell, Ng, sky, lmt = _problem()
    (a, b, w0, P), m, planes = _oracle_stack(uvw, freq, cell, Ng, sky)
    gs = GpuStack(uvw, freq, cell, Ng, sky, w0, P)
    x = uvw.reshape(-1, 3)
    wr = x[:, 2] - a * x[:, 0] - b * x[:, 1]
    scale = np.max(np.abs(x))
    assert abs(gs.range_m[0] - wr.min()) < 1e-12 * scale and abs(gs.range_m[1] - wr.max()) < 1e-12 * scale
    assert P >= 8
    got = gs.planes.cpu().numpy()
    for p in range(P):
        assert cases.rel_l2(got[p], planes[p]) < 1e-6, p
    gs.close()


# (span h, n_time, tiling): rectangular bricks, flat bricks, two visibilities per thread
TILINGS = [
    (6.0, 24, ("rect", 8, 2, 1)),
    (6.0, 24, ("flat", 64, 1)),
    (6.0, 37, ("rect", 16, 3, 1)),
    (2.0, 60, ("rect", 8, 1, 2)),
    (2.0, 60, ("flat", 96, 2)),
]


@pytest.mark.parametrize("case", TILINGS)
def test_stack_predict_matches_oracle(case):
    span, nt, tiling = case
    uvw, freq, cell, Ng, sky, lmt = _problem(span_h=span, n_time=nt)
    (a, b, w0, P), m, planes = _oracle_stack(uvw, freq, cell, Ng, sky)
    V, dV = wstack.predict(m, planes, w0, DW, a, b, lmt)
    gs = GpuStack(uvw, freq, cell, Ng, sky, w0, P)
    if tiling[0] == "rect":
        gs.ctx.psc_set_tiling(*tiling[1:])
    else:
        gs.ctx.psc_set_flat_tiling(*tiling[1:])
    Vg, dVg = gs.predict(lmt)
    assert cases.rel_l2(Vg, V) < TOL_V
    for p in range(4):
        assert cases.rel_l2(dVg[p], dV[p]) < TOL_V, p
    gs.close()


def test_stack_is_the_w_term_and_n_planes_0_restores_the_grid():
    """The stacked GPU model is within the gridding floor of the direct sum
    with the w-term; psc_set_wstack(0) returns bit for bit to the snapshot
    grid, which is 5e-3 off."""
    uvw, freq, cell, Ng, sky, lmt = _problem()
    (a, b, w0, P), m, planes = _oracle_stack(uvw, freq, cell, Ng, sky)
    gs = GpuStack(uvw, freq, cell, Ng, sky, w0, P)
    n_ant = gs.n_ant
    Vw = closed_form.visibilities(uvw, freq, n_ant, sky, lmt, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, w_term=True)
    Vg, _ = gs.predict(lmt)
    assert cases.rel_l2(Vg, Vw) < 1e-4
    gs.ctx.psc_set_wstack(None, 0)
    Vs, _ = gs.predict(lmt)
    ref = _abi.Context(n_ant, uvw.shape[0], len(freq), gs.uvw, freq, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, 1,
                       64, Ng, cell, 32, 20, gs.grid)
    Vr, _ = _predict(ref, gs.shape, lmt)
    assert np.array_equal(Vs, Vr)
    assert cases.rel_l2(Vs, Vw) > 20 * cases.rel_l2(Vg, Vw)
    ref.close()
    gs.close()


def _obs(uvw, freq, sky, lmt, sigma=1e-5, seed=7):
    Vw = closed_form.visibilities(uvw, freq, _n_ant(uvw), sky, lmt, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, w_term=True)
    vobs = (Vw + I.complex_noise(Vw.shape, sigma, seed)).astype(np.complex64)
    return vobs, np.full(vobs.shape, 1.0 / sigma ** 2, dtype=np.float32)


def test_stack_residual_grad_matches_oracle():
    uvw, freq, cell, Ng, sky, lmt = _problem()
    (a, b, w0, P), m, planes = _oracle_stack(uvw, freq, cell, Ng, sky)
    vobs, w = _obs(uvw, freq, sky, lmt)
    lm = 0.5 * lmt
    chi2, g, H, X = wstack.chi2_grad_normal(m, planes, w0, DW, a, b, lm, vobs, w)
    gs = GpuStack(uvw, freq, cell, Ng, sky, w0, P)
    up = lambda x, dt: torch.from_numpy(np.ascontiguousarray(x)).cuda().to(dt)
    chi2g, gg, Hg, Xg = gs.ctx.psc_residual_grad(lm, up(vobs, torch.complex64), up(w, torch.float32), 1.0, cross=True)
    V, dV = wstack.predict(m, planes, w0, DW, a, b, lm)
    chi2_scale = float(np.sum(w * np.abs(vobs - V) ** 2) + 2.0 * np.sum(w * np.abs(vobs - V) * np.abs(V)))
    assert abs(chi2g - chi2) < TOL_V * chi2_scale
    gscale = 2.0 * np.sum(w[None] * np.abs(vobs - V)[None] * np.abs(dV))
    assert np.max(np.abs(gg - g)) < TOL_V * gscale
    assert np.max(np.abs(Hg - H)) < TOL_V * np.max(np.abs(H))
    assert np.max(np.abs(Xg - X)) < TOL_V * np.max(np.abs(H))
    gs.close()


def test_stack_solve_matches_oracle_and_removes_the_residual_w_bias():
    """Data with the full w-term over 6 hours: the stacked solve equals the
    oracle's and recovers the offsets to the noise level; the snapshot-only
    model's solve on the same data is off by arcseconds."""
    uvw, freq, cell, Ng, sky, lmt = _problem(n_time=16)
    (a, b, w0, P), m, planes = _oracle_stack(uvw, freq, cell, Ng, sky)
    vobs, w = _obs(uvw, freq, sky, lmt)
    n_ant = _n_ant(uvw)

    def ev(p):
        c, g, H, X = wstack.chi2_grad_normal(m, planes, w0, DW, a, b, p, vobs, w)
        G, A = psc.assemble_full(n_ant, g, H, X)
        return c, G, A
    sol_o, _ = LM.solve_full(ev, np.zeros_like(lmt))
    gs = GpuStack(uvw, freq, cell, Ng, sky, w0, P)
    vd = torch.from_numpy(vobs).cuda()
    wd = torch.from_numpy(w).cuda()
    sol, rep = gs.ctx.psc_solve_offsets(vd, wd, 1.0)
    assert _abi.STOP_REASONS[rep.reason] in ("step", "chi2")
    assert np.max(np.abs(sol - sol_o)) < 0.1 * I.ARCSEC
    assert np.max(np.abs(sol - lmt)) < 0.5 * I.ARCSEC
    gs.ctx.psc_set_wstack(None, 0)
    sol_s, _ = gs.ctx.psc_solve_offsets(vd, wd, 1.0)
    assert np.max(np.abs(sol_s - lmt)) > 1.0 * I.ARCSEC
    gs.close()


def test_stack_arguments_are_checked():
    uvw, freq, cell, Ng, sky, lmt = _problem(n_time=8)
    (a, b, w0, P), m, planes = _oracle_stack(uvw, freq, cell, Ng, sky)
    gs = GpuStack(uvw, freq, cell, Ng, sky, w0, P)
    ctx = gs.ctx
    for bad in ((gs.planes, P, w0 + DW, DW, a, b),          # misses the lowest residual w
                (gs.planes, P - 1, w0, DW, a, b) if P > 2 else (gs.planes, 2, w0, 0.1, a, b),
                (gs.planes, 1, w0, DW, a, b),
                (gs.planes, P, w0, -DW, a, b),
                (None, P, w0, DW, a, b)):
        with pytest.raises(_abi.PscError):
            ctx.psc_set_wstack(*bad)
    with pytest.raises(_abi.PscError):
        ctx.psc_set_grid_precision(_abi.PSC_GRID_BF16)      # stack set: FP32 only
    with pytest.raises(_abi.PscError):
        ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)
    plain = _abi.Context(gs.n_ant, uvw.shape[0], len(freq), gs.uvw, freq, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, 1,
                         64, Ng, cell, 32, 20, gs.grid)
    vis = [torch.zeros(gs.shape, dtype=torch.complex64, device="cuda")] * 2
    with pytest.raises(_abi.PscError):
        _abi.Batch([ctx, plain], vis, None)                 # stacked and plain contexts mixed
    plain.close()
    ctx.psc_set_wstack(None, 0)
    ctx.psc_set_grid_precision(_abi.PSC_GRID_BF16)
    with pytest.raises(_abi.PscError):
        ctx.psc_set_wstack(gs.planes, P, w0, DW, a, b)      # BF16 copy set
    ctx.psc_set_grid_precision(_abi.PSC_GRID_F32)
    ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)
    with pytest.raises(_abi.PscError):
        ctx.psc_set_wstack(gs.planes, P, w0, DW, a, b)      # exact kernel set
    ctx.psc_set_kernel_model(_abi.PSC_KERNEL_GAUSS)
    ctx.psc_set_wstack(gs.planes, P, w0, DW, a, b)
    with pytest.raises(_abi.PscError):
        _abi.psc_model_grid_wstack(np.zeros((1, 4)), Ng, cell, 1, 0.0, DW, gs.planes)
    gs.close()


def test_stack_on_the_64_channel_workload_sampled():
    """vla27_l64ch solved as one interval of all 600 time steps, with the
    benchmark's stack (dw from the interpolation bound at 1e-6: 33 planes of
    2048^2) and brick shape (flat bricks of 128): 48 visibilities, sampled
    between two pairs of planes, against the oracle, which builds only the four
    planes they read.  The stack's extent comes from the oracle's plane and
    residual w; the GPU fits its own plane and moves its own components."""
    wl = I.make_workload("vla27_l64ch")
    Ng, cell = wl.n_grid, wl.cell_rad
    a, b = wsnap.plane_fit(wl.uvw_m)
    f_c = 0.5 * (float(np.min(wl.freq_hz)) + float(np.max(wl.freq_hz)))
    s4 = wstack.stack_sources(wl.sky, a, b, wl.ap_kind, f_c, wl.diam_m, wl.alpha_per_dlambda)
    wr = wstack.residual_w(wl.uvw_m, wl.freq_hz, a, b)
    dw = math.sqrt(8e-6) / (2.0 * math.pi * float(np.max(np.abs(s4[:, 3]))))
    w0 = math.floor(wr.min() / dw) * dw
    P = int(math.ceil((wr.max() - w0) / dw)) + 1
    assert P >= 20
    # GPU: its own plane and stack components, the oracle's extent
    uvw_d = torch.from_numpy(np.ascontiguousarray(wl.uvw_m)).cuda()
    ga, gb = _abi.psc_snapshot_plane(uvw_d, wl.n_time * wl.n_bl)
    comp = _abi.psc_wstack_components(wl.sky, ga, gb, wl.ap_kind, wl.diam_m, wl.alpha_per_dlambda, f_c)
    planes = torch.empty((P, Ng, Ng), dtype=torch.complex64, device="cuda")
    _abi.psc_model_grid_wstack(comp, Ng, cell, P, w0, dw, planes)
    grid = torch.empty((Ng, Ng), dtype=torch.complex64, device="cuda")
    _abi.psc_model_grid_components(comp[:, :3], Ng, cell, grid)
    ctx = _abi.Context(wl.n_ant, wl.n_time, wl.n_chan, uvw_d, wl.freq_hz, wl.ap_kind, wl.diam_m,
                       wl.alpha_per_dlambda, wl.decorrelation, wl.image.shape[0], Ng, cell, wl.support,
                       wl.oversample, grid)
    ctx.psc_set_flat_tiling(128, 1)
    ctx.psc_set_wstack(planes, P, w0, dw, ga, gb)
    lm = wl.lm_true[0]
    shape = (wl.n_time, wl.n_bl, wl.n_chan)
    vg = torch.empty(shape, dtype=torch.complex64, device="cuda")
    dg = torch.empty((4,) + shape, dtype=torch.complex64, device="cuda")
    ctx.psc_predict(lm, vg, dg)
    # samples: 24 visibilities whose lower plane is pa, 24 whose lower plane is pb
    q = (wr - w0) / dw
    p = np.minimum(np.floor(q).astype(np.int64), P - 2)
    rng = np.random.default_rng(12)
    pa, pb = P // 2, 2
    idx = []
    for pk in (pa, pb):
        cand = np.flatnonzero(p.ravel() == pk)
        assert cand.size >= 24
        idx.append(rng.choice(cand, 24, replace=False))
    idx = np.concatenate(idx)
    ti, bi, ci = np.unravel_index(idx, shape)
    f = (q - p).ravel()[idx]
    du = 1.0 / (Ng * cell)
    V = np.zeros(idx.size, dtype=np.complex128)
    dV = np.zeros((4, idx.size), dtype=np.complex128)
    for k in (pa, pa + 1, pb, pb + 1):
        h = np.where(p.ravel()[idx] == k, 1.0 - f, 0.0) + np.where(p.ravel()[idx] + 1 == k, f, 0.0)
        sel = np.flatnonzero(h)
        flux = s4[:, 2] * np.exp(2j * np.pi * (w0 + k * dw) * s4[:, 3])
        gk = model_grid.grid_from_components(s4[:, :3], Ng, du, flux=flux)
        m = psc.Model(uvw_m=wl.uvw_m, freq_hz=wl.freq_hz, n_ant=wl.n_ant, grid=gk, cell_rad=cell,
                      support=wl.support, oversample=wl.oversample, ap_kind=wl.ap_kind, diam_m=wl.diam_m,
                      alpha_per_dlambda=wl.alpha_per_dlambda, decorrelation=wl.decorrelation)
        Vk, dVk = psc.predict_points(m, lm, ti[sel], bi[sel], ci[sel])
        V[sel] += h[sel] * Vk
        dV[:, sel] += h[sel][None] * dVk
    assert cases.rel_l2(vg.cpu().numpy()[ti, bi, ci], V) < TOL_V
    dgs = dg.cpu().numpy()[:, ti, bi, ci]
    for c in range(4):
        assert cases.rel_l2(dgs[c], dV[c]) < TOL_V, c
    ctx.close()


def test_stacked_batch_equals_single_solves():
    """Three stacked contexts (the 6-hour track, offsets of three seeds) solved
    as one batch -- one persistent launch of the stacked kernel per LM
    iteration -- give the same offsets, bit for bit, as three single solves."""
    uvw, freq, cell, Ng, sky, _ = _problem(n_time=16)
    (a, b, w0, P), m, planes = _oracle_stack(uvw, freq, cell, Ng, sky)
    stacks, vis, truths = [], [], []
    for seed in (3, 4, 5):
        lmt = I.true_offsets(_n_ant(uvw), 20.0 * I.ARCSEC, seed)
        vobs, _ = _obs(uvw, freq, sky, lmt, seed=seed)
        stacks.append(GpuStack(uvw, freq, cell, Ng, sky, w0, P))
        vis.append(torch.from_numpy(vobs).cuda())
        truths.append(lmt)
    single = [gs.ctx.psc_solve_offsets(v, None, 1e10) for gs, v in zip(stacks, vis)]
    sols, reps = _abi.psc_solve_batch([gs.ctx for gs in stacks], vis, None, w_scale=[1e10] * 3)
    for k in range(3):
        assert np.array_equal(sols[k], single[k][0]), k
        assert reps[k].n_iter == single[k][1].n_iter
        assert np.max(np.abs(sols[k] - truths[k])) < 0.5 * I.ARCSEC
    for gs in stacks:
        gs.close()
