"""GPU parity of the component model grid and the W-snapshot calls, through
the C ABI: psc_model_grid_components against the oracle's direct component
DFT (relative L2 1e-6, as the image grid), psc_snapshot_plane against the
oracle's least-squares plane, and the whole W-snapshot path (plane ->
moved components -> grid -> context) against the oracle's snapshot
prediction (1e-5) and against the direct sum with the w-term."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import closed_form, lm as LM, model_grid, psc, wsnap

import cases

TOL_V = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("n_comp,ng", [(1, 130), (13, 256), (200, 520), (64, 1024)])
def test_component_grid_matches_oracle(n_comp, ng):
    """Components off the pixel centres; grid sizes ragged against the 128 x 64 tiles."""
    rng = np.random.default_rng(n_comp)
    cell = 5.0 * I.ARCSEC
    half = 0.45 * ng * cell / 4
    src = np.stack([rng.uniform(-half, half, n_comp), rng.uniform(-half, half, n_comp),
                    rng.uniform(-1.0, 2.0, n_comp)], axis=1)
    ref = model_grid.grid_from_components(src, ng, 1.0 / (ng * cell))
    out = torch.empty((ng, ng), dtype=torch.complex64, device="cuda")
    _abi.psc_model_grid_components(src, ng, cell, out)
    assert cases.rel_l2(out.cpu().numpy(), ref) < 1e-6


def test_component_grid_equals_image_grid_for_pixel_sources():
    N, ng, cell = 64, 256, 10.0 * I.ARCSEC
    sky = I.sky_points(30, 4.0 * I.ARCMIN, N, cell, ("loguniform", 0.1, 1.0), 3)
    img = torch.from_numpy(I.sky_image(sky, N, cell).astype(np.float32)).cuda()
    g_img = torch.empty((ng, ng), dtype=torch.complex64, device="cuda")
    _abi.psc_model_grid(N, ng, cell, 32, 20, img, g_img)
    g_cmp = torch.empty_like(g_img)
    _abi.psc_model_grid_components(sky, ng, cell, g_cmp)
    assert cases.rel_l2(g_cmp.cpu().numpy(), g_img.cpu().numpy()) < 1e-6


def _ew(n=6, seed=0):
    rng = np.random.default_rng(seed)
    return np.stack([np.sort(rng.uniform(-300.0, 300.0, n)), np.zeros(n), np.zeros(n)], axis=1)


@pytest.mark.parametrize("layout", ["ew", "y"])
def test_snapshot_plane_matches_oracle(layout):
    enu = _ew() if layout == "ew" else I.y_layout(27, 1000.0, 2)
    ha = np.linspace(-0.1, 0.1, 40) * 15 * I.DEG
    uvw = I.uvw_tracks(enu, 34 * I.DEG, 30 * I.DEG, ha)
    a, b = _abi.psc_snapshot_plane(torch.from_numpy(np.ascontiguousarray(uvw)).cuda(), uvw.shape[0] * uvw.shape[1])
    ra, rb = wsnap.plane_fit(uvw)
    assert abs(a - ra) < 1e-10 * (1 + abs(ra)) and abs(b - rb) < 1e-10 * (1 + abs(rb))
    if layout == "ew":
        assert abs(a) < 1e-10 and b == pytest.approx(-1.0 / math.tan(30 * I.DEG), rel=1e-10)


def _snapshot_problem():
    kind, N, cell_as, Ng = cases.DISK_SMALL
    enu = _ew()
    ha = np.linspace(-0.5, 0.5, 10) * 15 * I.DEG
    uvw = I.uvw_tracks(enu, 34 * I.DEG, 30 * I.DEG, ha)
    freq = np.array([1.4e9])
    cell = cell_as * I.ARCSEC
    sky = I.sky_points(10, 12.0 * I.ARCMIN, N, cell, ("loguniform", 0.1, 1.0), 1)
    lmt = I.true_offsets(enu.shape[0], 20.0 * I.ARCSEC, 1)
    return enu, uvw, freq, cell, Ng, sky, lmt


def _gpu_snapshot_ctx(uvw, freq, n_ant, cell, Ng, sky):
    """plane -> moved components -> grid -> context, all through the ABI."""
    uvw_d = torch.from_numpy(np.ascontiguousarray(uvw)).cuda()
    a, b = _abi.psc_snapshot_plane(uvw_d, uvw.shape[0] * uvw.shape[1])
    comp = _abi.psc_snapshot_components(sky, a, b, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, float(freq[0]))
    grid = torch.empty((Ng, Ng), dtype=torch.complex64, device="cuda")
    _abi.psc_model_grid_components(comp, Ng, cell, grid)
    ctx = _abi.Context(n_ant, uvw.shape[0], len(freq), uvw_d, freq, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, 1,
                       64, Ng, cell, 32, 20, grid)
    return ctx, (uvw_d, grid), (a, b)


def test_snapshot_prediction_matches_oracle_and_the_w_term():
    enu, uvw, freq, cell, Ng, sky, lmt = _snapshot_problem()
    n_ant = enu.shape[0]
    ctx, keep, (a, b) = _gpu_snapshot_ctx(uvw, freq, n_ant, cell, Ng, sky)
    shape = (uvw.shape[0], uvw.shape[1], 1)
    vg = torch.empty(shape, dtype=torch.complex64, device="cuda")
    dg = torch.empty((4,) + shape, dtype=torch.complex64, device="cuda")
    ctx.psc_predict(lmt, vg, dg)
    snap = wsnap.snapshot_sources(sky, *wsnap.plane_fit(uvw), "disk", 1.4e9, 25.0, I.ALPHA_PER_DLAMBDA_DISK)
    m = psc.Model(uvw_m=uvw, freq_hz=freq, n_ant=n_ant, grid=model_grid.grid_from_components(snap, Ng, 1.0 / (Ng * cell)),
                  cell_rad=cell, support=32, oversample=20, ap_kind="disk", diam_m=25.0,
                  alpha_per_dlambda=I.ALPHA_PER_DLAMBDA_DISK, decorrelation=1)
    V, dV = psc.predict(m, lmt)
    assert cases.rel_l2(vg.cpu().numpy(), V) < TOL_V
    for p in range(4):
        assert cases.rel_l2(dg.cpu().numpy()[p], dV[p]) < TOL_V
    Vw = closed_form.visibilities(uvw, freq, n_ant, sky, lmt, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, w_term=True)
    assert cases.rel_l2(vg.cpu().numpy(), Vw) < 1e-4
    ctx.close()


def test_snapshot_solve_removes_the_w_bias():
    """Data with the w-term (direct sum): the snapshot model's GPU solve equals
    the oracle's and lands within 0.5 arcsec, the co-planar model's is off by
    arcseconds (2")."""
    enu, uvw, freq, cell, Ng, sky, lmt = _snapshot_problem()
    n_ant = enu.shape[0]
    Vw = closed_form.visibilities(uvw, freq, n_ant, sky, lmt, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, w_term=True)
    sig = 1e-5
    vobs = (Vw + I.complex_noise(Vw.shape, sig, 7)).astype(np.complex64)
    ctx, keep, _ = _gpu_snapshot_ctx(uvw, freq, n_ant, cell, Ng, sky)
    vd = torch.from_numpy(vobs).cuda()
    sol, rep = ctx.psc_solve_offsets(vd, None, 1.0 / sig ** 2)
    snap = wsnap.snapshot_sources(sky, *wsnap.plane_fit(uvw), "disk", 1.4e9, 25.0, I.ALPHA_PER_DLAMBDA_DISK)
    m = psc.Model(uvw_m=uvw, freq_hz=freq, n_ant=n_ant, grid=model_grid.grid_from_components(snap, Ng, 1.0 / (Ng * cell)),
                  cell_rad=cell, support=32, oversample=20, ap_kind="disk", diam_m=25.0,
                  alpha_per_dlambda=I.ALPHA_PER_DLAMBDA_DISK, decorrelation=1)
    w = np.full(vobs.shape, 1.0 / sig ** 2)

    def ev(p):
        c, g, H, X = psc.chi2_grad_normal(m, p, vobs, w)
        G, A = psc.assemble_full(n_ant, g, H, X)
        return c, G, A
    sol_o, _ = LM.solve_full(ev, np.zeros_like(lmt))
    assert np.max(np.abs(sol - sol_o)) < 0.1 * I.ARCSEC
    assert np.max(np.abs(sol - lmt)) < 0.5 * I.ARCSEC
    # the co-planar model on the same data
    grid0 = torch.empty((Ng, Ng), dtype=torch.complex64, device="cuda")
    _abi.psc_model_grid_components(sky, Ng, cell, grid0)
    ctx0 = _abi.Context(n_ant, uvw.shape[0], 1, keep[0], freq, "disk", 25.0, I.ALPHA_PER_DLAMBDA_DISK, 1,
                        64, Ng, cell, 32, 20, grid0)
    sol0, _ = ctx0.psc_solve_offsets(vd, None, 1.0 / sig ** 2)
    assert np.max(np.abs(sol0 - lmt)) > 1.0 * I.ARCSEC
    ctx.close()
    ctx0.close()


def test_snapshot_plane_rejects_collinear_baselines():
    enu = _ew()
    uvw = I.uvw_tracks(enu, 34 * I.DEG, 30 * I.DEG, np.zeros(1))          # one instant, one line
    with pytest.raises(_abi.PscError):
        _abi.psc_snapshot_plane(torch.from_numpy(np.ascontiguousarray(uvw)).cuda(), uvw.shape[1])


def test_component_grid_without_components_is_zero():
    out = torch.full((130, 130), 1.0 + 1.0j, dtype=torch.complex64, device="cuda")
    _abi.psc_model_grid_components(np.zeros((0, 3)), 130, 5.0 * I.ARCSEC, out)
    assert not torch.any(out).item()
