"""The caller's tabulated aperture (PSC_AP_TABLE) on the GPU against the
FP64 oracle's table path (oracle/aperture.py): the uniform disk's samples
reproduce the disk path, and a disk with a central blockage -- an a-priori
primary-beam effect the closed forms do not cover -- matches the oracle in
prediction, derivatives, sums and solves, with the brick and the track
kernels and through the allocation-free call."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import aperture, lm as LM, psc

import cases
from gpu_cases import GpuProblem

TOL = 1e-5
SMALL_AP = ("disk", 512, 5.0, 1024)
EPS = 0.2


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _table_model(m, samples):
    return psc.Model(**{**m.__dict__, "ap_kind": "table", "ap_table": samples})


def _obs(m, lmt, sigma=1e-3, seed=7):
    V, _ = psc.predict(m, lmt, False)
    vobs = (V + I.complex_noise(V.shape, sigma, seed)).astype(np.complex64)
    return vobs, np.full(V.shape, 1.0 / sigma ** 2, dtype=np.float32)


def _close(got, ref, tol=TOL):
    assert cases.rel_l2(got, ref) < tol
    assert np.max(np.abs(got - ref)) <= 2 * tol * np.max(np.abs(ref))


def test_disk_samples_reproduce_the_disk_path():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=6, n_time=20, freqs=(1.2e9, 1.4e9), sigma_arcsec=30.0)
    Vd, dVd = GpuProblem(m, img).predict(lmt)
    Vt, dVt = GpuProblem(_table_model(m, aperture.disk_table_samples(20001)), img).predict(lmt)
    _close(Vt, Vd, 1e-6)
    for p in range(4):
        _close(dVt[p], dVd[p], 1e-6)


@pytest.mark.parametrize("spec,kv", [(cases.DISK_SMALL, 0), (SMALL_AP, 2)])
def test_blocked_disk_matches_oracle(spec, kv):
    m, _, lmt, img = cases.problem(spec, n_ant=6, n_time=37, freqs=(1.3e9, 1.4e9, 1.5e9), sigma_arcsec=30.0)
    mt = _table_model(m, aperture.annulus_table_samples(4001, EPS))
    V, dV = psc.predict(mt, lmt)
    gp = GpuProblem(mt, img)
    Vg, dVg = gp.predict(lmt)
    _close(Vg, V)
    for p in range(4):
        _close(dVg[p], dV[p])
    if kv:
        gp.ctx.psc_set_track_tiling(kv)
    vobs, w = _obs(mt, lmt)
    lm = 0.5 * lmt
    chi2, g, H, X = psc.chi2_grad_normal(mt, lm, vobs, w)
    got = gp.ctx.psc_residual_grad(lm, gp.upload(vobs), gp.upload(w, torch.float32), 1.0, cross=True)
    Vl, dVl = psc.predict(mt, lm)
    R = vobs - Vl
    assert abs(got[0] - chi2) < TOL * chi2
    gscale = 2.0 * np.sum(w[None] * np.abs(R)[None] * np.abs(dVl))
    assert np.max(np.abs(got[1] - g)) < TOL * gscale
    assert np.max(np.abs(got[2] - H)) < TOL * np.max(np.abs(H))
    assert np.max(np.abs(got[3] - X)) < TOL * np.max(np.abs(H))


def test_blocked_disk_solve_matches_oracle_and_noalloc_equals_the_context():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=7, n_time=12, freqs=(1.3e9, 1.4e9), n_src=8)
    mt = _table_model(m, aperture.annulus_table_samples(4001, EPS))
    vobs, w = _obs(mt, lmt)

    def ev(p):
        c, g, H, X = psc.chi2_grad_normal(mt, p, vobs, w)
        G, A = psc.assemble_full(mt.n_ant, g, H, X)
        return c, G, A
    sol_o, _ = LM.solve_full(ev, np.zeros((mt.n_ant, 2)))
    gp = GpuProblem(mt, img)
    dv, dw = gp.upload(vobs), gp.upload(w, torch.float32)
    sol_g, rep = gp.ctx.psc_solve_offsets(dv, dw, 1.0)
    assert np.max(np.abs(sol_g - sol_o)) < 0.1 * I.ARCSEC
    ref = gp.ctx.psc_residual_grad(0.5 * lmt, dv, dw, 1.0, cross=True)
    nt, nbl, nc = gp.shape
    got = _abi.psc_residual_grad_noalloc(mt.n_ant, nt, nc, gp.uvw, mt.freq_hz, "table", mt.diam_m,
                                         mt.alpha_per_dlambda, mt.decorrelation, img.shape[0], mt.grid.shape[0],
                                         mt.cell_rad, mt.support, mt.oversample, gp.grid, 0.5 * lmt, dv, dw, 1.0,
                                         cross=True, ap_table=mt.ap_table)
    assert got[0] == ref[0] and all(np.array_equal(a, b) for a, b in zip(got[1:], ref[1:]))


def test_table_refusals():
    m, _, _, img = cases.problem(cases.DISK_SMALL, n_ant=4, n_time=4)
    for bad in (np.array([1.0]), np.array([1.0, np.nan, 0.0])):
        with pytest.raises(_abi.PscError) as e:
            GpuProblem(_table_model(m, bad), img)
        assert e.value.status == _abi.PSC_ERR_ARG
    with pytest.raises(_abi.PscError):
        _abi.psc_snapshot_components(np.array([[1e-3, 0.0, 1.0]]), 0.01, 0.02, "table", 25.0,
                                     I.ALPHA_PER_DLAMBDA_DISK, 1.4e9)
    gp = GpuProblem(_table_model(m, aperture.disk_table_samples(101)), img)
    with pytest.raises(_abi.PscError):
        gp.ctx.psc_set_kernel_model(_abi.PSC_KERNEL_EXACT_DISK)
