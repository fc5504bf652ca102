"""psc_residual_grad_noalloc: the allocation-free fused evaluation.

It serves callers that cannot call cudaMalloc, for example code whose device
memory belongs to another allocator, or a real-time loop where
cudaMalloc/cudaFree (which can synchronise the device) are not acceptable.
It keeps its scratch in the library's static device array.  The test calls it
through the C ABI twice in a row, at different offsets.  Each result must
equal bit for bit that of psc_residual_grad on the same inputs with the same
tiling (the same kernels on the same inputs), and match the FP64 oracle at the
parity tolerances.  The second call shows that what the first left in the
shared array does not leak into the next.  This file is collected last and
builds everything it needs, so it passes alone in a fresh process as well as
after the other tests.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import psc

import cases
from gpu_cases import GpuProblem

TOL = 1e-5


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _noalloc(gp, m, lm, vobs, w):
    nt, nbl, nc = gp.shape
    return _abi.psc_residual_grad_noalloc(
        m.n_ant, nt, nc, gp.uvw, m.freq_hz, m.ap_kind, m.diam_m, m.alpha_per_dlambda, m.decorrelation,
        gp.grid_n_img, m.grid.shape[0], m.cell_rad, m.support, m.oversample, gp.grid, lm, vobs, w, 1.0, cross=True)


def test_noalloc_matches_residual_grad_on_two_calls():
    m, _, lmt, img = cases.problem(cases.DISK_SMALL, n_ant=7, n_time=40,
                                   freqs=(1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), sigma_arcsec=30.0)
    V, _ = psc.predict(m, lmt, False)
    vobs = (V + I.complex_noise(V.shape, 1e-3, 7)).astype(np.complex64)
    w = np.full(V.shape, 1e6, dtype=np.float32)
    gp = GpuProblem(m, img)                     # default tiling (32, 4), like the allocation-free path
    gp.grid_n_img = img.shape[0]
    dv, dw = gp.upload(vobs), gp.upload(w, torch.float32)
    for lm in (0.5 * lmt, np.zeros_like(lmt)):
        ref = gp.ctx.psc_residual_grad(lm, dv, dw, 1.0, cross=True)
        got = _noalloc(gp, m, lm, dv, dw)
        # same kernels, inputs and launch shape: identical results
        assert got[0] == ref[0]
        for k in (1, 2, 3):
            assert np.array_equal(got[k], ref[k]), k
        # and the oracle's, at the parity tolerances
        chi2, g, H, X = psc.chi2_grad_normal(m, lm, vobs.astype(np.complex128), w.astype(np.float64))
        Vm, dV = psc.predict(m, lm)
        R = vobs - Vm
        scale_chi = chi2 + np.sum(2 * w * np.abs(R) * np.abs(Vm))
        assert abs(got[0] - chi2) <= TOL * scale_chi
        gsum = np.zeros_like(g)                 # sum |2 w R dV| per gradient entry: its cancellation scale
        ij = m.antenna_pairs()
        for b, (i, j) in enumerate(ij):
            a = 2 * np.sum(w[:, b] * np.abs(R[:, b])[None] * np.abs(dV[:, :, b]), axis=(1, 2))
            gsum[i] += a[0], a[1]
            gsum[j] += a[2], a[3]
        assert np.all(np.abs(got[1] - g) <= TOL * gsum)
        assert np.max(np.abs(got[2] - H)) <= TOL * np.max(np.abs(H))
        assert np.max(np.abs(got[3] - X)) <= TOL * np.max(np.abs(H))


def test_noalloc_rejects_problems_beyond_its_scratch():
    # 512 antennas (130,816 baselines), one time step and channel: the partial
    # sums alone exceed the 16 MiB scratch.  Every input is allocated at the
    # full size of this problem, so nothing is read out of bounds even if the
    # check did not fire.
    n_ant, ng = 512, 1024
    n_bl = n_ant * (n_ant - 1) // 2
    uvw = torch.zeros((1, n_bl, 3), dtype=torch.float64, device="cuda:0")
    vis = torch.zeros((1, n_bl, 1), dtype=torch.complex64, device="cuda:0")
    grid = torch.zeros((ng, ng), dtype=torch.complex64, device="cuda:0")
    with pytest.raises(_abi.PscError) as e:
        _abi.psc_residual_grad_noalloc(n_ant, 1, 1, uvw, np.array([1.4e9]), "disk", 25.0,
                                       I.ALPHA_PER_DLAMBDA_DISK, 1, 64, ng, 1e-4, 32, 20, grid,
                                       np.zeros((n_ant, 2)), vis)
    assert e.value.status == _abi.PSC_ERR_ARG
    assert "bytes of scratch" in str(e.value)
