"""psc_residual_grad_noalloc: the allocation-free fused evaluation.

It serves callers that cannot call cudaMalloc, for example code whose device
memory belongs to another allocator, or a real-time loop where
cudaMalloc/cudaFree (which can synchronise the device) are not acceptable.
It keeps its scratch in the library's static device array.  The test calls it
through the C ABI twice in a row, at different offsets, and checks each result
against psc_residual_grad on the same inputs.  The second call shows that
what the first left in the shared array does not leak into the next.  This
file is collected last and builds everything it needs, so it passes alone in
a fresh process as well as after the other tests.
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
        assert abs(got[0] - ref[0]) <= TOL * abs(ref[0])
        gscale = np.max(np.abs(ref[2]))          # normal blocks set the scale of g terms
        assert np.max(np.abs(got[1] - ref[1])) <= TOL * max(np.max(np.abs(ref[1])), 1e-12 * gscale)
        assert np.max(np.abs(got[2] - ref[2])) <= TOL * np.max(np.abs(ref[2]))
        assert np.max(np.abs(got[3] - ref[3])) <= TOL * np.max(np.abs(ref[2]))


def test_noalloc_rejects_problems_beyond_its_scratch():
    n_ant = 512                                  # 130,816 baselines: > 16 MiB of partial sums
    dummy = torch.zeros(8, dtype=torch.float64, device="cuda:0")
    vis = torch.zeros(8, dtype=torch.complex64, device="cuda:0")
    with pytest.raises(_abi.PscError) as e:
        _abi.psc_residual_grad_noalloc(n_ant, 1, 1, dummy, np.array([1.4e9]), "disk", 25.0,
                                       I.ALPHA_PER_DLAMBDA_DISK, 1, 64, 1024, 1e-4, 32, 20, vis,
                                       np.zeros((n_ant, 2)), vis)
    assert e.value.status == _abi.PSC_ERR_ARG
    assert "bytes of scratch" in str(e.value)
