"""psc_features (stencil kernel) against the oracle's features."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import inputs as I
from oracle import features as F, psc

import cases
from gpu_cases import GpuProblem

SIG = 30.0 * I.ARCSEC


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("spec,n_ant,nt,freqs,stride", [
    (cases.DISK_SMALL, 7, 40, (1.2e9, 1.3e9, 1.4e9, 1.5e9, 1.6e9), 1),
    (cases.DISK_SMALL, 6, 45, (1.3e9, 1.4e9), 2),
    (cases.GAUSS_SMALL, 5, 12, (1.4e9,), 3),
    # bricks of exactly one warp (kept steps x channels = 32), four to a block;
    # 15 and 21 baselines leave the last block partly empty
    (cases.DISK_SMALL, 6, 12, tuple(1.3e9 + 0.03e9 * k for k in range(8)), 3),
    (cases.GAUSS_SMALL, 7, 60, tuple(1.3e9 + 0.0125e9 * k for k in range(16)), 30),
])
def test_features_match_oracle(spec, n_ant, nt, freqs, stride):
    m, _, lmt, img = cases.problem(spec, n_ant=n_ant, n_time=nt, freqs=freqs, sigma_arcsec=30.0)
    V, _ = psc.predict(m, lmt, False)
    vobs = (V + I.complex_noise(V.shape, 1e-3, 9)).astype(np.complex64)
    w = np.full(V.shape, 1e6, dtype=np.float32)
    ref = F.features(m, vobs, w, SIG, stride)
    gp = GpuProblem(m, img)
    got = gp.ctx.psc_features(gp.upload(vobs), gp.upload(w, torch.float32), 1.0, SIG, stride).cpu().numpy()
    assert np.max(np.abs(got[:, :2] - ref[:, :2])) < 1e-4
    assert np.max(np.abs(got[:, 2:27] / ref[:, 2:27] - 1.0)) < 1e-5
    assert np.max(np.abs(got[:, 27:] - ref[:, 27:])) < 1e-5 * max(1.0, np.max(np.abs(ref[:, 27:])))
