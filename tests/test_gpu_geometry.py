"""psc_uvw (baseline coordinates from antenna positions) against the FP64
oracle's rotation matrices, and a solve on a geometry built by it."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi, inputs as I
from oracle import geometry as G

DEG = math.pi / 180.0


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("n_ant,n_time,lat,dec", [(2, 1, 34.0, 30.0), (27, 60, 34.0, 30.0), (197, 3, -30.0, -60.0),
                                                  (64, 17, 0.0, 89.0)])
def test_uvw_matches_oracle(n_ant, n_time, lat, dec):
    rng = np.random.default_rng(n_ant)
    enu = rng.normal(0.0, 2000.0, (n_ant, 3)) * np.array([1.0, 1.0, 0.01])
    ha = np.linspace(-1.5, 1.5, n_time) * 15 * DEG
    out = torch.empty((n_time, n_ant * (n_ant - 1) // 2, 3), dtype=torch.float64, device="cuda")
    _abi.psc_uvw(enu, lat * DEG, dec * DEG, ha, out)
    ref = G.uvw(enu, lat * DEG, dec * DEG, ha)
    assert np.max(np.abs(out.cpu().numpy() - ref)) < 1e-9 * np.max(np.abs(ref))


def test_uvw_refusals():
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    with pytest.raises(_abi.PscError):
        _abi.psc_uvw(np.zeros((1, 3)), 0.5, 0.5, [0.0], out)              # one antenna
    with pytest.raises(_abi.PscError):
        _abi.psc_uvw(np.zeros((2, 3)), 2.0, 0.5, [0.0], out)              # latitude out of range
    with pytest.raises(_abi.PscError):
        _abi.psc_uvw(np.array([[0.0, 0.0, 0.0], [np.nan, 0.0, 0.0]]), 0.5, 0.5, [0.0], out)
