"""The learned initial estimate's network on the GPU (BF16 tensor-core GEMMs,
FP32 accumulation) against the FP64 oracle with the same BF16 rounding
points: forward output, per-parameter gradients, one AdamW step, and a
short training run that must lower the loss."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_1709_08681_gb300 import _abi
from oracle import mlp as O


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def init_params(seed):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in O.SHAPES:
        if name.startswith("W"):
            p[name] = rng.normal(0, math.sqrt(2.0 / shp[0]), shp)
        elif name.startswith("b"):
            p[name] = rng.normal(0, 0.02, shp)
        elif name == "mu":
            p[name] = rng.normal(0, 0.2, shp)
        else:
            p[name] = rng.uniform(0.5, 2.0, shp)
    return O.pack(p).astype(np.float32)


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("B", [1, 37, 300])
def test_forward_and_grad_match_oracle(B):
    rng = np.random.default_rng(B)
    flat = init_params(1)
    x = rng.normal(0, 1, (B, O.N_IN)).astype(np.float32)
    t = rng.normal(0, 1, (B, O.N_OUT)).astype(np.float32)
    net = _abi.Mlp(512)
    net.psc_mlp_set_params(flat)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    y = net.psc_mlp_forward(xd).cpu().numpy()
    yo, _ = O.forward(flat.astype(np.float64), x.astype(np.float64))
    assert rel(y, yo) < 2e-3
    loss, g = net.psc_mlp_grad(xd, td)
    lo, go = O.loss_and_grad(flat.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(loss - lo) < 2e-3 * lo
    off = 0
    for name, shp in O.SHAPES:
        n = int(np.prod(shp))
        if name in O.TRAINED:
            assert rel(g[off:off + n], go[off:off + n]) < 2e-2, name
        else:
            assert np.all(g[off:off + n] == 0)
        off += n


def test_adamw_step_matches_oracle():
    rng = np.random.default_rng(4)
    flat = init_params(2)
    x = rng.normal(0, 1, (64, O.N_IN)).astype(np.float32)
    t = rng.normal(0, 1, (64, O.N_OUT)).astype(np.float32)
    net = _abi.Mlp(64)
    net.psc_mlp_set_params(flat)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    _, g = net.psc_mlp_grad(xd, td)
    net.psc_mlp_train_step(xd, td, 1e-3)
    got = net.psc_mlp_get_params()
    ref, _, _ = O.adamw_step(flat.astype(np.float64), g.astype(np.float64), np.zeros(O.N_PARAMS),
                             np.zeros(O.N_PARAMS), 1, 1e-3)
    assert np.max(np.abs(got - ref)) < 1e-6


def test_training_lowers_the_loss():
    """Fit a smooth function of the inputs; the loss must drop by 10x."""
    rng = np.random.default_rng(5)
    flat = init_params(3)
    flat[O.N_PARAMS - 104:O.N_PARAMS - 52] = 0.0        # mu
    flat[O.N_PARAMS - 52:] = 1.0                          # s
    x = rng.normal(0, 1, (2048, O.N_IN)).astype(np.float32)
    t = np.stack([np.tanh(x[:, 0] + 0.5 * x[:, 1]), 0.5 * x[:, 2] * x[:, 3]], axis=1).astype(np.float32)
    net = _abi.Mlp(256)
    net.psc_mlp_set_params(flat)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    first = net.psc_mlp_train_step(xd[:256], td[:256], 1e-3, want_loss=True)
    last = None
    for it in range(400):
        k = (it * 256) % 2048
        last = net.psc_mlp_train_step(xd[k:k + 256], td[k:k + 256], 1e-3, want_loss=(it == 399))
    assert last < 0.1 * first
