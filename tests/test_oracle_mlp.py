"""Pins of the oracle MLP (oracle/mlp.py): finite differences of the FP64
backward pass, GELU against scipy's normal CDF, AdamW against torch's, and
the bfloat16 rounding against torch's conversion."""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import mlp


def _params(seed=0, scale=0.3):
    rng = np.random.default_rng(seed)
    p = {}
    for name, shp in mlp.SHAPES:
        if name.startswith("W"):
            p[name] = rng.normal(0, scale / math.sqrt(shp[0]), shp)
        elif name.startswith("b"):
            p[name] = rng.normal(0, 0.05, shp)
        elif name == "mu":
            p[name] = rng.normal(0, 0.1, shp)
        else:
            p[name] = rng.uniform(0.5, 2.0, shp)
    return mlp.pack(p)


def test_parameter_count():
    assert mlp.N_PARAMS == 145666 + 104


def test_gelu_is_x_times_normal_cdf():
    z = np.linspace(-6, 6, 101)
    assert np.allclose(mlp.gelu(z), z * stats.norm.cdf(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-8)


def test_backward_matches_finite_differences_in_fp64():
    rng = np.random.default_rng(1)
    flat = _params()
    x = rng.normal(0, 1, (6, mlp.N_IN))
    t = rng.normal(0, 1, (6, mlp.N_OUT))
    L, g = mlp.loss_and_grad(flat, x, t, bf=False)
    mask = mlp.trained_mask()
    idx = rng.choice(np.flatnonzero(mask), 60, replace=False)
    h = 1e-6
    for i in idx:
        e = np.zeros_like(flat)
        e[i] = h
        fd = (mlp.loss_and_grad(flat + e, x, t, bf=False)[0] - mlp.loss_and_grad(flat - e, x, t, bf=False)[0]) / (2 * h)
        assert abs(fd - g[i]) < 1e-6 * max(1.0, abs(g[i]))
    assert np.all(g[~mask] == 0.0)


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(2)
    x = np.concatenate([rng.normal(0, 1, 1000), rng.normal(0, 1e-3, 1000), [0.0, -0.0, 1.0, 3.0039062]])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(mlp.bf16(x), ref)


def test_adamw_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    w0 = rng.normal(0, 1, 40)
    grads = [rng.normal(0, 1, 40) for _ in range(3)]
    p = torch.nn.Parameter(torch.tensor(w0, dtype=torch.float64))
    opt = torch.optim.AdamW([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8, weight_decay=1e-4)
    for g in grads:
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    # the oracle's update on the trained part of a full-length vector
    flat = np.zeros(mlp.N_PARAMS)
    flat[:40] = w0
    m = np.zeros(mlp.N_PARAMS)
    v = np.zeros(mlp.N_PARAMS)
    for k, g in enumerate(grads, start=1):
        gg = np.zeros(mlp.N_PARAMS)
        gg[:40] = g
        flat, m, v = mlp.adamw_step(flat, gg, m, v, k, 1e-2)
    assert np.allclose(flat[:40], p.detach().numpy(), rtol=1e-12, atol=1e-14)
