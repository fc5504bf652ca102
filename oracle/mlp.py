"""Oracle: the learned initial estimate's MLP, forward, backward and AdamW (FP64).

Test infrastructure only (see ``oracle/__init__``).  Not a construct of the
paper (the learned initial estimate is an addition to the method).

Network: 52 -> 256 -> 256 -> 256 -> 2, GELU (exact, 0.5 x (1 + erf(x / sqrt 2)))
after the three hidden layers, input standardised by fixed (mu, s).  Flat
parameter vector (FP32 on the GPU):
    W1 [52][256], b1 [256], W2 [256][256], b2, W3 [256][256], b3,
    W4 [256][2], b4 [2], mu [52], s [52]
(W stored [in][out], y = x W + b).  Loss: L = (1/B) sum_b sum_o (y_bo - t_bo)^2.

Precision model of the GPU kernels, reproduced here when ``bf16=True``: every
GEMM operand (weights, the standardised input, GELU outputs, and the output
gradients entering the backward GEMMs) is rounded to bfloat16 (round to
nearest even on the FP32 bit pattern); sums, biases, GELU and the optimiser
are FP32 on the GPU and FP64 here.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

N_IN, N_HID, N_OUT = 52, 256, 2
SHAPES = [("W1", (N_IN, N_HID)), ("b1", (N_HID,)), ("W2", (N_HID, N_HID)), ("b2", (N_HID,)),
          ("W3", (N_HID, N_HID)), ("b3", (N_HID,)), ("W4", (N_HID, N_OUT)), ("b4", (N_OUT,)),
          ("mu", (N_IN,)), ("s", (N_IN,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)
TRAINED = ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")


def unpack(flat):
    out, off = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = np.asarray(flat[off:off + n], dtype=np.float64).reshape(shp)
        off += n
    return out


def pack(p):
    return np.concatenate([np.asarray(p[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def bf16(x):
    """Round to bfloat16 (nearest even) via the FP32 bit pattern; returns float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + special.erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + special.erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(flat, x, bf=True):
    """Output [B][2] and the cache for ``backward``."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    p = unpack(flat)
    xn = (np.asarray(x, dtype=np.float64) - p["mu"]) / p["s"]
    a = [r(xn)]
    zs = []
    for k in (1, 2, 3):
        z = a[-1] @ r(p["W%d" % k]) + p["b%d" % k]
        zs.append(z)
        a.append(r(gelu(z)))
    y = a[-1] @ r(p["W4"]) + p["b4"]
    return y, (a, zs, p)


def loss_and_grad(flat, x, t, bf=True):
    """(L, gradient vector shaped like ``flat``; zero for mu and s)."""
    r = bf16 if bf else (lambda v: np.asarray(v, dtype=np.float64))
    y, (a, zs, p) = forward(flat, x, bf)
    B = y.shape[0]
    t = np.asarray(t, dtype=np.float64)
    L = float(np.sum((y - t) ** 2) / B)
    g = {name: np.zeros(shp) for name, shp in SHAPES}
    dy = 2.0 * (y - t) / B
    g["W4"] = a[3].T @ r(dy)
    g["b4"] = dy.sum(axis=0)
    da = r(dy) @ r(p["W4"]).T
    for k in (3, 2, 1):
        dz = da * gelu_grad(zs[k - 1])
        g["W%d" % k] = a[k - 1].T @ r(dz)
        g["b%d" % k] = dz.sum(axis=0)
        if k > 1:
            da = r(dz) @ r(p["W%d" % k]).T
    return L, pack(g)


def adamw_step(flat, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, wd=1e-4):
    """One AdamW update (decoupled weight decay) of the trained entries;
    ``step`` counts from 1.  Returns (flat, m, v)."""
    flat = np.array(flat, dtype=np.float64)
    m = beta1 * np.asarray(m) + (1 - beta1) * grad
    v = beta2 * np.asarray(v) + (1 - beta2) * grad * grad
    mh = m / (1 - beta1 ** step)
    vh = v / (1 - beta2 ** step)
    mask = trained_mask()
    upd = lr * (mh / (np.sqrt(vh) + eps) + wd * flat)
    flat = np.where(mask, flat - upd, flat)
    return flat, m, v


def trained_mask():
    mask = np.zeros(N_PARAMS, dtype=bool)
    off = 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        mask[off:off + n] = name in TRAINED
        off += n
    return mask
