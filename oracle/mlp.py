"""FP64 reference of the warm-start network (not in the paper; test infrastructure only).

A stack of linear layers z_l = a_{l-1} W_l^T + b_l with ReLU between hidden layers and a
linear output, trained on the mean squared error L = mean((y - t)^2).  The backward pass is
the textbook chain rule:
    dL/dy = 2 (y - t) / (B * out)
    dW_l = dz_l^T a_{l-1},  db_l = sum_rows dz_l,  da_{l-1} = dz_l W_l,  dz_{l-1} = da_{l-1} * 1[z_{l-1} > 0]

With `bf16=True` the reference rounds to bfloat16 (round to nearest even) at the points where
the GPU stores BF16 operands -- the network input, each weight matrix, each hidden activation
and each layer's output cotangent -- and keeps everything else in float64; the GPU then
differs from it only by FP32 accumulation order.  Pinned by: central finite differences of
the FP64 loss (tests/test_oracle_mlp.py) and PyTorch autograd on the same network.
"""
from __future__ import annotations

import numpy as np


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float values to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def _r(x, on):
    return bf16_round(x) if on else np.asarray(x, dtype=np.float64)


def forward(params, X, bf16=False):
    """Returns (y, cache) for params = [(W [out][in], b [out]), ...], X [B][in]."""
    a = _r(X, bf16)
    cache = []
    n = len(params)
    for l, (W, b) in enumerate(params):
        Wr = _r(W, bf16)
        z = a @ Wr.T + np.asarray(b, np.float64)
        cache.append((a, Wr, z))
        if l + 1 < n:
            a = _r(np.maximum(z, 0.0), bf16)
        else:
            a = z
    return a, cache


def loss_grad(params, X, T, bf16=False):
    """(loss, [(dW, db), ...]) of mean((y - t)^2)."""
    y, cache = forward(params, X, bf16)
    B, out = y.shape
    e = y - np.asarray(T, np.float64)
    loss = float(np.mean(e * e))
    dz = 2.0 * e / (B * out)
    grads = [None] * len(params)
    for l in range(len(params) - 1, -1, -1):
        a, Wr, z = cache[l]
        dzr = _r(dz, bf16)
        grads[l] = (dzr.T @ a, dz.sum(axis=0))
        if l > 0:
            da = dzr @ Wr
            dz = da * (cache[l - 1][2] > 0)
    return loss, grads
