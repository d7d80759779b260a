"""Plain FP64 multilayer perceptron: the reference for the library's BF16 MLP.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Same model and parameter layout as the library: y = W3^T relu(W2^T relu(W1^T x
+ b1) + b2) + b3 per sample, W_k stored [fan_in][fan_out], parameters
flattened as W1, b1, W2, b2, W3, b3; inputs scaled by in_scale, targets by
out_scale; loss 1/(2B) sum (y - t out_scale)^2.  Backpropagation written out
by hand; pinned by central finite differences (tests/test_oracle_mlp.py).
"""
from __future__ import annotations

import numpy as np


def unpack(p: np.ndarray, n_in: int, w: int, n_out: int):
    dims = [(n_in, w), (w, w), (w, n_out)]
    out, o = [], 0
    for fi, fo in dims:
        W = p[o:o + fi * fo].reshape(fi, fo)
        o += fi * fo
        b = p[o:o + fo]
        o += fo
        out.append((W, b))
    return out


def forward(p, x, n_in, w, n_out, in_scale=1.0):
    (W1, b1), (W2, b2), (W3, b3) = unpack(np.asarray(p, dtype=np.float64), n_in, w, n_out)
    X = np.asarray(x, dtype=np.float64) * in_scale
    Z1 = X @ W1 + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ W2 + b2
    H2 = np.maximum(Z2, 0.0)
    Y = H2 @ W3 + b3
    return Y, (X, H1, H2)


def loss_and_grad(p, x, t, n_in, w, n_out, in_scale=1.0, out_scale=1.0):
    (W1, b1), (W2, b2), (W3, b3) = unpack(np.asarray(p, dtype=np.float64), n_in, w, n_out)
    Y, (X, H1, H2) = forward(p, x, n_in, w, n_out, in_scale)
    B = X.shape[0]
    R = Y - np.asarray(t, dtype=np.float64) * out_scale
    loss = 0.5 * np.sum(R ** 2) / B
    dY = R / B
    gW3 = H2.T @ dY
    gb3 = dY.sum(axis=0)
    dH2 = (dY @ W3.T) * (H2 > 0)
    gW2 = H1.T @ dH2
    gb2 = dH2.sum(axis=0)
    dH1 = (dH2 @ W2.T) * (H1 > 0)
    gW1 = X.T @ dH1
    gb1 = dH1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return loss, g


def to_bf16(a: np.ndarray) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
