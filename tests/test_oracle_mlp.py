"""Pins of the oracle MLP (CPU only): backpropagation against central finite
differences of the loss, and the bfloat16 rounding helper against exactly
representable values and the round-to-nearest-even rule."""
import numpy as np

from oracle.mlp import loss_and_grad, to_bf16


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    n_in, w, n_out, B = 6, 5, 4, 3
    npar = n_in * w + w + w * w + w + w * n_out + n_out
    p = rng.normal(size=npar)
    x = rng.normal(size=(B, n_in))
    t = rng.normal(size=(B, n_out))
    loss, g = loss_and_grad(p, x, t, n_in, w, n_out, in_scale=0.7, out_scale=1.3)
    fd = np.zeros_like(p)
    h = 1e-6
    for i in range(npar):
        e = np.zeros_like(p)
        e[i] = h
        fd[i] = (loss_and_grad(p + e, x, t, n_in, w, n_out, 0.7, 1.3)[0]
                 - loss_and_grad(p - e, x, t, n_in, w, n_out, 0.7, 1.3)[0]) / (2 * h)
    assert np.abs(fd - g).max() < 1e-7 * max(1.0, np.abs(g).max())


def test_bf16_rounding():
    assert to_bf16(np.array([1.0, -2.5, 0.0]))[1] == -2.5
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: ties to even -> 1
    assert to_bf16(np.array([1.0 + 2 ** -8]))[0] == 1.0
    assert to_bf16(np.array([1.0 + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    x = np.random.default_rng(1).normal(size=1000)
    assert np.all(np.abs(to_bf16(x) - x) <= 2 ** -8 * np.abs(x) + 1e-45)
