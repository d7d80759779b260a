"""Input helpers of sgdg_workloads (host only): bfloat16 rounding of apply
inputs and the full-size sample positions."""
import numpy as np

import sgdg_workloads as W


def test_round_to_bf16_exact_cases():
    # bfloat16 keeps 8 significant bits: spacing 2^-7 on [1, 2)
    x = np.array([1.0, 1.0 + 2.0 ** -7, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -2.5, 0.0, 3.0e-39, 1e30])
    y = W.round_to_bf16(x)
    assert y[0] == 1.0 and y[1] == 1.0 + 2.0 ** -7
    assert y[2] == 1.0                              # a tie rounds to the even neighbour
    assert y[3] == 1.0 + 2.0 ** -6                  # 1 + 1.5 * 2^-7: tie, to the even neighbour above
    assert y[4] == -2.5 and y[5] == 0.0
    assert y.dtype == np.float64
    # every result is a bfloat16 value: its float32 pattern has 16 zero low bits
    bits = y.astype(np.float32).view(np.uint32)
    assert np.all(bits & 0xFFFF == 0)
    # rounding error within half a unit in the last place (2^-8 relative)
    u = W.uniform_vector(10000, seed=2)
    r = W.round_to_bf16(u)
    nz = u != 0
    assert np.max(np.abs(r[nz] - u[nz]) / np.abs(u[nz])) <= 2.0 ** -8
    assert np.array_equal(W.round_to_bf16(r), r)   # idempotent


def test_grid_samples_cover_every_grid_and_the_ragged_edges():
    shapes = [(9, 1025), (25, 263), (81, 66), (3, 3)]
    s = W.grid_samples(shapes, 3, seed=5)
    assert len(s) == 3 * len(shapes)
    for i, (n1, n2) in enumerate(shapes):
        mine = [t for t in s if t[0] == i]
        assert (i, n1 - 1, n2 - 1) in mine
        assert all(0 <= k1 < n1 and 0 <= k2 < n2 for _, k1, k2 in mine)
    assert s == W.grid_samples(shapes, 3, seed=5)  # seeded
