"""Writes the expected sampled outputs of the strip operator at a size where
the oracle's whole apply is out of reach (d = 2, L = 9: 123 M coefficients).

Outputs y = A^(delta) u (Sect. 4.2, blockwise definition) at the positions
`sgdg_workloads.grid_samples(shapes, 2, seed=SAMPLE_SEED)`, for
u = uniform_vector(size, seed=INPUT_SEED) and for its bfloat16-rounded copy
`round_to_bf16(u)`.  Every value comes from `oracle.operator.apply_rows`;
nothing here reads the CUDA library.  Run from the repository root:

    python tests/golden/make_apply_samples.py 9

(about 10 minutes and 10 GB of host memory at L = 9: the finest-level
assembly of every factor dominates).
"""
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import numpy as np  # noqa: E402

import sgdg_workloads as W  # noqa: E402
from oracle.operator import SparseGridOperator  # noqa: E402

INPUT_SEED = 29
SAMPLE_SEED = 31


def main(L: int) -> None:
    t0 = time.time()
    prob = W.transport_2d(L=L, sigma=0.1)
    op = SparseGridOperator(prob)
    u = W.uniform_vector(op.size, seed=INPUT_SEED)
    ub = W.round_to_bf16(u)
    rows = W.grid_samples(op.shape, 2, seed=SAMPLE_SEED)
    out = op.apply_rows([u, ub], rows)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), f"apply_samples_transport2d_L{L}.txt")
    with open(path, "w") as f:
        f.write(f"# y = A^(delta) u of transport_2d(L={L}, sigma=0.1) at sampled outputs (Sect. 4.2, blockwise)\n")
        f.write(f"# oracle.operator.apply_rows; u = uniform_vector(size={op.size}, seed={INPUT_SEED}); "
                f"ub = round_to_bf16(u); positions grid_samples(shapes, 2, seed={SAMPLE_SEED})\n")
        f.write("# written by tests/golden/make_apply_samples.py\n")
        f.write("# grid k1 k2 y[s=0] y[s=1] yb[s=0] yb[s=1]\n")
        for n, (i, k1, k2) in enumerate(rows):
            f.write(f"{i} {k1} {k2} {float(out[0, n, 0])!r} {float(out[0, n, 1])!r} {float(out[1, n, 0])!r} {float(out[1, n, 1])!r}\n")
    print(f"wrote {path}: {len(rows)} positions in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 9)
