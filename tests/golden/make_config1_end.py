"""Writes the end state of the d = 1 free-streaming configuration (x in
[0,1], v in [-1,1], L = 6, dt = 1/32, 16 strips to T = 0.5; exact solution
u0(x - v t, v)) from the oracle's strip solver (Sect. 2 strips, FGMRES + CT,
tol 1e-12): the unique nodal values of U^-(T) at seeded positions, their
l2 norm over all nodes, and the relative l2 error against the exact
solution at the nodes of the finest full grid.  Every value comes from
oracle/; nothing here reads the CUDA library.  From the repository root:

    python tests/golden/make_config1_end.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import numpy as np  # noqa: E402

import sgdg_workloads as W  # noqa: E402
from oracle.solver import StripSolver, full_grid_values, nodal_values  # noqa: E402

SAMPLE_SEED = 37
N_SAMPLES = 200


def main() -> None:
    prob = W.free_streaming_1d(L=6)
    s = StripSolver(prob, tol=1e-12)
    U = s.run()[-1]
    T = prob.n_strips * prob.dt
    nod = nodal_values(s.op, U, R=1)
    idx = W.sample_indices(nod.size, N_SAMPLES, seed=SAMPLE_SEED)
    fine = full_grid_values(s.op, U)
    xs = s.op.hx.levels[prob.L].coords[:, 0]
    vs = s.op.hv.levels[prob.L].coords[:, 0]
    ex = prob.exact(T, xs[:, None], vs[None, :])
    err = float(np.linalg.norm(fine - ex) / np.linalg.norm(ex))
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "config1_end_L6.txt")
    with open(path, "w") as f:
        f.write("# d=1 free streaming, L=6, dt=1/32, 16 strips (T=0.5): oracle end state U^-(T)\n")
        f.write("# written by tests/golden/make_config1_end.py (oracle StripSolver, tol 1e-12)\n")
        f.write(f"# n_nodal {nod.size}\n# nodal_l2 {float(np.linalg.norm(nod))!r}\n")
        f.write(f"# exact_rel_l2_error_finest_grid {err!r}\n")
        f.write(f"# samples: sample_indices(n_nodal, {N_SAMPLES}, seed={SAMPLE_SEED}); index value\n")
        for i in idx:
            f.write(f"{int(i)} {float(nod[i])!r}\n")
    print(f"wrote {path}: error vs exact {err:.3e}, {nod.size} nodal values")


if __name__ == "__main__":
    main()
