"""The source part of the strip right-hand side (Sect. 2, b_j) in the oracle.

* the gradient load int g d_p phi_i equals -int (d_p g) phi_i for g vanishing
  on the boundary (integration by parts), in 1-D and 2-D;
* a solution inside the discrete space (hat functions in x and v, linear in
  t, zero on the boundary) is reproduced to the solver tolerance: the scheme
  is consistent, so every term of b_j - the (f, w) part, delta (f, d_t w) and
  delta (f, beta . grad w) - must be present and right;
* dropping the streamline-diffusion part of the source breaks that (planted);
* a smooth manufactured solution converges (second order at the nodes).
"""
import numpy as np
import pytest

import sgdg_workloads as W
from oracle.assembly import assemble_load, assemble_load_grad
from oracle.mesh import Hierarchy
from oracle.solver import StripSolver, nodal_values


@pytest.mark.parametrize("d", [1, 2])
def test_gradient_load_integration_by_parts(d):
    mesh = W.interval_mesh(0.0, 1.0, 4) if d == 1 else W.square_mesh(0.0, 1.0, 2)
    lev = Hierarchy(mesh, 2).levels[2]
    if d == 1:
        g = lambda p: p[:, 0] ** 2 * (1 - p[:, 0]) ** 2
        dg = [lambda p: 2 * p[:, 0] * (1 - p[:, 0]) ** 2 - 2 * p[:, 0] ** 2 * (1 - p[:, 0])]
    else:
        g = lambda p: p[:, 0] * (1 - p[:, 0]) * p[:, 1] * (1 - p[:, 1])
        dg = [lambda p: (1 - 2 * p[:, 0]) * p[:, 1] * (1 - p[:, 1]),
              lambda p: p[:, 0] * (1 - p[:, 0]) * (1 - 2 * p[:, 1])]
    for ax in range(d):
        lhs = assemble_load_grad(lev, g, ax)
        rhs = -assemble_load(lev, dg[ax])
        assert np.abs(lhs - rhs).max() < 1e-14 * max(1.0, np.abs(rhs).max())
    # a constant has zero gradient load away from the boundary rows, total zero
    assert abs(assemble_load_grad(lev, None, 0).sum()) < 1e-13


def _nodal_error(prob, S, U, T):
    op = S.op
    vals = nodal_values(op, U, 1)
    err, off = 0.0, 0
    for (l1, l2) in op.grids:
        n1, n2 = op.grid_shape(l1, l2)
        x = op.hx.levels[l1].coords[:, 0]
        v = op.hv.levels[l2].coords[:, 0]
        ex = prob.exact(T, x[:, None], v[None, :])
        err = max(err, np.abs(vals[off:off + n1 * n2].reshape(n1, n2) - ex).max())
        off += n1 * n2
    return err


def _run(prob, drop_sd=False):
    S = StripSolver(prob, tol=1e-12)
    if drop_sd:
        orig = S.source_rhs

        def no_sd(t0):
            d0 = S.prob.delta
            S.prob.delta = 0.0
            try:
                return orig(t0)
            finally:
                S.prob.delta = d0
        S.source_rhs = no_sd
    ends = S.run()
    return _nodal_error(prob, S, ends[-1], prob.dt * prob.n_strips)


def test_discrete_solution_is_reproduced():
    prob = W.discrete_manufactured_1d(L=2)
    assert _run(prob) < 1e-9


def test_planted_missing_sd_source_fails():
    prob = W.discrete_manufactured_1d(L=2)
    assert _run(prob, drop_sd=True) > 1e-5


def test_smooth_manufactured_convergence():
    e2 = _run(W.manufactured_1d(L=2, n_strips=2))
    e3 = _run(W.manufactured_1d(L=3, n_strips=2))
    assert e3 < e2 / 3.0, (e2, e3)
