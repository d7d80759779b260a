"""Pins of the oracle's inflow data g (Sect. 2: b_j holds
-int_{I_j} <g, w>_{Gamma^-} dt with <u, w>_Gamma = int (beta . n) u w).

A solution inside the discrete space that does not vanish on the boundary,
u* = a(t) X(x) V(v) with X, V linear and a linear in t, with f = d_t u* +
beta . grad u* + sigma u* and g = u* on Gamma^-: the weak form is consistent,
so the strip solutions reproduce u* up to the solver tolerance at every node
of every component grid.  beta = (v, x - 1/2) (d = 1) and (v1, v2, x2 - 1/2,
1/2 - x1) (d = 2) put inflow on every side of both boxes.  A planted mistake,
the same problem with g dropped, misses u* by a large margin.
"""
import numpy as np
import pytest

import sgdg_workloads as W
from oracle.solver import StripSolver, nodal_values


def _nodal_exact(op, exact, t):
    out = []
    for (l1, l2) in op.grids:
        X = op.hx.levels[l1].coords
        V = op.hv.levels[l2].coords
        if X.shape[1] == 1:
            out.append(exact(t, X[:, 0][:, None], V[:, 0][None, :]).ravel())
        else:
            out.append(exact(t, X[:, None, :], V[None, :, :]).ravel())
    return np.concatenate(out)


@pytest.mark.parametrize("make", [lambda: W.inflow_manufactured_1d(L=3), lambda: W.inflow_manufactured_2d(L=2)],
                         ids=["d1", "d2"])
def test_inflow_solution_is_reproduced(make):
    prob = make()
    s = StripSolver(prob, tol=1e-12)
    ends = s.run()
    for j, U in enumerate(ends):
        got = nodal_values(s.op, U)
        ref = _nodal_exact(s.op, prob.exact, (j + 1) * prob.dt)
        assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max(), j


def test_dropping_g_misses_the_solution():
    prob = W.inflow_manufactured_1d(L=3, n_strips=1)
    prob.g = []
    s = StripSolver(prob, tol=1e-12)
    U = s.run()[0]
    got = nodal_values(s.op, U)
    ref = _nodal_exact(s.op, prob.exact, prob.dt)
    assert np.abs(got - ref).max() > 1e-2 * np.abs(ref).max()
