"""Pins of the oracle's inflow data g (Sect. 2: b_j holds
-int_{I_j} <g, w>_{Gamma^-} dt with <u, w>_Gamma = int (beta . n) u w).

A solution inside the discrete space that does not vanish on the boundary,
u* = a(t) X(x) V(v) with X, V linear and a linear in t, with f = d_t u* +
beta . grad u* + sigma u* and g = u* on Gamma^-: the weak form is consistent,
so the strip solutions reproduce u* up to the solver tolerance at every node
of every component grid.  beta = (v, x - 1/2) (d = 1) and (v1, v2, x2 - 1/2,
1/2 - x1) (d = 2) put inflow on every side of both boxes.  A planted mistake,
the same problem with g dropped, misses u* by a large margin.

With a time factor in beta (Sect. 4.2), beta_v = (1 - 3t)(x - 1/2): the
inflow boundary Gamma^-(t) changes within a strip, the inflow integral is the
strip's 3-point Gauss sum with each part gated by the sign of the time
factor, and the source terms carry time factors.  The same reproduction pin
holds; dropping the gate, or freezing the source's time factor, fails.
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


def test_time_dependent_inflow_solution_is_reproduced():
    """beta_v = (1 - 3t)(x - 1/2) changes sign at t = 1/3, inside the third
    strip: the inflow side of the v-boundary moves from x > 1/2 to x < 1/2
    within it.  The source carries the time factor (1 - 3t) a(t), g = u* on
    Gamma^-(t).  The strip solutions reproduce u* at every node."""
    prob = W.inflow_time_dependent_1d(L=3)
    assert prob.n_strips * prob.dt > 1.0 / 3.0 > 2 * prob.dt
    s = StripSolver(prob, tol=1e-12)
    ends = s.run()
    for j, U in enumerate(ends):
        got = nodal_values(s.op, U)
        ref = _nodal_exact(s.op, prob.exact, (j + 1) * prob.dt)
        assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max(), j


def test_time_dependent_inflow_solution_is_reproduced_2d():
    """d = 2: E1 = (1 - 3t)(x2 - 1/2) changes sign inside the third strip,
    E2 = (1 + t)(1/2 - x1) keeps its sign; u* is reproduced at every node."""
    prob = W.inflow_time_dependent_2d(L=1)
    s = StripSolver(prob, tol=1e-12)
    ends = s.run()
    for j, U in enumerate(ends):
        got = nodal_values(s.op, U)
        ref = _nodal_exact(s.op, prob.exact, (j + 1) * prob.dt)
        assert np.abs(got - ref).max() < 1e-8 * np.abs(ref).max(), j


def test_planted_mistake_ungated_time_dependent_inflow_fails(monkeypatch):
    """Dropping the gate (both inflow parts active on the whole strip, each
    weighted by the time factor) misses u* in the strip with the sign change."""
    prob = W.inflow_time_dependent_1d(L=3, n_strips=3)
    orig = StripSolver._gauss_weights

    def ungated(self, t0, ft, bt, gate=None):
        return orig(self, t0, ft, bt, None)

    monkeypatch.setattr(StripSolver, "_gauss_weights", ungated)
    s = StripSolver(prob, tol=1e-12)
    U = s.run()[-1]
    got = nodal_values(s.op, U)
    ref = _nodal_exact(s.op, prob.exact, 3 * prob.dt)
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()


def test_planted_mistake_source_time_factor_frozen_fails():
    """The source's factor (1 - 3t) a(t) frozen at the strip start misses u*."""
    prob = W.inflow_time_dependent_1d(L=3, n_strips=1)
    prob.f[3] = W.Source(0.5, prob.f[3].fx, None, lambda t: 0.0 * np.asarray(t) + 1.0)
    s = StripSolver(prob, tol=1e-12)
    U = s.run()[0]
    got = nodal_values(s.op, U)
    ref = _nodal_exact(s.op, prob.exact, prob.dt)
    assert np.abs(got - ref).max() > 1e-3 * np.abs(ref).max()
