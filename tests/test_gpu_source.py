"""Strips with a source f on the GPU (Sect. 2, b_j with the streamline-
diffusion pairing (f, w + delta (d_t w + beta . grad w))).

* the library reproduces a solution inside the discrete space (hat functions
  in x and v, linear in t) to its solver tolerance, FP64 and mixed;
* smooth manufactured solutions (d = 1 and d = 2): the strips agree with
  the oracle's strips on the canonical nodal values within 1e-8.
"""
import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_05988_gb300 as P
    P.load_library()
    return P


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _solver(P, prob, prec):
    return P.Solver(prob, precision=P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32, rtol=1e-11,
                    restart=30, inner_its=30, inner_rtol=1e-4)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_discrete_solution_is_reproduced(P, prec):
    from oracle.operator import SparseGridOperator
    from oracle.solver import nodal_values
    prob = W.discrete_manufactured_1d(L=3)
    op = SparseGridOperator(prob)
    s = _solver(P, prob, prec)
    s.set_initial()
    for j in range(prob.n_strips):
        st = s.advance_strip()
        assert st.rel_residual <= 1e-11
    U = np.empty(s.n_spatial)
    s.get_end_value(U, on_device=False)
    vals = nodal_values(op, U, R=1)
    T = prob.dt * prob.n_strips
    off, err, scale = 0, 0.0, 0.0
    for (l1, l2) in op.grids:
        n1, n2 = op.grid_shape(l1, l2)
        ex = prob.exact(T, op.hx.levels[l1].coords[:, 0][:, None], op.hv.levels[l2].coords[:, 0][None, :])
        err = max(err, np.abs(vals[off:off + n1 * n2].reshape(n1, n2) - ex).max())
        scale = max(scale, np.abs(ex).max())
        off += n1 * n2
    assert err < 1e-8 * scale


@pytest.mark.parametrize("case", ["d1-fp64", "d1-mixed", "d2-fp64"])
def test_source_strip_parity(P, case):
    from oracle.solver import StripSolver, nodal_values
    d, prec = case.split("-")
    prob = (W.manufactured_1d(L=4, n_strips=2, seed=3) if d == "d1"
            else W.manufactured_2d(L=2, n_strips=2, dt=1.0 / 16.0, seed=1))
    ref = StripSolver(prob, tol=1e-12)
    ends_ref = ref.run()
    s = _solver(P, prob, prec)
    s.set_initial()
    for j in range(prob.n_strips):
        st = s.advance_strip()
        assert st.rel_residual <= 1e-11
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        a = nodal_values(ref.op, U, R=1)
        b = nodal_values(ref.op, ends_ref[j], R=1)
        assert _rel(a, b) < 1e-8, (j, _rel(a, b))


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


@pytest.mark.parametrize("case", ["d1-fp64", "d1-mixed", "d2-fp64", "d2-mixed"])
def test_inflow_data_solution_is_reproduced_and_matches_oracle(P, case):
    """Nonzero inflow data g on Gamma^- (b_j's -int <g, w>_{Gamma^-} dt, Sect. 2):
    u* = a(t) X(x) V(v) linear in t, x and v with f and g = u* on Gamma^-
    (inflow on every side of both boxes) is reproduced by the library to the
    solver tolerance at every node, and the strips agree with the oracle's."""
    from oracle.solver import StripSolver, nodal_values
    d, prec = case.split("-")
    prob = W.inflow_manufactured_1d(L=3) if d == "d1" else W.inflow_manufactured_2d(L=2)
    ref = StripSolver(prob, tol=1e-12)
    ends_ref = ref.run()
    s = _solver(P, prob, prec)
    s.set_initial()
    for j in range(prob.n_strips):
        st = s.advance_strip()
        assert st.rel_residual <= 1e-11
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        got = nodal_values(ref.op, U, R=1)
        ex = _nodal_exact(ref.op, prob.exact, (j + 1) * prob.dt)
        assert np.abs(got - ex).max() < 1e-8 * np.abs(ex).max(), j
        assert _rel(got, nodal_values(ref.op, ends_ref[j], R=1)) < 1e-8, j
    s.close()
