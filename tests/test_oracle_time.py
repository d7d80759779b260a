"""Pins of the oracle's time-dependent coefficients (Sect. 4.2: beta(t, x, v)
and sigma(t, x, v) in tensor form, the block formula as a quadrature sum
over the strip's time points tau_mu).

* The quadrature form against the literal space-time weak form (Sect. 2,
  Eq. 5) assembled by brute force with beta and sigma evaluated pointwise
  in (t, x, v) and Gamma^-(t) selected per time point, on a strip where the
  v-component of beta changes sign (d = 1, L = 2; d = 2, L = 1).
* Constant time factors (ft = 1 given explicitly) reproduce the exact time
  matrices of the time-constant path.
* Planted mistake: freezing the coefficients at the strip's start instead of
  at every tau_mu fails the brute-force comparison.
* A solution pin independent of the block formula: with beta = 0 and
  delta = 0 every nodal coefficient follows u' = -sigma(t) u, and DG(1)
  (= 2-stage Radau IIA, third order at the strip ends) approaches
  exp(-int sigma) at third order in dt.
"""
from dataclasses import replace

import numpy as np
import scipy.sparse as sp

import sgdg_workloads as W
from oracle import operator as O
from oracle.brute import full_matrix
from oracle.operator import SparseGridOperator


def _blocks_vs_brute(prob, terms, t0):
    op = SparseGridOperator(prob)
    L, R = prob.L, op.R
    Af = full_matrix(prob, L, L, t0=t0)
    err, scale = 0.0, 0.0
    for (l1, l2) in op.grids:
        P = sp.kron(sp.kron(op.hx.embed(L, l1), op.hv.embed(L, l2)), sp.identity(R)).tocsr()
        for (m1, m2) in op.grids:
            Pp = sp.kron(sp.kron(op.hx.embed(L, m1), op.hv.embed(L, m2)), sp.identity(R)).tocsr()
            Ab = (P.T @ (Pp.T @ Af.T).T)
            n1, n2 = op.grid_shape(m1, m2)
            Ak = np.zeros_like(Ab)
            for c in range(n1 * n2 * R):
                e = np.zeros(n1 * n2 * R)
                e[c] = 1.0
                Ak[:, c] = op.apply_block(terms, (l1, l2), (m1, m2), e.reshape(n1, n2, R)).ravel()
            err = max(err, np.abs(Ab - Ak).max())
            scale = max(scale, np.abs(Ab).max())
    return err / scale


def test_sign_change_inside_the_strip():
    prob = W.time_dependent_1d(L=2)
    c = prob.beta[1].ft
    assert c(np.array([0.5]))[0] > 0 > c(np.array([0.625]))[0]


def test_time_dependent_block_formula_vs_brute_force_1d():
    prob = W.time_dependent_1d(L=2)
    t0 = 0.5                                   # cos(3 t) changes sign inside (0.5, 0.625)
    assert _blocks_vs_brute(prob, O.kron_terms(prob, t0), t0) < 1e-13


def test_time_dependent_block_formula_vs_brute_force_2d():
    prob = W.time_dependent_2d(L=1)
    t0 = 0.25                                  # cos(6 t) changes sign inside (0.25, 0.3125)
    c = prob.beta[2].ft
    assert c(np.array([t0]))[0] > 0 > c(np.array([t0 + prob.dt]))[0]
    assert _blocks_vs_brute(prob, O.kron_terms(prob, t0), t0) < 1e-13


def test_constant_time_factors_reproduce_exact_time_matrices():
    prob = W.transport_2d(L=1, sigma=0.2)
    one = lambda t: np.ones_like(np.asarray(t, dtype=float))
    p1 = replace(prob, beta=[replace(b, ft=one) for b in prob.beta], sigma=replace(prob.sigma, ft=one))
    assert O.is_time_dependent(p1) and not O.is_time_dependent(prob)
    op0, op1 = SparseGridOperator(prob), SparseGridOperator(p1)
    op1.set_time(0.3)
    u = W.uniform_vector(op0.size, seed=5)
    y0, y1 = op0.apply(u), op1.apply(u)
    assert np.linalg.norm(y1 - y0) < 1e-13 * np.linalg.norm(y0)


def test_planted_mistake_frozen_at_strip_start_fails():
    prob = W.time_dependent_1d(L=2)
    t0 = 0.5
    frozen = O.kron_terms(O._frozen(prob, t0))     # coefficients of t0 on the whole strip
    assert _blocks_vs_brute(prob, frozen, t0) > 1e-4


def test_decay_ode_third_order():
    """beta = 0, delta = 0, sigma = 2 (1 + t): u(t) = u0 exp(-2 t - t^2).  The
    strip solutions' end values (nodal, any node) converge at order ~3."""
    from oracle.solver import StripSolver, nodal_values
    errs = []
    T = 0.5
    for n in (2, 4, 8):
        prob = W.time_dependent_1d(L=1, dt=T / n, n_strips=n)
        prob = replace(prob, beta=[W.Product(0.0), W.Product(0.0)], delta=0.0,
                       sigma=W.Product(2.0, None, None, lambda t: 1.0 + np.asarray(t)))
        S = StripSolver(prob, tol=1e-13)
        U0 = nodal_values(S.op, _u0_coeffs(S), R=1)
        UT = nodal_values(S.op, S.run()[-1], R=1)
        exact = np.exp(-2 * T - T ** 2)
        mask = np.abs(U0) > 1e-3 * np.abs(U0).max()
        errs.append(np.abs(UT[mask] / U0[mask] - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 2.7), (errs, rates)


def _u0_coeffs(S):
    """Coefficients of the initial L2 projection P u0 on the sparse grid (the
    strip scheme starts from it): solve M_sg c = (u0, phi)."""
    import scipy.sparse.linalg as spla
    mu = S.initial_mass_u0()
    n = mu.size
    A = spla.LinearOperator((n, n), matvec=S.mass_spatial)
    c, info = spla.cg(A, mu, rtol=1e-14, maxiter=5000)
    return c
