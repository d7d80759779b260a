"""Pins of the oracle's strip operator (CPU only).

* time matrices against their closed forms for the Legendre basis;
* DG(1) in time is the 2-stage Radau IIA method: the end-value amplification
  of a pure reaction problem equals R(z) = (1 + z/3) / (1 - 2z/3 + z^2/6);
* the Kronecker block formula of Sect. 4.2 (with the delta on K~ taken from
  the weak form) against a literal full-grid assembly of the weak form
  (Sect. 2) - and a planted mistake (the block formula as printed, without
  delta on K~) must fail that comparison;
* the energy identity of the stability lemma (Sect. 3, sigma = 0).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import sgdg_workloads as W
from oracle import operator as O
from oracle.brute import energy_terms, full_matrix
from oracle.operator import SparseGridOperator, time_matrices


def test_time_matrices_closed_form():
    for dt in (1.0 / 32, 0.3):
        Mt, Tt, Ct, Gt = time_matrices(dt, 1)
        assert np.allclose(Mt, dt * np.diag([1.0, 1.0 / 3.0]), rtol=1e-14, atol=1e-16)
        assert np.allclose(Tt, [[0.0, 2.0], [0.0, 0.0]], atol=1e-14)
        assert np.allclose(Ct, [[0.0, 0.0], [0.0, 4.0 / dt]], rtol=1e-14, atol=1e-12)
        assert np.allclose(Gt, [[1.0, -1.0], [-1.0, 1.0]], atol=1e-15)


@pytest.mark.parametrize("z", [-0.1, -1.0, -7.5])
def test_dg1_is_radau_iia(z):
    dt = 0.25
    sigma = -z / dt
    Mt, Tt, Ct, Gt = time_matrices(dt, 1)
    e0 = O.eta_at(1, 0.0)
    e1 = O.eta_at(1, 1.0)
    c = np.linalg.solve(Tt + Gt + sigma * Mt, e0)     # y0 = 1
    R = (1 + z / 3) / (1 - 2 * z / 3 + z * z / 6)
    assert abs(e1 @ c - R) < 1e-14


def _blocks_vs_brute(prob, terms):
    op = SparseGridOperator(prob)
    L, R = prob.L, op.R
    Af = full_matrix(prob, L, L)
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


@pytest.mark.parametrize("prob", [W.free_streaming_1d(L=2), W.transport_2d(L=1, sigma=0.3)],
                         ids=["d1_free_streaming", "d2_field_sigma"])
def test_block_formula_vs_brute_force(prob):
    op = SparseGridOperator(prob)
    assert _blocks_vs_brute(prob, op.terms) < 1e-13


def test_planted_mistake_printed_block_formula_fails():
    """The block formula exactly as printed (K~ without delta) disagrees with
    the weak form when sigma != 0: the comparison above would catch it."""
    prob = W.transport_2d(L=1, sigma=0.3)
    Mt, Tt, Ct, Gt = time_matrices(prob.dt, 1)
    ops = O.spatial_operators(prob)
    good = O.kron_terms(prob)
    kt = [(X, V) for X, V in ops["Kt"]]
    bad = [(tau, X, V) for tau, X, V in good if (X, V) not in kt]
    assert len(bad) == len(good) - len(kt) > 0
    bad += [(Mt, X, V) for X, V in ops["Kt"]]          # + K~ instead of + delta K~
    assert _blocks_vs_brute(prob, bad) > 1e-8          # the correct list agrees to ~1e-15


def test_planted_mistake_sign_of_inflow_fails():
    prob = W.free_streaming_1d(L=2)
    ops = O.spatial_operators(prob)
    Mt = time_matrices(prob.dt, 1)[0]
    gx = [X for X, _ in ops["G"]]
    bad = [((-tau if X in gx else tau), X, V) for tau, X, V in O.kron_terms(prob)]
    assert sum(X in gx for _, X, _ in bad) > 0
    assert _blocks_vs_brute(prob, bad) > 1e-8


@pytest.mark.parametrize("prob", [W.free_streaming_1d(L=2), W.transport_2d(L=1, sigma=0.0)],
                         ids=["d1", "d2"])
def test_energy_identity(prob):
    """sigma = 0: A(v, v) = int 1/2|v|^2_dOmega + delta||d_t v + d_beta v||^2
    + 1/2||v_0^+||^2 + 1/2||v_1^-||^2 (Sect. 3)."""
    op = SparseGridOperator(prob)
    L, R = prob.L, op.R
    rng = np.random.default_rng(3)
    # a random sparse-grid function, embedded into the full grid (L, L)
    u = rng.uniform(-1, 1, op.size)
    ufull = np.zeros(op.hx.levels[L].n * op.hv.levels[L].n * R)
    for i, (l1, l2) in enumerate(op.grids):
        P = sp.kron(sp.kron(op.hx.embed(L, l1), op.hv.embed(L, l2)), sp.identity(R))
        ufull += P @ op.block(u, i).ravel()
    lhs = u @ op.apply(u)
    rhs = energy_terms(prob, L, L, ufull)
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


def test_blockwise_apply_matches_dense_and_ordering_rule():
    """Both factor orders of the ordering rule give the same block (exact
    arithmetic); the dense assembled matrix times u equals the blockwise apply."""
    prob = W.transport_2d(L=2, sigma=0.1)
    op = SparseGridOperator(prob)
    rng = np.random.default_rng(5)
    u = rng.uniform(-1, 1, op.size)
    y = op.apply(u)
    # re-do every block with the other factor order
    y2 = np.zeros_like(y)
    for i, (l1, l2) in enumerate(op.grids):
        acc = 0.0
        for j, (m1, m2) in enumerate(op.grids):
            ub = op.block(u, j)
            for tau, X, V in op.terms:
                S1, S2 = op.fx.proj(X, l1, m1), op.fv.proj(V, l2, m2)
                if m1 + l2 <= l1 + m2:
                    w = op.right(S2, op.left(S1, ub))
                else:
                    w = op.left(S1, op.right(S2, ub))
                acc = acc + op.time(tau, w)
        y2[op.offsets[i]:op.offsets[i + 1]] = acc.ravel()
    assert np.abs(y - y2).max() < 1e-12 * np.abs(y).max()


@pytest.mark.parametrize("prob", [W.transport_2d(L=3, sigma=0.1), W.free_streaming_1d(L=4)],
                         ids=["d2_L3", "d1_L4"])
def test_sampled_outputs_match_blockwise_apply(prob):
    """apply_rows (rows of the projected factors from the finest-level matrix,
    used where the whole apply is out of reach) returns the blockwise apply's
    outputs: first and last rows and columns and interior ones, every grid,
    two input vectors at once."""
    op = SparseGridOperator(prob)
    us = [W.uniform_vector(op.size, seed=3), W.uniform_vector(op.size, seed=4)]
    rows = [(i, k1, k2) for i, (n1, n2) in enumerate(op.shape)
            for k1 in sorted({0, n1 - 1, n1 // 2}) for k2 in sorted({0, n2 - 1, n2 // 3})]
    out = op.apply_rows(us, rows)
    for q, u in enumerate(us):
        y = op.apply(u)
        ref = np.array([op.block(y, i)[k1, k2] for (i, k1, k2) in rows])
        assert np.abs(out[q] - ref).max() < 1e-13 * np.abs(ref).max()
