"""The recursions of the library's linear-cost sweep equal the blockwise
double loop of Sect. 4.2, in exact arithmetic (CPU).

Written here in numpy from the oracle's projected factors and embeddings,
per Kronecker term a = (tau_a, X_a, V_a), grids i = (i, L - i), P the
prolongation E, R its transpose, subscript 1 or 2 the dimension:

* branch A (sources i' <= i): Z_0 = 0, S_i = U_i V_a^T + P_1 Z_i,
  Z_{i+1} = S_i R_2^T, Y_i += tau_a X_a S_i;
* branch B (sources i' > i): Z_{L-1} = (R_1 X_a) U_L,
  Z_i = (R_1 Z_{i+1}) P_2^T + (R_1 X_a) U_{i+1}, Y_i += tau_a Z_i (V_a P_2)^T.

They must give the oracle's blockwise apply (the paper's double loop with its
ordering rule) to rounding, for d = 1, 2, 3, with inflow terms and sigma;
dropping the prolongation in branch A (a plausible slip) does not.
"""
import numpy as np
import pytest

import sgdg_workloads as W
from oracle.operator import SparseGridOperator


def _sweep(op, u, drop_prolongation=False):
    L, R = op.L, op.R
    U = [op.block(u, i) for i in range(L + 1)]
    Y = [np.zeros_like(Ui) for Ui in U]
    Ex, Ev = op.hx.E, op.hv.E            # E[l]: level l -> l + 1
    left, right, time = op.left, op.right, op.time
    for tau, Xf, Vf in op.terms:
        X = [op.fx.proj(Xf, l, l) for l in range(L + 1)]
        V = [op.fv.proj(Vf, l, l) for l in range(L + 1)]
        # branch A: S_i on (i, L - i)
        Z = None
        for i in range(L + 1):
            S = right(V[L - i], U[i])
            if Z is not None and not drop_prolongation:
                S = S + left(Ex[i - 1], Z)               # P_1: x level i - 1 -> i
            Y[i] += time(tau, left(X[i], S))
            if i < L:
                Z = right(Ev[L - i - 1].T.tocsr(), S)    # R_2: v level L - i -> L - i - 1
        # branch B: Z_i on (i, L - i - 1)
        Z = None
        for i in range(L - 1, -1, -1):
            RX = (Ex[i].T @ X[i + 1]).tocsr()            # R_1 X_a: x level i + 1 -> i
            Zi = left(RX, U[i + 1])
            if Z is not None:
                Zi = Zi + left(Ex[i].T.tocsr(), right(Ev[L - i - 2], Z))   # (R_1 Z_{i+1}) P_2^T
            Z = Zi
            VP = (V[L - i] @ Ev[L - i - 1]).tocsr()     # V_a P_2: v level L - i - 1 -> L - i
            Y[i] += time(tau, right(VP, Z))
    return np.concatenate([y.ravel() for y in Y])


@pytest.mark.parametrize("make", [lambda: W.inflow_manufactured_1d(L=4), lambda: W.transport_2d(L=3, sigma=0.1),
                                  lambda: W.free_streaming_1d(L=3), lambda: W.transport_3d(L=1)],
                         ids=["d1_inflow", "d2_transport", "d1_periodic", "d3"])
def test_sweep_recursions_equal_the_blockwise_apply(make):
    prob = make()
    op = SparseGridOperator(prob)
    u = W.uniform_vector(op.size, seed=81)
    ref = op.apply(u)
    got = _sweep(op, u)
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()


def test_sweep_without_prolongation_differs():
    prob = W.transport_2d(L=3, sigma=0.1)
    op = SparseGridOperator(prob)
    u = W.uniform_vector(op.size, seed=82)
    ref = op.apply(u)
    assert np.abs(_sweep(op, u, drop_prolongation=True) - ref).max() > 1e-3 * np.abs(ref).max()
