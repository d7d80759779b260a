"""Pins of the oracle's Vlasov-Poisson field update (CPU only).

* the periodic P1 Poisson solve of a cosine source against the exact
  potential phi = -(alpha/k^2) cos(k x1) (second-order convergence) and the
  exact field energy 1/2 int |E|^2 = 4 pi^2 (alpha/k)^2 on [0, 4 pi]^2;
* the density of u0 against the closed form (1 + alpha cos(k x1)) int g dv.
"""
import numpy as np
import pytest

import sgdg_workloads as W
from oracle.field import density_u0, poisson
from oracle.operator import SparseGridOperator

ALPHA, K = 0.01, 0.5


def _setup(L):
    prob = W.landau_4d(L=L, alpha=ALPHA, k=K)
    return prob, SparseGridOperator(prob)


def test_poisson_cosine_converges_second_order():
    errs = []
    for L in (2, 3, 4):
        prob, op = _setup(L)
        x = op.hx.levels[L].coords
        rho = 1.0 + ALPHA * np.cos(K * x[:, 0])
        phi, E, energy = poisson(op, rho)
        exact = -(ALPHA / K ** 2) * np.cos(K * x[:, 0])
        errs.append(np.abs(phi - exact).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(rates > 1.8), (errs, rates)
    assert errs[-1] < 5e-3 * ALPHA / K ** 2
    exact_energy = 4 * np.pi ** 2 * (ALPHA / K) ** 2      # 1/2 (alpha/k)^2 * 2 pi * 4 pi
    assert abs(energy - exact_energy) < 0.02 * exact_energy


def test_planted_sign_error_in_poisson_fails():
    """Solving with the source's sign flipped would give +phi_exact: the pin
    above distinguishes it."""
    prob, op = _setup(3)
    x = op.hx.levels[3].coords
    rho = 1.0 + ALPHA * np.cos(K * x[:, 0])
    phi_bad, _, _ = poisson(op, 2.0 - rho)
    exact = -(ALPHA / K ** 2) * np.cos(K * x[:, 0])
    assert np.abs(phi_bad - exact).max() > 0.5 * ALPHA / K ** 2


def test_density_of_u0():
    prob, op = _setup(3)
    x = op.hx.levels[3].coords
    rho = density_u0(op, prob)
    g = 1.0   # int exp(-|v|^2/2)/(2 pi) over [-6,6]^2 = erf(6/sqrt 2)^2 = 1 - 4e-9
    assert np.allclose(rho, (1.0 + ALPHA * np.cos(K * x[:, 0])) * g, rtol=2e-3, atol=0)
