"""Pins of the oracle's Vlasov-Poisson field update (CPU only).

* the periodic P1 Poisson solve of a cosine source against the exact
  potential phi = -(alpha/k^2) cos(k x1) (second-order convergence) and the
  exact field energy 1/2 int |E|^2 = 4 pi^2 (alpha/k)^2 on [0, 4 pi]^2;
* the density of u0 against the closed form (1 + alpha cos(k x1)) int g dv.
"""
import numpy as np

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


def _vp_first_strip(alpha, L=2, eps=1e-8):
    from oracle.field import density_u0, vp_strip
    from oracle.solver import StripSolver
    prob = W.landau_4d(L=L, alpha=alpha, k=K, n_strips=1, dt=0.25)
    s = StripSolver(prob, tol=1e-12)
    op = s.op
    MU = s.initial_mass_u0()
    # U^-_0: the spanning-set vector of the projection of u0 is not needed as
    # such; f^(0) only enters through its H1 distance, taken from the
    # oracle's own solve of the first strip's mass problem M_sg U = (u0, phi)
    U0 = np.linalg.lstsq(op.dense(op.mass_terms())[::2, ::2], MU, rcond=None)[0]
    return prob, s, vp_strip(s, prob, U0, density_u0(op, prob), MU, 0.0, eps)


def test_vp_fixed_point_uniform_density_is_immediate():
    """alpha = 0: the density is uniform, the field vanishes, the strip
    solution of an x-independent state is constant in time - the fixed point
    of Sect. 5.3 stops after its first solve with a zero field."""
    prob, s, (u, E, its, crit) = _vp_first_strip(0.0)
    assert its == 1 and np.abs(E).max() < 1e-12 and crit < 1e-8


def test_vp_fixed_point_converges_and_is_consistent():
    """alpha = 0.01: a few alternations reach the tolerance; the returned
    solution solves the strip with the field it returns, and that field is
    the midpoint field of the solution to within the tolerance."""
    from oracle.field import density, install_field, poisson
    from oracle.norms import h1_norm
    prob, s, (u, E, its, crit) = _vp_first_strip(0.01)
    assert 2 <= its <= 10 and crit < 1e-8
    op = s.op
    rho = density(op, u.reshape(-1, op.R)[:, 0])
    _, E_mid, _ = poisson(op, rho)
    assert np.abs(E_mid - E).max() < 1e-8
    install_field(op, prob, E)
    b = s.rhs(s.initial_mass_u0(), 0.0)
    r = op.apply(u) - b
    assert np.linalg.norm(r) < 1e-10 * np.linalg.norm(b)
    assert h1_norm(op, u) > 0
