"""Pins of the oracle's norms and, through them, of its whole strip-solve path.

* Table 1 (Sect. 5.1), d = 1, r = 1: the error of the periodic advection
  problem (Eq. 25) in the streamline-diffusion norm (Eq. 11) after one period
  with 2^(L+1) strips (paper levels L = 1..6).  The oracle's errors come out
  3-9% above the printed ones, whether measured against the exact solution
  or against the paper's reference, the P2 interpolant in V_{L+1} (the two
  differ by under 0.5%; test below).  The test asks each error to lie within
  [1.0, 1.12] times the printed one from L = 2 to 6, and each estimated order
  within 0.05 of the printed order from L = 3 on (1.37, 1.49, 1.50, 1.50).
  A planted mistake, a streamline-diffusion parameter off by a factor 2,
  moves the error by about 40% and fails the band.
* The H^1(J x Omega) norm of Algorithm 1's stop test: closed forms for a
  function constant in space (constant and linear in time) and for a
  function linear in x; the Gram-form evaluation against the independent
  evaluation from finest-full-grid values and cell quadrature on random
  spanning-set vectors.
"""
import os

import numpy as np
import pytest

import sgdg_workloads as W
from oracle.norms import SparseInterpolant, h1_norm, h1_norm_nodal, sd_norm_error, sd_norm_error_interp
from oracle.operator import SparseGridOperator
from oracle.solver import StripSolver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table1():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_error_d1_r1.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                Lp, h, err, order = line.split()
                rows[int(Lp)] = (float(err), float(order))
    return rows


def _sd_error(Lp, delta_factor=1.0):
    prob = W.periodic_advection_1d(L=Lp - 1)
    prob.delta *= delta_factor
    s = StripSolver(prob, tol=1e-11)
    sols = []
    s.run(solutions=sols)
    return sd_norm_error(prob, s.op, sols, prob.exact)[0]


def test_table1_error_and_order_d1_r1():
    ref = _table1()
    errs = {Lp: _sd_error(Lp) for Lp in range(1, 7)}
    for Lp in range(2, 7):
        ratio = errs[Lp] / ref[Lp][0]
        assert 1.0 <= ratio <= 1.12, (Lp, errs[Lp], ref[Lp][0])
    for Lp in range(3, 7):
        order = np.log2(errs[Lp - 1] / errs[Lp])
        assert abs(order - ref[Lp][1]) <= 0.05, (Lp, order, ref[Lp][1])


def test_table1_band_rejects_wrong_delta():
    ref = _table1()
    for fac in (0.5, 2.0):
        ratio = _sd_error(3, fac) / ref[3][0]
        assert not (1.0 <= ratio <= 1.12), (fac, ratio)


def _constant_in_space(op, coef_t):
    """Spanning-set coefficients of coef_t[s] eta_s(t) * 1: the constant P1
    function on grid (0, L) (all nodal values 1), zero elsewhere."""
    u = np.zeros(op.size)
    blk = op.block(u, 0)
    blk[:, :, :] = np.asarray(coef_t)[None, None, :]
    return u


@pytest.mark.parametrize("make", [lambda: W.free_streaming_1d(L=2, n_strips=1),
                                  lambda: W.transport_2d(L=1, sigma=0.0)], ids=["d1", "d2"])
def test_h1_norm_closed_forms(make):
    prob = make()
    op = SparseGridOperator(prob)
    lo_x, hi_x = np.array(prob.mesh_x.lo), np.array(prob.mesh_x.hi)
    lo_v, hi_v = np.array(prob.mesh_v.lo), np.array(prob.mesh_v.hi)
    vol = np.prod(hi_x - lo_x) * np.prod(hi_v - lo_v)
    dt = prob.dt
    # 1: |J| |Omega|
    assert h1_norm(op, _constant_in_space(op, [1.0, 0.0])) ** 2 == pytest.approx(dt * vol, rel=1e-12)
    # eta_1(t) = 2 (t - t0)/dt - 1: int eta_1^2 = dt/3, int (eta_1')^2 = 4/dt
    assert h1_norm(op, _constant_in_space(op, [0.0, 1.0])) ** 2 == pytest.approx((dt / 3 + 4 / dt) * vol,
                                                                                 rel=1e-12)
    # x_1 on grid (L, 0) (eta_0): int_J int x1^2 + 1 = dt (|Omega| (<x1^2> + 1))
    L = op.L
    u = np.zeros(op.size)
    blk = op.block(u, L)
    x1 = op.hx.levels[L].coords[:, 0]
    blk[:, :, 0] = x1[:, None]
    mean_x1sq = (hi_x[0] ** 3 - lo_x[0] ** 3) / (3 * (hi_x[0] - lo_x[0]))
    assert h1_norm(op, u) ** 2 == pytest.approx(dt * vol * (mean_x1sq + 1.0), rel=1e-12)


@pytest.mark.parametrize("make", [lambda: W.free_streaming_1d(L=3, n_strips=1),
                                  lambda: W.transport_2d(L=2, sigma=0.1)], ids=["d1", "d2"])
def test_h1_gram_equals_nodal_quadrature(make):
    prob = make()
    op = SparseGridOperator(prob)
    for seed in (1, 2):
        u = W.uniform_vector(op.size, seed=seed)
        a, b = h1_norm(op, u), h1_norm_nodal(op, u)
        assert abs(a - b) < 1e-10 * b, (a, b)


def test_sparse_interpolant_telescopes_to_the_full_grid_one():
    """For u = q(x) g(v) with q quadratic (held exactly by the coarsest P2
    space) the combination sum over |l| = L+1 minus |l| = L telescopes to q
    times the level-(L+1) interpolant of g: the full-grid interpolant on
    (L+1, L+1).  A wrong sign or level range breaks it."""
    prob = W.periodic_advection_1d(L=2)
    I = SparseInterpolant(prob, 2)
    fn = lambda t, x, v: (x * x - x) * np.sin(2 * np.pi * v) * np.cos(t)
    X, V = I.Hx.levels[3].coords[:, 0], I.Hv.levels[3].coords[:, 0]
    assert np.abs(I(fn, 0.3) - fn(0.3, X[:, None], V[None, :])).max() < 1e-13
    # a full product is not in the sparse space: the interpolant differs
    g = lambda t, x, v: np.sin(2 * np.pi * x) * np.sin(2 * np.pi * v)
    assert np.abs(I(g, 0.0) - g(0.0, X[:, None], V[None, :])).max() > 1e-7


def test_interpolant_reference_changes_table1_errors_little():
    """Table 1's reference (the P2 interpolant in V_{L+1}) against the exact
    solution as reference: within 0.5% at paper levels 1-3, since the
    interpolation error is of higher order than the scheme's.  (Both stay
    about 8% above the printed errors from level 2 on; the streamline term,
    which depends on U alone here because d_t u + beta . grad u = 0, carries
    over 90% of the norm.)"""
    for Lp in (1, 2, 3):
        prob = W.periodic_advection_1d(L=Lp - 1)
        s = StripSolver(prob, tol=1e-11)
        sols = []
        s.run(solutions=sols)
        e = sd_norm_error(prob, s.op, sols, prob.exact)[0]
        ei = sd_norm_error_interp(prob, s.op, sols, prob.exact)[0]
        assert abs(ei / e - 1.0) < 5e-3, (Lp, e, ei)
