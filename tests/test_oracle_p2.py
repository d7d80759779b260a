"""Pins of the oracle's continuous P2 spaces (Sect. 2 with r = 2; Table 1's
r = 2 column).

* Element matrices against the textbook closed forms on one interval of
  length h: mass h/30 [[4, -1, 2], [-1, 4, 2], [2, 2, 16]] and stiffness
  1/(3h) [[7, 1, -8], [1, 7, -8], [-8, -8, 16]] (nodes: end points, then the
  midpoint).
* The embedding: rows sum to one, quadratics are carried exactly (d = 1, 2),
  the Galerkin projection of the fine mass is the coarse mass, and the
  nested embeddings compose.
* Mass rows integrate the basis (total |Omega|); Green's identity
  D_p + D_p^T = the face masses on a non-periodic box (d = 2).
* Table 1 (Sect. 5.1), d = 1, r = 2: the dof column is the rank of the
  spanning set (paper levels 1-3), and the streamline-diffusion error of the
  periodic advection problem after one period lies within 5% of the printed
  error with the estimated order within 0.05 of the printed one (paper levels
  1-4; level 5 gives 1.003 times the printed error and order 2.499).  Planted mistake: P2 in
  space with time-DG degree 1 misses the printed errors.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import sgdg_workloads as W
from oracle.assembly import Factor, FactorStore, assemble_level
from oracle.mesh import P2Hierarchy
from oracle.norms import sd_norm_error
from oracle.operator import SparseGridOperator
from oracle.solver import StripSolver

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _table():
    rows = {}
    with open(os.path.join(GOLDEN, "table1_error_d1_r2.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                Lp, h, dof, err, order = line.split()
                rows[int(Lp)] = (int(dof), float(err), float(order))
    return rows


def test_element_matrices_closed_forms():
    h = 0.25
    hier = P2Hierarchy(W.interval_mesh(0.0, h, 1), 0)
    lev = hier.levels[0]
    assert lev.n == 3 and lev.cells.shape == (1, 3)
    perm = lev.cells[0]                      # local (end, end, mid) -> global
    M = assemble_level(lev, Factor("vol")).toarray()[np.ix_(perm, perm)]
    K = assemble_level(lev, Factor("vol", 1.0, (), 1, 1)).toarray()[np.ix_(perm, perm)]
    M_ref = h / 30.0 * np.array([[4, -1, 2], [-1, 4, 2], [2, 2, 16]])
    K_ref = 1.0 / (3.0 * h) * np.array([[7, 1, -8], [1, 7, -8], [-8, -8, 16]])
    assert np.abs(M - M_ref).max() < 1e-15
    assert np.abs(K - K_ref).max() < 1e-12


@pytest.mark.parametrize("mesh", [W.interval_mesh(-1.0, 1.0, 4), W.square_mesh(0.0, 1.0, 2)], ids=["d1", "d2"])
def test_embedding_carries_quadratics(mesh):
    hier = P2Hierarchy(mesh, 2)
    f = lambda X: 0.3 + X[:, 0] ** 2 - 0.7 * X[:, 0] * X[:, -1] + 0.2 * X[:, -1]
    for l in range(2):
        E = hier.E[l]
        assert np.abs(E @ np.ones(E.shape[1]) - 1.0).max() < 1e-14
        assert np.abs(E @ f(hier.levels[l].coords) - f(hier.levels[l + 1].coords)).max() < 1e-14
    E20 = hier.embed(2, 0)
    assert np.abs(E20 @ f(hier.levels[0].coords) - f(hier.levels[2].coords)).max() < 1e-14


@pytest.mark.parametrize("mesh,vol", [(W.interval_mesh(0.0, 1.0, 4, periodic=True), 1.0),
                                      (W.square_mesh(-1.0, 1.0, 2), 4.0)], ids=["d1_periodic", "d2"])
def test_mass_galerkin_and_total(mesh, vol):
    hier = P2Hierarchy(mesh, 2)
    fs = FactorStore(hier)
    M2 = fs.fine(Factor("vol"))
    assert abs(M2.sum() - vol) < 1e-13
    for l in range(2):
        M_coarse = assemble_level(hier.levels[l], Factor("vol"))
        assert np.abs((fs.proj(Factor("vol"), l, l) - M_coarse).toarray()).max() < 1e-14


def test_green_identity_p2():
    hier = P2Hierarchy(W.square_mesh(0.0, 1.0, 2), 1)
    lev = hier.levels[1]
    for p in (1, 2):
        D = assemble_level(lev, Factor("vol", 1.0, (), 0, p))      # int d_p phi_j phi_i
        faces = sum(side * assemble_level(lev, Factor("face", 1.0, (), 0, 0, (), (p - 1, side)))
                    for side in (-1, 1))
        assert np.abs((D + D.T - faces).toarray()).max() < 1e-13


@pytest.mark.parametrize("Lp", [1, 2, 3])
def test_table1_dof_r2_is_rank_of_spanning_set(Lp):
    dof = _table()[Lp][0]
    mesh = lambda: W.interval_mesh(0, 1, 4, periodic=True)
    prob = W.Problem(name="dof", d=1, mesh_x=mesh(), mesh_v=mesh(), L=Lp - 1, r=0, dt=1.0, delta=0.0,
                     n_strips=1, beta=[W.Product(0.0)] * 2, sigma=W.Product(0.0), u0=[], order=2)
    op = SparseGridOperator(prob)
    G = op.dense(op.mass_terms())
    ev = np.linalg.eigvalsh(0.5 * (G + G.T))
    assert int(np.sum(ev > 1e-10 * ev.max())) == dof


def _sd_error(Lp, time_degree=2):
    prob = W.periodic_advection_1d(L=Lp - 1, r=2)
    prob.r = time_degree
    s = StripSolver(prob, tol=1e-11)
    sols = []
    s.run(solutions=sols)
    return sd_norm_error(prob, s.op, sols, prob.exact)[0]


def test_table1_error_and_order_d1_r2():
    ref = _table()
    errs = {Lp: _sd_error(Lp) for Lp in (1, 2, 3, 4)}
    for Lp, e in errs.items():
        assert 0.95 <= e / ref[Lp][1] <= 1.05, (Lp, e, ref[Lp][1])
    for Lp in (2, 3, 4):
        order = np.log2(errs[Lp - 1] / errs[Lp])
        assert abs(order - ref[Lp][2]) <= 0.05, (Lp, order, ref[Lp][2])


def test_planted_mistake_time_degree_one_misses_table1():
    ref = _table()
    e = _sd_error(3, time_degree=1)
    assert not (0.95 <= e / ref[3][1] <= 1.05), e / ref[3][1]
