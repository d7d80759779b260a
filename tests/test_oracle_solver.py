"""Pins of the oracle's solver path (CPU only).

* L = 0: the sparse grid is one full grid, the CT preconditioner is the exact
  inverse and the outer Krylov solve takes one iteration;
* the CT residual restriction (Algorithm 1) gives the same lower-grid residual
  from either parent grid, because the lower grid's test functions lie in
  both parents' spaces;
* dim V_L (Table 1, "dof" column) equals the rank of the Gram matrix of the
  spanning set (Sect. 4.1) for the periodic P1 spaces of Sect. 5.1;
* mass conservation for periodic problems with sigma = f = 0 (test function
  w = 1 lies in V_L);
* free streaming converges to the exact solution u0(x - v t, v).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import sgdg_workloads as W
from oracle.assembly import assemble_load
from oracle.brute import _cell_data
from oracle.operator import SparseGridOperator
from oracle.solver import (ComponentSolver, StripSolver,
                           full_grid_values, nodal_values, richardson)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_L0_ct_is_exact_inverse():
    prob = W.free_streaming_1d(L=0, n_strips=2)
    s = StripSolver(prob, tol=1e-12)
    s.run()
    assert s.outer_its == [1, 1]


def test_component_direct_solve_equals_gmres():
    """The assembled component block equals the blockwise apply_diag column
    by column, and its LU solve equals the GMRES solve on the same block."""
    prob = W.transport_2d(L=2, sigma=0.1)
    op = SparseGridOperator(prob)
    direct = ComponentSolver(op, tol=1e-13)
    krylov = ComponentSolver(op, tol=1e-13, direct_max=0)
    rng = np.random.default_rng(5)
    for (l1, l2) in op.grids:
        n1, n2 = op.grid_shape(l1, l2)
        A = direct.block_matrix(l1, l2)
        u = rng.uniform(-1, 1, (n1, n2, op.R))
        assert np.abs(A @ u.ravel() - op.apply_diag(l1, l2, u).ravel()).max() < 1e-13 * np.abs(A).max()
        r = rng.uniform(-1, 1, (n1, n2, op.R))
        xd, xk = direct.solve(l1, l2, r), krylov.solve(l1, l2, r)
        assert np.linalg.norm(xd - xk) < 1e-10 * np.linalg.norm(xd)
    assert krylov.iterations and max(krylov.iterations) > 1


def test_ct_restriction_from_either_parent():
    prob = W.transport_2d(L=3, sigma=0.1)
    op = SparseGridOperator(prob)
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, op.size)
    b = rng.uniform(-1, 1, op.size)
    r = op.apply(u) - op.apply_mass(b)     # a residual: test-function evaluations
    L = op.L
    for l in range(L):
        via1 = op.left(op.hx.E[l].T.tocsr(), op.block(r, l + 1))      # from (l+1, L-1-l)
        via2 = op.right(op.hv.E[L - 1 - l].T.tocsr(), op.block(r, l))  # from (l, L-l)
        assert np.abs(via1 - via2).max() < 1e-13 * np.abs(via1).max()


def _load_table(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append(line.split())
    return rows


@pytest.mark.parametrize("row", [r for r in _load_table("table1_dof.txt")
                                 if (int(r[0]) == 1 and int(r[1]) <= 4) or (int(r[0]) == 2 and int(r[1]) <= 2)],
                         ids=lambda r: f"d{r[0]}_L{r[1]}")
def test_table1_dof_is_rank_of_spanning_set(row):
    d, Lp, dof = int(row[0]), int(row[1]), int(row[2])
    if d == 1:
        mesh = lambda: W.interval_mesh(0, 1, 4, periodic=True)
    else:
        mesh = lambda: W.square_mesh(0, 1, 4, periodic=True)
    prob = W.Problem(name="dof", d=d, mesh_x=mesh(), mesh_v=mesh(), L=Lp - 1, r=0, dt=1.0,
                     delta=0.0, n_strips=1, beta=[W.Product(0.0)] * (2 * d),
                     sigma=W.Product(0.0), u0=[])
    op = SparseGridOperator(prob)
    G = op.dense(op.mass_terms())
    ev = np.linalg.eigvalsh(0.5 * (G + G.T))
    rank = int(np.sum(ev > 1e-10 * ev.max()))
    assert rank == dof


def test_mass_conservation_periodic():
    prob = W.periodic_advection_1d(L=2)
    prob.u0 = prob.u0 + [W.Product(1.0)]                    # u0 = 1 + sin(2 pi (x + v))
    prob.n_strips = 4
    s = StripSolver(prob, tol=1e-12)
    ends = s.run()
    op = s.op
    ones = []
    for (l1, l2) in op.grids:
        ex = op.fx.embed(l1).T @ assemble_load(op.hx.levels[op.L], None)
        ev = op.fv.embed(l2).T @ assemble_load(op.hv.levels[op.L], None)
        ones.append(np.outer(ex, ev).ravel())
    w = np.concatenate(ones)
    masses = [w @ U for U in ends]
    assert np.allclose(masses, 1.0, rtol=1e-10, atol=0)


def _l2_error(op, U, exact, t):
    L = op.L
    F = full_grid_values(op, U)
    lx, lv = op.hx.levels[L], op.hv.levels[L]
    px, wx, lamx, _ = _cell_data(lx, 5)
    pv, wv, lamv, _ = _cell_data(lv, 5)
    err = 0.0
    for cx in range(px.shape[0]):
        ux = F[lx.cells[cx]]
        for cv in range(pv.shape[0]):
            val = lamx @ ux[:, lv.cells[cv]] @ lamv.T
            ex = exact(t, px[cx][:, 0][:, None], pv[cv][:, 0][None, :])
            err += np.sum(np.outer(wx[cx], wv[cv]) * (val - ex) ** 2)
    return np.sqrt(err)


def test_free_streaming_converges():
    errs = []
    for L in (2, 3, 4):
        prob = W.free_streaming_1d(L=L, n_strips=4)
        s = StripSolver(prob, tol=1e-10)
        ends = s.run()
        errs.append(_l2_error(s.op, ends[-1], prob.exact, 4 * prob.dt))
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert errs[-1] < 5e-3
    assert np.all(rates > 1.2), (errs, rates)


def test_richardson_and_fgmres_agree():
    """Algorithm 1 (Richardson + CT) and FGMRES + CT reach the same function."""
    prob = W.free_streaming_1d(L=2, n_strips=1)
    s = StripSolver(prob, tol=1e-12)
    b = s.rhs(s.initial_mass_u0())
    x1, _, _ = s.solve_strip(b)
    x2, its = richardson(s.op, s.comp, b, tol=1e-13)
    n1 = nodal_values(s.op, x1, R=2)
    n2 = nodal_values(s.op, x2, R=2)
    assert np.abs(n1 - n2).max() < 1e-9 * np.abs(n1).max()
    assert its < 60


def _hat_values(lev, pts):
    """H[a, k] = phi_k(pts[a]) for the P1 basis of one mesh level, from the
    cells' geometry (barycentric coordinates), independent of the embeddings."""
    cc, cells = lev.cell_coords, lev.cells
    d = pts.shape[1]
    H = np.zeros((pts.shape[0], lev.n))
    for a, p in enumerate(pts):
        for c in range(cells.shape[0]):
            v0 = cc[c, 0]
            J = (cc[c, 1:] - v0).T
            lam_r = np.linalg.solve(J, p - v0)
            lam = np.concatenate([[1.0 - lam_r.sum()], lam_r])
            if lam.min() >= -1e-12:
                for k, l in zip(cells[c], lam):
                    H[a, k] += l
                break
        else:
            raise AssertionError("point outside the mesh")
    return H


@pytest.mark.parametrize("make,targets", [
    (lambda: W.free_streaming_1d(L=3, n_strips=1), [(0, 0), (1, 2), (2, 2), (3, 1)]),
    (lambda: W.transport_2d(L=2, sigma=0.0), [(0, 0), (1, 1), (2, 0)]),
], ids=["d1", "d2"])
def test_coarse_values_are_point_values(make, targets):
    """coarse_values (the warm start's coarse view) against the sparse-grid
    function evaluated at the coarse grid's node coordinates by summing every
    component grid's P1 (x) P1 basis functions there."""
    from oracle.solver import coarse_values
    prob = make()
    op = SparseGridOperator(prob)
    rng = np.random.default_rng(5)
    for R in (1, 2):
        U = rng.uniform(-1, 1, op.size // op.R * R)
        for lx, lv in targets:
            X = op.hx.levels[lx].coords
            V = op.hv.levels[lv].coords
            ref = np.zeros((X.shape[0], V.shape[0], R))
            off = 0
            for (l1, l2) in op.grids:
                n1, n2 = op.grid_shape(l1, l2)
                u = U[off:off + n1 * n2 * R].reshape(n1, n2, R)
                off += n1 * n2 * R
                ref += np.einsum("ai,ijs,bj->abs", _hat_values(op.hx.levels[l1], X), u,
                                 _hat_values(op.hv.levels[l2], V))
            got = coarse_values(op, U, R, lx, lv)
            assert np.abs(got - ref.ravel()).max() < 1e-12 * max(1.0, np.abs(ref).max())
