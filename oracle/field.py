"""Vlasov-Poisson field update (Sect. 5.3), plainly.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Per strip, from the end value U^-_{j-1} (u0 before the first strip):
  rho(x) = int U dv: sum over the component grids of the x-part of
           U_l (int phi^(2) dv), embedded into the finest x level;
           before the first strip the P1 interpolant of int u0 dv;
  -Delta phi = 1 - rho on the periodic Omega_x (P1, finest level): the
           source's mean is removed and phi has zero mean (bordered system
           [[K, m], [m^T, 0]], m = M 1, solved directly);
  E = -grad phi on every finest cell; beta = (v, -E) is installed in the
           problem as cell-constant factors.

``vp_strip``: the fixed point of Sect. 5.3 on one strip.  Starting from
f^(0) = U^-_{j-1} (constant in time on the strip) and its field E^(0), it
alternates a strip solve with the field frozen, f^(k+1) from E^(k), and the
field of the new solution at the strip midpoint (the midpoint rule),
E^(k+1) from f^(k+1), until
    ||E^(k+1) - E^(k)||_{L^inf(I_j x Omega_x)} + ||f^(k+1) - f^(k)||_{H^1(I_j x Omega)} < eps
(E is constant in time on the strip, so the first norm is the largest cell
value of any component; the second is ``norms.h1_norm_nodal`` of the
difference of the strip functions).  The returned solution is f^(k+1) of the last
solve, the field the one it was solved with.

Pinned by tests/test_oracle_field.py: the Poisson solution of a cosine
density against the exact potential (second-order convergence), the density
of u0, Landau-type energy of a single mode, and the fixed point's
consistency (at convergence the returned strip solution solves the strip
with the field of its own midpoint density, to the tolerance).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import sgdg_workloads as W

from .assembly import CellField, Factor, assemble_level, assemble_load
from .operator import SparseGridOperator, kron_terms


def density_u0(op: SparseGridOperator, prob) -> np.ndarray:
    lev = op.hx.levels[op.L]
    rho = np.zeros(lev.n)
    for pr in prob.u0:
        fx = pr.fx(lev.coords) if pr.fx is not None else np.ones(lev.n)
        integ = assemble_load(op.hv.levels[op.L], pr.fv).sum()
        rho += pr.coef * fx * integ
    return rho


def density(op: SparseGridOperator, U: np.ndarray) -> np.ndarray:
    """rho at the finest x vertices from a spatial sparse-grid vector U."""
    L = op.L
    rho = np.zeros(op.hx.levels[L].n)
    off = 0
    for (l1, l2) in op.grids:
        n1, n2 = op.grid_shape(l1, l2)
        Ul = U[off:off + n1 * n2].reshape(n1, n2)
        off += n1 * n2
        mv = assemble_load(op.hv.levels[l2], None)
        rho += op.hx.embed(L, l1) @ (Ul @ mv)
    return rho


def poisson(op: SparseGridOperator, rho: np.ndarray):
    """phi (vertices) and E (per finest cell, shape (d, nc)) of -Delta phi = 1 - rho."""
    lev = op.hx.levels[op.L]
    d = lev.coords.shape[1]
    M = assemble_level(lev, Factor("vol"))
    K = sum(assemble_level(lev, Factor("vol", 1.0, (), i, i)) for i in range(1, d + 1))
    b = M @ (1.0 - rho)
    m = M @ np.ones(lev.n)
    b = b - m * (b.sum() / m.sum())
    A = sp.bmat([[K, sp.csr_matrix(m[:, None])], [sp.csr_matrix(m[None, :]), None]]).tocsc()
    sol = spla.spsolve(A, np.concatenate([b, [0.0]]))
    phi = sol[:-1]
    cc = lev.cell_coords
    v0 = cc[:, 0, :]
    J = np.transpose(cc[:, 1:, :] - v0[:, None, :], (0, 2, 1))
    Jinv = np.linalg.inv(J)
    dphi = phi[lev.cells[:, 1:]] - phi[lev.cells[:, :1]]          # (nc, d)
    grad = np.einsum("cak,ca->ck", Jinv, dphi)                    # J^{-T} dphi
    E = -grad.T
    area = np.abs(np.linalg.det(J)) / (1.0 if d == 1 else 2.0)
    energy = 0.5 * float(np.sum(area * np.sum(E ** 2, axis=0)))
    return phi, E, energy


def install_field(op: SparseGridOperator, prob, E: np.ndarray) -> None:
    """beta_{d+i} = -E_i(x) as cell-constant factors; rebuilds the term list."""
    d = prob.d
    for i in range(d):
        prob.beta[d + i] = W.Product(prob.beta[d + i].coef, CellField(E[i]), None)
    op.terms = kron_terms(prob)


def constant_in_time(U: np.ndarray, R: int) -> np.ndarray:
    """The strip vector of a spatial function constant on the strip
    (coefficient of eta_0 = 1; higher Legendre coefficients zero)."""
    u = np.zeros((U.size, R))
    u[:, 0] = U
    return u.ravel()


def vp_strip(solver, prob, U_prev: np.ndarray, rho_prev: np.ndarray, MU: np.ndarray, t0: float,
             eps: float, max_fp: int = 50):
    """One strip of the Vlasov-Poisson fixed point (Sect. 5.3).

    solver: an oracle StripSolver of the problem (its operator's field is
    replaced); U_prev: U^-_{j-1}; rho_prev: its density (the caller passes
    the interpolant of int u0 dv before the first strip); MU: M_sg U^-_{j-1}
    (or (u0, phi) for the first strip).  Returns (u, E, iterations, last
    criterion value); iterations counts the strip solves."""
    from .norms import h1_norm_nodal
    op = solver.op
    R = op.R
    b = solver.rhs(MU, t0)
    _, E, _ = poisson(op, rho_prev)
    f_prev = constant_in_time(U_prev, R)
    crit = np.inf
    for k in range(1, max_fp + 1):
        install_field(op, prob, E)
        u, _, _ = solver.solve_strip(b)
        rho = density(op, u.reshape(-1, R)[:, 0])          # midpoint: eta_0 = 1, eta_1(1/2) = 0
        _, E_new, _ = poisson(op, rho)
        crit = float(np.abs(E_new - E).max()) + h1_norm_nodal(op, u - f_prev)
        if crit < eps:
            return u, E, k, crit
        E, f_prev = E_new, u
    return u, E, max_fp, crit
