"""Norms of sparse-grid functions: the streamline-diffusion norm of an error
over all strips (Sect. 3, Eq. 11), against the exact solution or against
Table 1's reference (the sparse-grid interpolant of level L + 1 and order
r + 1, Sect. 5.1), and the H^1(J x Omega) norm of one strip function (the
stop test of Algorithm 1, Sect. 4.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

For a discrete solution U (one strip vector per strip) and an exact solution
u, e = U - u and

  |||e|||_delta^2 = sum_j int_{I_j} sigma ||e||^2 + delta ||d_t e + d_beta e||^2
                    + |e|^2_{dOmega} dt
                  + sum_{j<N} ||[e]_j||^2 + ||e_0^+||^2 + ||e_N^-||^2,

with the jump [e]_j = e_j^+ - e_j^-.  The exact solution solves the
homogeneous equation (f = 0), is continuous in time, so

  d_t e + d_beta e = (d_t U + d_beta U) + sigma u  and  [e]_j = [U]_j.

Only domains without a boundary part (every axis periodic) are handled here:
the |e|^2_{dOmega} term is then absent.

Quadrature: the sparse-grid function is represented exactly on the finest
full grid (L, L) (``full_grid_values``); on every pair of finest cells the
collapsed Gauss rule of ``assembly.simplex_rule`` with q points per
direction integrates the squared errors (polynomial parts exactly for q >= 2;
the exact solution's contribution to the error to the rule's accuracy), and
Gauss-Legendre with 2r + 1 points per strip integrates in time (the
polynomial parts of the integrands have degree <= 2r in t).  The spatial
basis is the Lagrange basis of the levels' order (P1, or P2 for r = 2).
"""
from __future__ import annotations

import numpy as np

from .assembly import Factor, gauss01
from .brute import _cell_data
from .mesh import lagrange_basis
from .operator import eta
from .solver import full_grid_values


def _products(prob, X, V, p):
    """beta_p on all (x point, v point) pairs."""
    b = prob.beta[p]
    fx = b.fx(X) if b.fx is not None else np.ones(X.shape[0])
    fv = b.fv(V) if b.fv is not None else np.ones(V.shape[0])
    return b.coef * np.outer(fx, fv)


def _cell_basis(lev, q):
    """Quadrature points and weights per cell, the level's Lagrange basis at
    the points (nq, nloc) and its gradients (nc, nq, nloc, d)."""
    if hasattr(lev, "cell_basis"):        # tensor-product level (oracle/tensor.py)
        return lev.cell_basis(q)
    pts, w, lam, glam = _cell_data(lev, q)
    phi, dphi = lagrange_basis(lev.order, lam)
    grad = np.einsum("qam,cmd->cqad", dphi, glam)
    return pts, w, phi, grad


class _FullGrid:
    """Point values and gradients of finest-full-grid P_r (x) P_r functions on
    every (x cell, v cell) pair's quadrature points."""

    def __init__(self, op, q, periodic_only=True, levels=None):
        L = op.L
        self.op = op
        self.lx, self.lv = (op.hx.levels[L], op.hv.levels[L]) if levels is None else levels
        if periodic_only and any(len(lev.bfaces) for lev in (self.lx, self.lv)):
            raise NotImplementedError("SD-norm errors only on domains without boundary (periodic)")
        self.px, self.wx, self.lamx, self.gx = _cell_basis(self.lx, q)
        self.pv, self.wv, self.lamv, self.gv = _cell_basis(self.lv, q)
        nx, nv = self.px.shape[0], self.pv.shape[0]
        q1, q2 = self.px.shape[1], self.pv.shape[1]
        self.shape = (nx, q1, nv, q2)
        # point coordinates broadcast over pairs
        self.Xp = self.px.reshape(-1, self.px.shape[2])      # (nx q1, d)
        self.Vp = self.pv.reshape(-1, self.pv.shape[2])      # (nv q2, d)
        self.W = np.einsum("ai,bj->aibj", self.wx, self.wv)  # (nx, q1, nv, q2)

    def nodal(self, U):
        """Nodal values on the finest full grid of a spatial sparse-grid vector."""
        return full_grid_values(self.op, U)

    def value(self, F):
        Fc = F[self.lx.cells][:, :, self.lv.cells]           # (nx, nloc, nv, nloc)
        return np.einsum("ia,xayb,jb->xiyj", self.lamx, Fc, self.lamv)

    def grad_x(self, F, axis):
        Fc = F[self.lx.cells][:, :, self.lv.cells]
        return np.einsum("xia,xayb,jb->xiyj", self.gx[..., axis], Fc, self.lamv)

    def grad_v(self, F, axis):
        Fc = F[self.lx.cells][:, :, self.lv.cells]
        return np.einsum("ia,xayb,yjb->xiyj", self.lamx, Fc, self.gv[..., axis])

    def exact(self, fn, t):
        """fn(t, x, v) on every quadrature point pair (d = 1: scalar coordinates)."""
        d = self.Xp.shape[1]
        if d == 1:
            val = fn(t, self.Xp[:, 0][:, None], self.Vp[:, 0][None, :])
        else:
            val = fn(t, self.Xp[:, None, :], self.Vp[None, :, :])
        return np.asarray(val).reshape(self.shape)

    def l2sq(self, vals):
        return float(np.sum(self.W * vals * vals))


def sd_norm_error(prob, op, strips, exact, q: int = 5):
    """|||U - u|||_delta over the strips (Eq. 11).

    strips: the strip solutions u_j (strip vectors, [coefficient][s], s
    fastest), j = 1..N, on strips I_j = ((j-1) dt, j dt); exact(t, x, v):
    the exact solution of the homogeneous problem.  Returns (norm, parts),
    parts = dict of the squared contributions."""
    fg = _FullGrid(op, q)
    d, dt, dl, R = prob.d, prob.dt, prob.delta, op.R
    sig = prob.sigma
    sigma_pts = None
    if sig.coef != 0.0:
        fx = sig.fx(fg.Xp) if sig.fx is not None else np.ones(fg.Xp.shape[0])
        fv = sig.fv(fg.Vp) if sig.fv is not None else np.ones(fg.Vp.shape[0])
        sigma_pts = (sig.coef * np.outer(fx, fv)).reshape(fg.shape)
    beta_pts = [_products(prob, fg.Xp, fg.Vp, p).reshape(fg.shape) for p in range(2 * d)]
    tq, tw = gauss01(2 * prob.r + 1)
    parts = {"sigma": 0.0, "streamline": 0.0, "jumps": 0.0, "initial": 0.0, "final": 0.0}
    prev_end = None
    N = len(strips)
    for j, u in enumerate(strips):
        t0 = j * dt
        us = u.reshape(-1, R)
        F = [fg.nodal(us[:, s]) for s in range(R)]
        val = [fg.value(Fs) for Fs in F]
        dbeta = []
        for s in range(R):
            acc = np.zeros(fg.shape)
            for p in range(2 * d):
                g = fg.grad_x(F[s], p) if p < d else fg.grad_v(F[s], p - d)
                acc = acc + beta_pts[p] * g
            dbeta.append(acc)
        for tau, w in zip(tq, tw):
            e_s = [eta(s, np.array([tau]), dt) for s in range(R)]
            Ut = sum(e_s[s][0][0] * val[s] for s in range(R))
            DU = sum(e_s[s][1][0] * val[s] + e_s[s][0][0] * dbeta[s] for s in range(R))
            ex = fg.exact(exact, t0 + tau * dt)
            if sigma_pts is not None:
                parts["sigma"] += w * dt * float(np.sum(fg.W * sigma_pts * (Ut - ex) ** 2))
                DU = DU + sigma_pts * ex
            parts["streamline"] += w * dt * dl * fg.l2sq(DU)
        e0 = [eta(s, np.array([0.0]), dt)[0][0] for s in range(R)]
        e1 = [eta(s, np.array([1.0]), dt)[0][0] for s in range(R)]
        start = sum(e0[s] * val[s] for s in range(R))
        end = sum(e1[s] * val[s] for s in range(R))
        if j == 0:
            parts["initial"] = fg.l2sq(start - fg.exact(exact, 0.0))
        else:
            parts["jumps"] += fg.l2sq(start - prev_end)
        if j == N - 1:
            parts["final"] = fg.l2sq(end - fg.exact(exact, N * dt))
        prev_end = end
    return float(np.sqrt(sum(parts.values()))), parts


class SparseInterpolant:
    """The interpolant of a function of (x, v) in the sparse grid space of
    level L + 1 with P2 elements (d = 1), written on the P2 full grid
    (L + 1, L + 1): the combination technique, sum over |l| = L + 1 minus sum
    over |l| = L of the full-grid nodal interpolants (exact for
    interpolation, Sect. 4.3)."""

    def __init__(self, prob, L: int):
        from .mesh import P2Hierarchy
        if prob.d != 1:
            raise NotImplementedError("d = 1")
        self.L = L
        self.Hx, self.Hv = P2Hierarchy(prob.mesh_x, L + 1), P2Hierarchy(prob.mesh_v, L + 1)
        self.Ex = [self.Hx.embed(L + 1, l) for l in range(L + 2)]
        self.Ev = [self.Hv.embed(L + 1, l) for l in range(L + 2)]
        self.combos = [(l, L + 1 - l, 1.0) for l in range(L + 2)] + [(l, L - l, -1.0) for l in range(L + 1)]

    def __call__(self, fn, t) -> np.ndarray:
        L = self.L
        acc = np.zeros((self.Hx.levels[L + 1].n, self.Hv.levels[L + 1].n))
        for l1, l2, c in self.combos:
            X, V = self.Hx.levels[l1].coords[:, 0], self.Hv.levels[l2].coords[:, 0]
            acc += c * (self.Ex[l1] @ (self.Ev[l2] @ np.asarray(fn(t, X[:, None], V[None, :])).T).T)
        return acc


def sd_norm_error_interp(prob, op, strips, exact, q: int = 5, dt_fd: float = 1e-6):
    """|||U - I u|||_delta with Table 1's reference (Sect. 5.1): I u is the
    interpolant of the exact solution in the sparse grid space of level
    L + 1 with elements of order r + 1, here in space at every time (d = 1,
    r = 1: ``SparseInterpolant``).  U (P1, level L) and I u are both written
    on the P2 full grid (L + 1, L + 1), where the norm's integrals are taken
    as in ``sd_norm_error``; d_t I u = I d_t u, with d_t u by a central
    difference of step dt_fd."""
    if prob.r != 1 or getattr(prob, "order", 1) != 1 or prob.d != 1:
        raise NotImplementedError("the interpolant reference is built for d = 1, r = 1")
    L, R, d, dt, dl = op.L, op.R, prob.d, prob.dt, prob.delta
    interp = SparseInterpolant(prob, L)
    Hx, Hv = interp.Hx, interp.Hv
    lx, lv = Hx.levels[L + 1], Hv.levels[L + 1]
    fg = _FullGrid(op, q, levels=(lx, lv))
    # a P1 function of level L at the P2 nodes of level L + 1 (the P1
    # vertices of level L + 2): the P1 embedding, on the same canonical order
    Px, Pv = Hx.p1.embed(L + 2, L), Hv.p1.embed(L + 2, L)
    dudt = lambda t, x, v: (exact(t + dt_fd, x, v) - exact(t - dt_fd, x, v)) / (2.0 * dt_fd)
    beta_pts = [_products(prob, fg.Xp, fg.Vp, p).reshape(fg.shape) for p in range(2 * d)]
    sig = prob.sigma
    sigma_pts = None
    if sig.coef != 0.0:
        fx = sig.fx(fg.Xp) if sig.fx is not None else np.ones(fg.Xp.shape[0])
        fv = sig.fv(fg.Vp) if sig.fv is not None else np.ones(fg.Vp.shape[0])
        sigma_pts = (sig.coef * np.outer(fx, fv)).reshape(fg.shape)

    def dbeta(F):
        return sum(beta_pts[p] * (fg.grad_x(F, p) if p < d else fg.grad_v(F, p - d)) for p in range(2 * d))

    tq, tw = gauss01(2 * prob.r + 1)
    parts = {"sigma": 0.0, "streamline": 0.0, "jumps": 0.0, "initial": 0.0, "final": 0.0}
    prev_end = None
    N = len(strips)
    for j, u in enumerate(strips):
        t0 = j * dt
        us = u.reshape(-1, R)
        F = [Px @ full_grid_values(op, us[:, s]) @ Pv.T for s in range(R)]
        val = [fg.value(Fs) for Fs in F]
        db = [dbeta(Fs) for Fs in F]
        for tau, w in zip(tq, tw):
            t = t0 + tau * dt
            e_s = [eta(s, np.array([tau]), dt) for s in range(R)]
            Ut = sum(e_s[s][0][0] * val[s] for s in range(R))
            DU = sum(e_s[s][1][0] * val[s] + e_s[s][0][0] * db[s] for s in range(R))
            Iu = interp(exact, t)
            DI = fg.value(interp(dudt, t)) + dbeta(Iu)
            if sigma_pts is not None:
                parts["sigma"] += w * dt * float(np.sum(fg.W * sigma_pts * (Ut - fg.value(Iu)) ** 2))
                DU = DU + sigma_pts * Ut
                DI = DI + sigma_pts * fg.value(Iu)
            parts["streamline"] += w * dt * dl * fg.l2sq(DU - DI)
        e0 = [eta(s, np.array([0.0]), dt)[0][0] for s in range(R)]
        e1 = [eta(s, np.array([1.0]), dt)[0][0] for s in range(R)]
        start = sum(e0[s] * val[s] for s in range(R))
        end = sum(e1[s] * val[s] for s in range(R))
        if j == 0:
            parts["initial"] = fg.l2sq(start - fg.value(interp(exact, 0.0)))
        else:
            parts["jumps"] += fg.l2sq(start - prev_end)
        if j == N - 1:
            parts["final"] = fg.l2sq(end - fg.value(interp(exact, N * dt)))
        prev_end = end
    return float(np.sqrt(sum(parts.values()))), parts


def h1_terms(op):
    """Kronecker terms of the H^1(J x Omega) Gram form on one strip:
    int_J (v, w) + (d_t v, d_t w) + sum_p (d_p v, d_p w) dt, p over the d
    axes of Omega_x and of Omega_v."""
    from .operator import time_matrices
    Mt, Tt, Ct, Gt = time_matrices(op.prob.dt, op.prob.r)
    d = op.prob.d
    vol = Factor("vol")
    terms = [(Mt + Ct, vol, vol)]
    for p in range(1, d + 1):
        terms.append((Mt, Factor("vol", 1.0, (), p, p), vol))
        terms.append((Mt, vol, Factor("vol", 1.0, (), p, p)))
    return terms


def h1_norm(op, u):
    """||U||_{H^1(J x Omega)} of the strip function with coefficients u: the
    Gram form applied blockwise (rows are test functions, so u . (G u) is
    the form of U with itself)."""
    g = op.apply(u, h1_terms(op))
    return float(np.sqrt(max(float(u @ g), 0.0)))


def h1_norm_nodal(op, u, q: int = 3):
    """The same H^1(J x Omega) norm from the function's unique values on the
    finest full grid (L, L) and quadrature on pairs of finest cells (exact:
    the integrands are polynomials of degree <= 2 per cell and in time).
    Unlike the Gram form of ``h1_norm``, whose value for a nearly vanishing
    function made of large spanning-set coefficients is limited by rounding
    to about sqrt(machine epsilon) times the coefficients' scale, this one
    loses only machine epsilon: the stop test of the fixed point uses it."""
    fg = _FullGrid(op, q, periodic_only=False)
    d, dt, R = op.prob.d, op.prob.dt, op.R
    us = u.reshape(-1, R)
    F = [fg.nodal(us[:, s]) for s in range(R)]
    val = [fg.value(Fs) for Fs in F]
    grads = [[fg.grad_x(Fs, p) for p in range(d)] + [fg.grad_v(Fs, p) for p in range(d)] for Fs in F]
    tq, tw = gauss01(3)
    acc = 0.0
    for tau, w in zip(tq, tw):
        e_s = [eta(s, np.array([tau]), dt) for s in range(R)]
        U = sum(e_s[s][0][0] * val[s] for s in range(R))
        Ut = sum(e_s[s][1][0] * val[s] for s in range(R))
        acc += w * dt * (fg.l2sq(U) + fg.l2sq(Ut))
        for p in range(2 * d):
            G = sum(e_s[s][0][0] * grads[s][p] for s in range(R))
            acc += w * dt * fg.l2sq(G)
    return float(np.sqrt(acc))
