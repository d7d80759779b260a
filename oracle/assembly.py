"""Finest-level FE factor matrices and their Galerkin projection (Sect. 4.2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sect. 4.2 reduces every 2d-dimensional matrix of the method to sums of
Kronecker products of d-dimensional factors (P1 matrices on Omega_x and
Omega_v), computed once on the finest level and carried to coarser levels by
the embedding:  X_{l,l'} = E_{L<-l}^T X_{L,L} E_{L<-l'}.

A factor is the bilinear form
    X[i, j] = int  w(y) * (D_trial phi_j)(y) * (D_test phi_i)(y)  dy
(row i = test function, column j = trial function), D_0 = value and
D_p = d/dy_p (1-based axis p), over the domain (``kind='vol'``) or over the
boundary faces on one box side (``kind='face'``).  The weight w is a constant
times a product of coefficient functions.  A sign restriction keeps only the
cells (faces) where a given function has a given sign, evaluated at the cell
(face) centroid: this splits the inflow boundary (Sect. 5.2) exactly when the
sign changes on mesh lines.

Quadrature: Gauss-Legendre with q points per direction on [0,1], collapsed
(Duffy) onto the simplex; exact for polynomial integrands of degree 2q-2 on
triangles and 2q-1 on intervals.  The basis is the Lagrange basis of the
level's order (P1, or P2 for r = 2); P2 gradients vary inside a cell and are
formed from the barycentric derivatives by the chain rule.

Pinned by tests/test_oracle_assembly.py: mass row sums = int phi_k, total
mass = |Omega|, Green's identity D_p + D_p^T = face masses (Sect. 3, proof of
the stability lemma), polynomial weights against closed forms, projection
against direct assembly on the coarse level.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, Tuple

import numpy as np
import scipy.sparse as sp

from .mesh import Hierarchy, Level, lagrange_basis

QUAD_Q = 4  # Gauss-Legendre points per collapsed direction


def gauss01(q: int):
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (x + 1.0), 0.5 * w


def simplex_rule(d: int, q: int = QUAD_Q):
    """Collapsed Gauss rule on the reference simplex {xi >= 0, sum xi <= 1}."""
    g, w = gauss01(q)
    if d == 0:
        return np.zeros((1, 0)), np.ones(1)
    if d == 1:
        return g[:, None], w
    if d == 2:
        a, b = np.meshgrid(g, g, indexing="ij")
        wa, wb = np.meshgrid(w, w, indexing="ij")
        pts = np.stack([a.ravel(), (b * (1 - a)).ravel()], axis=1)
        return pts, (wa * wb * (1 - a)).ravel()
    if d == 3:
        a, b, c = np.meshgrid(g, g, g, indexing="ij")
        wa, wb, wc = np.meshgrid(w, w, w, indexing="ij")
        pts = np.stack([a.ravel(), (b * (1 - a)).ravel(), (c * (1 - a) * (1 - b)).ravel()], axis=1)
        return pts, (wa * wb * wc * (1 - a) ** 2 * (1 - b)).ravel()
    raise NotImplementedError


@dataclass(frozen=True)
class Factor:
    kind: str                                   # 'vol' or 'face'
    coef: float = 1.0
    weight: Tuple[Callable, ...] = ()           # product of functions of y
    test: int = 0
    trial: int = 0
    restrict: Tuple = ()                        # ((fn, coef, sign), ...)
    face: Tuple[int, int] = (-1, 0)             # (axis, side) for kind == 'face'


class CellField:
    """A function that is constant on every cell of the finest level (values in
    the order of ``Level.cells``); used for the electric field of Sect. 5.3."""

    def __init__(self, values: np.ndarray):
        self.values = np.asarray(values, dtype=np.float64)


def _weight(f: Factor, pts: np.ndarray, nq: int = 1) -> np.ndarray:
    w = np.full(pts.shape[0], float(f.coef))
    for fn in f.weight:
        w = w * (np.repeat(fn.values, nq) if isinstance(fn, CellField) else fn(pts))
    return w


def _keep(f: Factor, centroids: np.ndarray) -> np.ndarray:
    keep = np.ones(centroids.shape[0], dtype=bool)
    for fn, c, s in f.restrict:
        vals = fn.values if isinstance(fn, CellField) else fn(centroids)
        keep &= (s * c * vals) > 0.0
    return keep


def assemble_level(lev: Level, f: Factor, q: int = QUAD_Q) -> sp.csr_matrix:
    if hasattr(lev, "assemble"):          # tensor-product level (oracle/tensor.py)
        return lev.assemble(f)
    n = lev.n
    if f.kind == "vol":
        cc = lev.cell_coords
        nc, d1, d = cc.shape
        keep = _keep(f, cc.mean(axis=1))
        cc, cells = cc[keep], lev.cells[keep]
        if cc.shape[0] == 0:
            return sp.csr_matrix((n, n))
        if any(isinstance(fn, CellField) for fn in f.weight):
            f = Factor(f.kind, f.coef, tuple(CellField(fn.values[keep]) if isinstance(fn, CellField) else fn
                                            for fn in f.weight), f.test, f.trial, (), f.face)
        v0 = cc[:, 0, :]
        J = np.transpose(cc[:, 1:, :] - v0[:, None, :], (0, 2, 1))   # columns = edges
        det = np.abs(np.linalg.det(J))
        Jinv = np.linalg.inv(J)
        rp, rw = simplex_rule(d, q)
        pts = v0[:, None, :] + np.einsum("cij,qj->cqi", J, rp)      # (nc, nq, d)
        lam = np.concatenate([1.0 - rp.sum(axis=1, keepdims=True), rp], axis=1)  # (nq, d+1)
        gref = np.vstack([-np.ones((1, d)), np.eye(d)])              # (d+1, d)
        gphys = np.einsum("cji,kj->cki", Jinv, gref)                 # (nc, d+1, d): grad lam_k
        wt = _weight(f, pts.reshape(-1, d), rp.shape[0]).reshape(pts.shape[0], -1)
        wq = wt * rw[None, :] * det[:, None]                          # (nc, nq)
        phi, dphi = lagrange_basis(lev.order, lam)                    # (nq, nloc), (nq, nloc, d+1)
        nloc = phi.shape[1]

        def D(a):
            if a == 0:
                return np.broadcast_to(phi[None, :, :], (cc.shape[0],) + phi.shape)
            if lev.order == 1:
                return np.broadcast_to(gphys[:, None, :, a - 1], (cc.shape[0], rp.shape[0], d1))
            # grad phi = sum_m (d phi / d lam_m) grad lam_m
            return np.einsum("qam,cm->cqa", dphi, gphys[:, :, a - 1])

        Ke = np.einsum("cq,cqi,cqj->cij", wq, D(f.test), D(f.trial))
        rows = np.repeat(cells, nloc, axis=1).ravel()
        cols = np.tile(cells, (1, nloc)).ravel()
        return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()

    # boundary faces on one side
    ax, side = f.face
    sel = (lev.bface_axis == ax) & (lev.bface_side == side)
    fc, faces = lev.bface_coords[sel], lev.bfaces[sel]
    keep = _keep(f, fc.mean(axis=1)) if fc.shape[0] else np.zeros(0, dtype=bool)
    fc, faces = fc[keep], faces[keep]
    if fc.shape[0] == 0:
        return sp.csr_matrix((n, n))
    nf, dv, d = fc.shape
    rp, rw = simplex_rule(dv - 1, q)
    f0 = fc[:, 0, :]
    Jf = np.transpose(fc[:, 1:, :] - f0[:, None, :], (0, 2, 1))      # (nf, d, d-1)
    if dv - 1 == 0:
        meas = np.ones(nf)
    else:
        meas = np.sqrt(np.abs(np.linalg.det(np.einsum("fki,fkj->fij", Jf, Jf))))
    pts = f0[:, None, :] + np.einsum("fij,qj->fqi", Jf, rp)
    lam = np.concatenate([1.0 - rp.sum(axis=1, keepdims=True), rp], axis=1)   # (nq, dv)
    wt = _weight(f, pts.reshape(-1, d)).reshape(nf, -1)
    wq = wt * rw[None, :] * meas[:, None]
    phi, _ = lagrange_basis(lev.order, lam)                                  # face basis (nq, nfloc)
    Ke = np.einsum("fq,qi,qj->fij", wq, phi, phi)
    rows = np.repeat(faces, phi.shape[1], axis=1).ravel()
    cols = np.tile(faces, (1, phi.shape[1])).ravel()
    return sp.coo_matrix((Ke.ravel(), (rows, cols)), shape=(n, n)).tocsr()


class FactorStore:
    """Finest-level assembly + Galerkin projection X_{l,l'} (Sect. 4.2)."""

    def __init__(self, hier: Hierarchy):
        self.h = hier
        self._fine = {}
        self._proj = {}
        self._emb = {}

    def embed(self, l: int) -> sp.csr_matrix:
        if l not in self._emb:
            self._emb[l] = self.h.embed(self.h.L, l)
        return self._emb[l]

    def fine(self, f: Factor) -> sp.csr_matrix:
        if f not in self._fine:
            self._fine[f] = assemble_level(self.h.levels[self.h.L], f)
        return self._fine[f]

    def proj(self, f: Factor, l: int, lp: int) -> sp.csr_matrix:
        key = (f, l, lp)
        if key not in self._proj:
            self._proj[key] = (self.embed(l).T @ self.fine(f) @ self.embed(lp)).tocsr()
        return self._proj[key]

    def test_row(self, f: Factor, l: int, k: int) -> sp.csr_matrix:
        """Row k of E_{L<-l}^T X_L (1 x n_L): the factor's bilinear form with
        the level-l test function k written in the finest basis."""
        if ("csc", l) not in self._emb:
            self._emb[("csc", l)] = self.embed(l).tocsc()
        return (self._emb[("csc", l)][:, [k]].T @ self.fine(f)).tocsr()

    def proj_row(self, row: sp.csr_matrix, lp: int) -> sp.csr_matrix:
        """Row k of X_{l,l'} from test_row(f, l, k): times E_{L<-l'}."""
        return (row @ self.embed(lp)).tocsr()


def assemble_load_grad(lev: Level, fn, axis: int, q: int = QUAD_Q) -> np.ndarray:
    """F[i] = int fn(y) (d/dy_axis phi_i)(y) dy on one level (fn=None: 1);
    axis is 0-based.  The gradient of a barycentric function is constant on
    a cell: grad lam = J^{-T} grad_ref lam."""
    cc = lev.cell_coords
    nc, d1, d = cc.shape
    v0 = cc[:, 0, :]
    J = np.transpose(cc[:, 1:, :] - v0[:, None, :], (0, 2, 1))     # J[c] columns: edge vectors
    det = np.abs(np.linalg.det(J))
    Jinv = np.linalg.inv(J)
    gref = np.concatenate([-np.ones((1, d)), np.eye(d)], axis=0)    # (d1, d): reference gradients
    grad = np.einsum("ad,cdk->cak", gref, Jinv)                    # (nc, d1, d) physical gradients
    rp, rw = simplex_rule(d, q)
    pts = v0[:, None, :] + np.einsum("cij,qj->cqi", J, rp)
    vals = fn(pts.reshape(-1, d)).reshape(nc, -1) if fn is not None else np.ones((nc, rp.shape[0]))
    if lev.order == 1:
        integ = np.einsum("cq,q,c->c", vals, rw, det)              # int fn over the cell
        fe = integ[:, None] * grad[:, :, axis]
    else:
        lam = np.concatenate([1.0 - rp.sum(axis=1, keepdims=True), rp], axis=1)
        _, dphi = lagrange_basis(lev.order, lam)
        G = np.einsum("qam,cm->cqa", dphi, grad[:, :, axis])        # d phi_a / dy_axis at the points
        fe = np.einsum("cq,q,c,cqa->ca", vals, rw, det, G)
    out = np.zeros(lev.n)
    np.add.at(out, lev.cells.ravel(), fe.ravel())
    return out


def assemble_load(lev: Level, fn, q: int = QUAD_Q) -> np.ndarray:
    """Load vector F[i] = int fn(y) phi_i(y) dy on one level (fn=None: 1)."""
    if hasattr(lev, "load"):              # tensor-product level (oracle/tensor.py)
        return lev.load(fn, q)
    cc = lev.cell_coords
    nc, d1, d = cc.shape
    v0 = cc[:, 0, :]
    J = np.transpose(cc[:, 1:, :] - v0[:, None, :], (0, 2, 1))
    det = np.abs(np.linalg.det(J))
    rp, rw = simplex_rule(d, q)
    pts = v0[:, None, :] + np.einsum("cij,qj->cqi", J, rp)
    lam = np.concatenate([1.0 - rp.sum(axis=1, keepdims=True), rp], axis=1)
    phi, _ = lagrange_basis(lev.order, lam)
    vals = fn(pts.reshape(-1, d)).reshape(nc, -1) if fn is not None else np.ones((nc, rp.shape[0]))
    fe = np.einsum("cq,q,c,qi->ci", vals, rw, det, phi)
    out = np.zeros(lev.n)
    np.add.at(out, lev.cells.ravel(), fe.ravel())
    return out
