"""Tensor-product Lagrange elements Q_r on box meshes of squares (Sect. 5.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sect. 5.1 builds the meshes of Table 1 from 4^d d-cubes.  On a uniform mesh
of squares the continuous Q_r space is the tensor product of the continuous
P_r spaces of the two axes, nested level by level like them: its nodes are
the products of the axes' nodes (axis 0 fastest, the oracle's canonical
order), its embedding is E_B (x) E_A, and a factor with a constant weight is
the Kronecker product of the two axes' one-dimensional factors (a derivative
on axis p acts on that axis' factor only).  Loads with a general function
and the point evaluations of the norms use the tensor Gauss rule on each
square with the products of the axes' basis functions.

Only what the constant-coefficient periodic problem of Table 1 needs is
here: d = 2, both axes periodic or not, volume factors with constant
weights, loads, point evaluation.  Anything else raises NotImplementedError.
Pinned by tests/test_oracle_tensor.py.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Tuple

import numpy as np
import scipy.sparse as sp

from .assembly import Factor, assemble_level
from .mesh import Hierarchy, P2Hierarchy


@dataclass
class _Interval:
    """A coarse 1-D mesh in the form the hierarchies read."""
    coords: np.ndarray
    cells: np.ndarray
    lo: Tuple[float]
    hi: Tuple[float]
    periodic: Tuple[bool]
    dim: int = 1


def axis_meshes(mesh) -> List[_Interval]:
    """The 1-D meshes of the axes of a box mesh whose vertices form a
    tensor lattice (the squares' corners)."""
    if mesh.dim != 2:
        raise NotImplementedError("tensor-product elements: d = 2 only")
    out = []
    xs = [np.unique(mesh.coords[:, ax]) for ax in range(2)]
    if xs[0].size * xs[1].size != mesh.coords.shape[0]:
        raise ValueError("the mesh vertices are not a tensor lattice")
    for ax in range(2):
        x = xs[ax]
        cells = np.stack([np.arange(x.size - 1), np.arange(1, x.size)], axis=1)
        out.append(_Interval(coords=x[:, None], cells=cells, lo=(mesh.lo[ax],), hi=(mesh.hi[ax],),
                             periodic=(bool(mesh.periodic[ax]),)))
    return out


class TensorLevel:
    """One level of Q_r: the product of level A (axis 0) and level B (axis 1)."""

    def __init__(self, A, B, order: int):
        self.A, self.B, self.order = A, B, order
        xa, xb = A.coords[:, 0], B.coords[:, 0]
        self.coords = np.stack([np.tile(xa, xb.size), np.repeat(xb, xa.size)], axis=1)
        na = A.n
        la, lb = A.cells.shape[1], B.cells.shape[1]
        # square (ca, cb) -> local node (a, b) = A node a of ca, B node b of cb
        self.cells = (A.cells[None, :, :, None] + na * B.cells[:, None, None, :]).reshape(
            A.cells.shape[0] * B.cells.shape[0], la * lb)
        nb_faces = len(A.bfaces) + len(B.bfaces)
        self.bfaces = np.zeros((nb_faces, 1), dtype=np.int64)   # only their count is read

    @property
    def n(self) -> int:
        return self.coords.shape[0]

    def assemble(self, f: Factor) -> sp.csr_matrix:
        if f.kind != "vol" or f.weight or f.restrict:
            raise NotImplementedError("tensor-product factors: volume, constant weight, no restriction")
        if f.test > 2 or f.trial > 2:
            raise NotImplementedError("d = 2")
        ax = lambda k, p: 1 if k == p else 0          # derivative on axis p (1-based) or value
        MA = assemble_level(self.A, Factor("vol", 1.0, (), ax(f.test, 1), ax(f.trial, 1)))
        MB = assemble_level(self.B, Factor("vol", 1.0, (), ax(f.test, 2), ax(f.trial, 2)))
        return (f.coef * sp.kron(MB, MA)).tocsr()

    def cell_basis(self, q: int):
        """Points (nc, nq, 2), weights (nc, nq), basis values (nq, nloc) and
        gradients (nc, nq, nloc, 2) on every square, the tensor products of
        the axes' cell data (squares ordered A fastest, as in ``cells``)."""
        from .norms import _cell_basis
        pa, wa, fa, ga = _cell_basis(self.A, q)
        pb, wb, fb, gb = _cell_basis(self.B, q)
        nca, qa = wa.shape
        ncb, qb = wb.shape
        la, lb = fa.shape[1], fb.shape[1]
        pts = np.empty((ncb, nca, qa, qb, 2))
        pts[..., 0] = pa[None, :, :, None, 0]
        pts[..., 1] = pb[:, None, None, :, 0]
        pts = pts.reshape(nca * ncb, qa * qb, 2)
        w = np.einsum("ai,bj->baij", wa, wb).reshape(nca * ncb, qa * qb)
        phi = np.einsum("ik,jl->ijkl", fa, fb).reshape(qa * qb, la * lb)
        g = np.empty((ncb, nca, qa, qb, la, lb, 2))
        g[..., 0] = np.einsum("aik,jl->aijkl", ga[..., 0], fb)[None]
        g[..., 1] = np.einsum("ik,bjl->bijkl", fa, gb[..., 0])[:, None]
        grad = g.reshape(nca * ncb, qa * qb, la * lb, 2)
        return pts, w, phi, grad

    def load(self, fn, q: int) -> np.ndarray:
        pts, w, phi, _ = self.cell_basis(q)
        nc, nq, _ = pts.shape
        vals = fn(pts.reshape(-1, 2)).reshape(nc, nq) if fn is not None else np.ones((nc, nq))
        fe = np.einsum("cq,cq,qa->ca", vals, w, phi)
        out = np.zeros(self.n)
        np.add.at(out, self.cells.ravel(), fe.ravel())
        return out


class TensorHierarchy(Hierarchy):
    """Levels 0..L of Q_r (r = 1, 2) on a box mesh of squares."""

    def __init__(self, mesh, L: int, order: int):
        self.mesh, self.d, self.L = mesh, 2, L
        H = Hierarchy if order == 1 else P2Hierarchy
        self.axes = [H(m, L) for m in axis_meshes(mesh)]
        A, B = self.axes
        self.levels = [TensorLevel(A.levels[l], B.levels[l], order) for l in range(L + 1)]
        self.E = [sp.kron(B.E[l], A.E[l]).tocsr() for l in range(L)]
