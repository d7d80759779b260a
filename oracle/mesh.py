"""Nested multilevel P1 spaces on uniformly refined simplicial meshes (Sect. 2).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Sect. 2 builds V_1 subset V_2 subset ... by uniform refinement of a coarse
mesh; Sect. 4.2 needs the matrix E of the embedding of a coarse level into a
finer one.  For continuous P1 elements the embedding evaluates the coarse
function at the fine vertices: a fine vertex that is a coarse vertex copies it,
an edge midpoint averages the two edge end points.

Refinement: 1D bisection, 2D red refinement (4 children through the edge
midpoints), 3D regular refinement after Bey (8 children: the four corner
tetrahedra and the inner octahedron cut along the diagonal between the
midpoints of edges 02 and 13), which maps a Kuhn (Freudenthal) tetrahedron
with its vertices in path order onto the Kuhn tetrahedra of the refined
lattice.  Vertex order on every level is canonical: vertices sorted
lexicographically by coordinates, last axis slowest.  Periodic axes identify
the vertex at the upper bound with the one at the lower bound.

Pinned by tests/test_oracle_mesh.py: vertex counts, E 1 = 1, E^T M_fine E =
M_coarse (with an independent exact mass), nestedness of the embeddings.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Dict, List, Tuple

import numpy as np
import scipy.sparse as sp


@dataclass
class Level:
    coords: np.ndarray        # (n, d) canonical order (master vertices only)
    cells: np.ndarray         # (nc, d+1) indices into coords
    cell_coords: np.ndarray   # (nc, d+1, d) unwrapped geometric vertex coords
    bfaces: np.ndarray        # (nf, d) indices into coords
    bface_coords: np.ndarray  # (nf, d, d) geometric coords of the face vertices
    bface_axis: np.ndarray    # (nf,) axis of the outward normal
    bface_side: np.ndarray    # (nf,) -1 (lower bound) or +1 (upper bound)
    order: int = 1            # polynomial order of the continuous Lagrange space

    @property
    def n(self) -> int:
        return self.coords.shape[0]


def lagrange_nodes(k: int, order: int) -> np.ndarray:
    """Barycentric coordinates (nloc, k) of the local nodes of the Lagrange
    element of order 1 or 2 on a simplex with k vertices: the vertices, then
    (order 2) the edge midpoints (i, j), i < j, in lexicographic order."""
    rows = [np.eye(k)[i] for i in range(k)]
    if order == 2:
        rows += [0.5 * (np.eye(k)[i] + np.eye(k)[j]) for i in range(k) for j in range(i + 1, k)]
    return np.array(rows)


def lagrange_basis(order: int, lam: np.ndarray):
    """Values phi (nq, nloc) and barycentric derivatives dphi (nq, nloc, k)
    (d phi_a / d lam_m) of the Lagrange basis of order 1 or 2 at points with
    barycentric coordinates lam (nq, k), nodes as in ``lagrange_nodes``.
    Order 2: lam_i (2 lam_i - 1) at vertex i, 4 lam_i lam_j at edge (i, j)."""
    nq, k = lam.shape
    if order == 1:
        return lam.copy(), np.broadcast_to(np.eye(k), (nq, k, k)).copy()
    edges = [(i, j) for i in range(k) for j in range(i + 1, k)]
    phi = np.empty((nq, k + len(edges)))
    dphi = np.zeros((nq, k + len(edges), k))
    for i in range(k):
        phi[:, i] = lam[:, i] * (2.0 * lam[:, i] - 1.0)
        dphi[:, i, i] = 4.0 * lam[:, i] - 1.0
    for e, (i, j) in enumerate(edges):
        phi[:, k + e] = 4.0 * lam[:, i] * lam[:, j]
        dphi[:, k + e, i] = 4.0 * lam[:, j]
        dphi[:, k + e, j] = 4.0 * lam[:, i]
    return phi, dphi


def _refine_raw(coords: np.ndarray, cells: np.ndarray):
    """Uniform refinement of an (unidentified) mesh.  Returns fine coords,
    fine cells and for every fine vertex its parent pair (a, b) (a == b for a
    vertex that already was a coarse vertex)."""
    d = coords.shape[1]
    nv = coords.shape[0]
    mid: Dict[Tuple[int, int], int] = {}
    new_coords = [c for c in coords]
    parents = [(i, i) for i in range(nv)]

    def m(a: int, b: int) -> int:
        key = (min(a, b), max(a, b))
        if key not in mid:
            mid[key] = len(new_coords)
            new_coords.append(0.5 * (coords[a] + coords[b]))
            parents.append(key)
        return mid[key]

    out = []
    for c in cells:
        if d == 1:
            a, b = c
            mab = m(a, b)
            out += [[a, mab], [mab, b]]
        elif d == 2:
            a, b, cc = c
            mab, mbc, mca = m(a, b), m(b, cc), m(cc, a)
            out += [[a, mab, mca], [mab, b, mbc], [mca, mbc, cc], [mab, mbc, mca]]
        elif d == 3:
            x0, x1, x2, x3 = c
            m01, m02, m03 = m(x0, x1), m(x0, x2), m(x0, x3)
            m12, m13, m23 = m(x1, x2), m(x1, x3), m(x2, x3)
            out += [[x0, m01, m02, m03], [m01, x1, m12, m13], [m02, m12, x2, m23], [m03, m13, m23, x3],
                    [m01, m02, m03, m13], [m01, m02, m12, m13], [m02, m03, m13, m23], [m02, m12, m13, m23]]
        else:
            raise NotImplementedError("oracle refinement supports d = 1, 2, 3")
    return np.array(new_coords), np.array(out, dtype=np.int64), parents


def _faces_of(cells: np.ndarray) -> np.ndarray:
    d1 = cells.shape[1]
    fs = []
    for c in cells:
        for drop in range(d1):
            fs.append(tuple(sorted(int(x) for k, x in enumerate(c) if k != drop)))
    return fs


def _identify(coords: np.ndarray, lo, hi, periodic):
    """Map every raw vertex to a master raw vertex (periodic identification)."""
    key_of = {}
    wrapped = []
    for i, x in enumerate(coords):
        y = x.copy()
        for ax in range(coords.shape[1]):
            if periodic[ax] and y[ax] == hi[ax]:
                y[ax] = lo[ax]
        k = tuple(y.tolist())
        wrapped.append(k)
        if k == tuple(x.tolist()):       # a master: already on the lower bound side
            key_of[k] = i
    rep = np.array([key_of[k] for k in wrapped], dtype=np.int64)
    return rep


class Hierarchy:
    """Levels 0..L of uniformly refined meshes with canonical vertex order."""

    def __init__(self, mesh, L: int):
        self.mesh = mesh
        self.d = mesh.dim
        self.L = L
        raw_coords = [np.asarray(mesh.coords, dtype=np.float64)]
        raw_cells = [np.asarray(mesh.cells, dtype=np.int64)]
        raw_parents = [None]
        for _ in range(L):
            c, e, p = _refine_raw(raw_coords[-1], raw_cells[-1])
            raw_coords.append(c)
            raw_cells.append(e)
            raw_parents.append(p)

        self.levels: List[Level] = []
        self._raw2can: List[np.ndarray] = []
        for l in range(L + 1):
            self._build_level(raw_coords[l], raw_cells[l])
        # embeddings E_{l+1 <- l}
        self.E: List[sp.csr_matrix] = []
        for l in range(L):
            self.E.append(self._embedding(l, raw_parents[l + 1]))

    def _build_level(self, rc: np.ndarray, rcells: np.ndarray):
        m = self.mesh
        rep = _identify(rc, m.lo, m.hi, m.periodic)
        masters = np.unique(rep)
        mc = rc[masters]
        order = np.lexsort(tuple(mc[:, ax] for ax in range(self.d)))
        can_of_master = np.empty(rc.shape[0], dtype=np.int64)
        can_of_master[masters[order]] = np.arange(masters.size)
        raw2can = can_of_master[rep]
        coords = mc[order]
        cells = raw2can[rcells]
        cell_coords = rc[rcells]
        # boundary faces: faces of exactly one cell, not on a periodic side
        counts: Dict[tuple, int] = {}
        for f in _faces_of(rcells):
            counts[f] = counts.get(f, 0) + 1
        bf, bfc, bax, bsd = [], [], [], []
        for f, cnt in counts.items():
            if cnt != 1:
                continue
            fc = rc[list(f)]
            found = False
            for ax in range(self.d):
                for side, bound in ((-1, m.lo[ax]), (+1, m.hi[ax])):
                    if np.all(fc[:, ax] == bound):
                        found = True
                        if not m.periodic[ax]:
                            bf.append(raw2can[list(f)])
                            bfc.append(fc)
                            bax.append(ax)
                            bsd.append(side)
            if not found:
                raise ValueError("boundary face not on a box side")
        self._raw2can.append(raw2can)
        self.levels.append(Level(
            coords=coords, cells=cells, cell_coords=cell_coords,
            bfaces=np.array(bf, dtype=np.int64).reshape(-1, self.d),
            bface_coords=np.array(bfc, dtype=np.float64).reshape(-1, self.d, self.d),
            bface_axis=np.array(bax, dtype=np.int64), bface_side=np.array(bsd, dtype=np.int64)))

    def _embedding(self, l: int, parents) -> sp.csr_matrix:
        """E_{l+1<-l}: nodal values on level l+1 of the level-l basis functions."""
        nf, nc = self.levels[l + 1].n, self.levels[l].n
        r2c_f, r2c_c = self._raw2can[l + 1], self._raw2can[l]
        E = sp.lil_matrix((nf, nc))
        done = np.zeros(nf, dtype=bool)
        for raw_f, (a, b) in enumerate(parents):
            i = r2c_f[raw_f]
            if done[i]:
                continue
            done[i] = True
            if a == b:
                E[i, r2c_c[a]] = 1.0
            else:
                E[i, r2c_c[a]] += 0.5
                E[i, r2c_c[b]] += 0.5
        assert done.all()
        return E.tocsr()

    def embed(self, lf: int, lc: int) -> sp.csr_matrix:
        """E_{lf <- lc} = E_{lf<-lf-1} ... E_{lc+1<-lc} (identity if lf == lc)."""
        M = sp.identity(self.levels[lc].n, format="csr")
        for l in range(lc, lf):
            M = (self.E[l] @ M).tocsr()
        return M


class P2Hierarchy(Hierarchy):
    """Levels 0..L of continuous P2 spaces on the same meshes (Sect. 2 with
    r = 2).  Uniform refinement puts the new vertices at the edge midpoints,
    so the P2 nodes of level l are the vertices of level l + 1: a P1
    hierarchy with L + 1 refinements supplies the node coordinates and their
    canonical order.  Cells keep the geometry of level l and list their six
    (d = 2) or three (d = 1) nodes in the order of ``lagrange_nodes``; the
    embedding evaluates the coarse basis at the fine nodes, which in every
    coarse cell are the points with barycentric coordinates in (1/4) Z."""

    def __init__(self, mesh, L: int):
        self.mesh = mesh
        self.d = mesh.dim
        self.L = L
        self.p1 = Hierarchy(mesh, L + 1)
        self._index = [self._node_index(self.p1.levels[l + 1].coords) for l in range(L + 1)]
        self.levels: List[Level] = [self._p2_level(l) for l in range(L + 1)]
        self.E: List[sp.csr_matrix] = [self._p2_embedding(l) for l in range(L)]

    def _key(self, x: np.ndarray) -> tuple:
        m = self.mesh
        lo, hi = np.asarray(m.lo, dtype=np.float64), np.asarray(m.hi, dtype=np.float64)
        y = np.array(x, dtype=np.float64)
        for ax in range(self.d):
            if m.periodic[ax] and y[ax] == hi[ax]:
                y[ax] = lo[ax]
        # box-relative coordinates on a 2^40 lattice: dyadic node positions
        # are integers there, rounding absorbs the midpoints' last bits
        return tuple(np.round((y - lo) / (hi - lo) * 2.0 ** 40).astype(np.int64).tolist())

    def _node_index(self, coords: np.ndarray) -> Dict[tuple, int]:
        return {self._key(x): i for i, x in enumerate(coords)}

    def _lookup(self, l: int, pts: np.ndarray) -> np.ndarray:
        idx = self._index[l]
        flat = pts.reshape(-1, self.d)
        return np.array([idx[self._key(x)] for x in flat], dtype=np.int64).reshape(pts.shape[:-1])

    def _p2_level(self, l: int) -> Level:
        geo = self.p1.levels[l]
        k = self.d + 1
        bary = lagrange_nodes(k, 2)
        cells = self._lookup(l, np.einsum("ak,ckd->cad", bary, geo.cell_coords))
        if geo.bface_coords.shape[0]:
            fb = lagrange_nodes(self.d, 2)
            bfaces = self._lookup(l, np.einsum("ak,fkd->fad", fb, geo.bface_coords))
        else:
            bfaces = np.zeros((0, lagrange_nodes(self.d, 2).shape[0]), dtype=np.int64)
        return Level(coords=self.p1.levels[l + 1].coords, cells=cells, cell_coords=geo.cell_coords,
                     bfaces=bfaces, bface_coords=geo.bface_coords, bface_axis=geo.bface_axis,
                     bface_side=geo.bface_side, order=2)

    def _p2_embedding(self, l: int) -> sp.csr_matrix:
        """E_{l+1<-l}: the level-l P2 basis at the level-(l+1) P2 nodes."""
        k = self.d + 1
        coarse = self.levels[l]
        ticks = [np.array(c) / 4.0 for c in np.ndindex(*([5] * k)) if sum(c) == 4]
        lam = np.array(ticks)                                     # fine nodes of one coarse cell
        phi, _ = lagrange_basis(2, lam)
        fine = self._lookup(l + 1, np.einsum("pk,ckd->cpd", lam, coarse.cell_coords))   # (nc, np)
        entries: Dict[Tuple[int, int], float] = {}
        for c in range(coarse.cells.shape[0]):
            for p in range(lam.shape[0]):
                for a in range(phi.shape[1]):
                    if phi[p, a] != 0.0:
                        entries[(int(fine[c, p]), int(coarse.cells[c, a]))] = float(phi[p, a])
        rows, cols = zip(*entries.keys())
        E = sp.csr_matrix((list(entries.values()), (rows, cols)),
                          shape=(self.levels[l + 1].n, coarse.n))
        return E
