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

    @property
    def n(self) -> int:
        return self.coords.shape[0]


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
