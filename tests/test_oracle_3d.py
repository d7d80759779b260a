"""Pins of the oracle's d = 3 path (6-D phase space; Sect. 2 and Table 1's
d = 3 rows, config "d=3 (6D)").

* Kuhn meshes under regular (Bey) refinement: (2^l + 1)^3 vertices and 6 8^l
  tetrahedra on level l of the unit cube, every tetrahedron of volume h^3/6
  whose vertices, ordered by coordinate sum, step by +h along the three axes
  in some order (the Kuhn lattice of the refined grid), 12 4^l boundary
  triangles;
* embeddings: partition of unity and reproduction of linear functions;
* factor matrices: total mass |Omega|, row sums = int phi_k, Green's identity
  D_p + D_p^T = signed face mass (Sect. 3), closed-form moments of
  polynomial weights, Galerkin projection = coarse assembly;
* the Kronecker block formula against a literal 6-D assembly of the weak form
  (Sect. 2, Eq. 5) at L = 1, all blocks, and the energy identity (Sect. 3);
* Table 1's d = 3 dof column: the rank of the spanning set's Gram matrix at
  L = 1 and, beyond, the count sum_l n(l) n(L - l) - sum_l n(l) n(L - 1 - l)
  with the periodic vertex counts n(l) = 64 8^l (checked on the meshes up to
  level 2).
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import sgdg_workloads as W
from oracle.assembly import Factor, assemble_level, assemble_load
from oracle.brute import energy_terms, full_matrix
from oracle.mesh import Hierarchy
from oracle.operator import SparseGridOperator

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.mark.parametrize("L", [0, 1, 2])
def test_kuhn_refinement(L):
    h = Hierarchy(W.cube_mesh(0, 1, 1), L)
    lev = h.levels[L]
    hh = 2.0 ** -L
    assert [lv.n for lv in h.levels] == [(2 ** l + 1) ** 3 for l in range(L + 1)]
    assert lev.cells.shape[0] == 6 * 8 ** L and lev.bfaces.shape[0] == 12 * 4 ** L
    cc = lev.cell_coords
    vol = np.abs(np.linalg.det(cc[:, 1:, :] - cc[:, :1, :])) / 6
    assert np.allclose(vol, hh ** 3 / 6, rtol=1e-13)
    for t in cc:
        steps = np.diff(t[np.argsort(t.sum(axis=1))], axis=0) / hh
        assert np.allclose(np.sort(np.abs(steps).argmax(axis=1)), [0, 1, 2])
        assert np.allclose(steps.sum(axis=1), 1.0) and np.all(steps > -1e-12)


@pytest.mark.parametrize("mesh", [W.cube_mesh(-1, 1, 1), W.cube_mesh(0, 1, 2, periodic=True)], ids=["box", "periodic"])
def test_embedding_partition_of_unity_and_linear(mesh):
    h = Hierarchy(mesh, 2)
    for l in range(2):
        E = h.E[l]
        assert np.allclose(E @ np.ones(E.shape[1]), 1.0, atol=0, rtol=0)
        if not any(mesh.periodic):
            for ax in range(3):
                assert np.array_equal(E @ h.levels[l].coords[:, ax], h.levels[l + 1].coords[:, ax])


def test_factor_matrices_3d():
    h = Hierarchy(W.cube_mesh(-1, 1, 1), 2)
    lev = h.levels[2]
    one = np.ones(lev.n)
    M = assemble_level(lev, Factor("vol"))
    assert abs(M.sum() - 8.0) < 1e-13
    assert np.allclose(M @ one, assemble_load(lev, None), rtol=1e-14, atol=1e-16)
    sq = lambda p: p[:, 2] ** 2
    assert abs(one @ assemble_level(lev, Factor("vol", 1.0, (sq,))) @ one - 8.0 / 3.0) < 1e-13
    for p in (1, 2, 3):
        D = assemble_level(lev, Factor("vol", 1.0, (), 0, p))
        G = sum(side * assemble_level(lev, Factor("face", 1.0, face=(p - 1, side))) for side in (-1, 1))
        assert abs(D + D.T - G).max() < 1e-14
        assert np.allclose(D @ lev.coords[:, p - 1], assemble_load(lev, None), atol=1e-14)
        S = assemble_level(lev, Factor("vol", 1.0, (), p, p))
        assert abs(lev.coords[:, p - 1] @ S @ lev.coords[:, p - 1] - 8.0) < 1e-13
    v1 = lambda p: p[:, 0]
    for f in [Factor("vol"), Factor("vol", 1.0, (v1,), 0, 3), Factor("face", 1.0, (v1,), face=(2, 1))]:
        E = h.embed(2, 0)
        assert abs(E.T @ assemble_level(lev, f) @ E - assemble_level(h.levels[0], f)).max() < 1e-14


def _blocks_vs_brute(prob):
    op = SparseGridOperator(prob)
    L, R = prob.L, op.R
    Af = full_matrix(prob, L, L)
    err, scale = 0.0, 0.0
    for (l1, l2) in op.grids:
        Pm = sp.kron(sp.kron(op.hx.embed(L, l1), op.hv.embed(L, l2)), sp.identity(R)).tocsr()
        for (m1, m2) in op.grids:
            Pp = sp.kron(sp.kron(op.hx.embed(L, m1), op.hv.embed(L, m2)), sp.identity(R)).tocsr()
            Ab = Pm.T @ (Pp.T @ Af.T).T
            n1, n2 = op.grid_shape(m1, m2)
            Ak = np.zeros_like(Ab)
            for c in range(n1 * n2 * R):
                e = np.zeros(n1 * n2 * R)
                e[c] = 1.0
                Ak[:, c] = op.apply_block(op.terms, (l1, l2), (m1, m2), e.reshape(n1, n2, R)).ravel()
            err = max(err, np.abs(Ab - Ak).max())
            scale = max(scale, np.abs(Ab).max())
    return err / scale


def test_block_formula_vs_brute_force_3d():
    prob = W.transport_3d(L=1)
    prob.sigma = W.Product(0.2)
    assert _blocks_vs_brute(prob) < 1e-13


def test_energy_identity_3d():
    prob = W.transport_3d(L=1)
    op = SparseGridOperator(prob)
    L, R = prob.L, op.R
    u = np.random.default_rng(4).uniform(-1, 1, op.size)
    ufull = np.zeros(op.hx.levels[L].n * op.hv.levels[L].n * R)
    for i, (l1, l2) in enumerate(op.grids):
        ufull += sp.kron(sp.kron(op.hx.embed(L, l1), op.hv.embed(L, l2)), sp.identity(R)) @ op.block(u, i).ravel()
    assert abs(u @ op.apply(u) - energy_terms(prob, L, L, ufull)) < 1e-12 * abs(energy_terms(prob, L, L, ufull))


def test_table1_dof_d3():
    rows = []
    with open(os.path.join(GOLDEN, "table1_dof.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#") and line.split()[0] == "3":
                rows.append((int(line.split()[1]), int(line.split()[2])))
    assert rows
    h = Hierarchy(W.cube_mesh(0, 1, 4, periodic=True), 2)
    n = [lv.n for lv in h.levels]
    assert n == [64 * 8 ** l for l in range(3)]
    cnt = lambda l: 64 * 8 ** l
    for Lp, dof in rows:
        L = Lp - 1
        formula = sum(cnt(l) * cnt(L - l) for l in range(L + 1)) - sum(cnt(l) * cnt(L - 1 - l) for l in range(L))
        assert formula == dof, (Lp, formula, dof)
    # L = 1 (paper's): one full grid; the Gram matrix of the spanning set has full rank
    prob = W.Problem(name="dof3", d=3, mesh_x=W.cube_mesh(0, 1, 4, periodic=True),
                     mesh_v=W.cube_mesh(0, 1, 4, periodic=True), L=0, r=0, dt=1.0, delta=0.0, n_strips=1,
                     beta=[W.Product(0.0)] * 6, sigma=W.Product(0.0), u0=[])
    op = SparseGridOperator(prob)
    G = op.dense(op.mass_terms())
    ev = np.linalg.eigvalsh(0.5 * (G + G.T))
    assert int(np.sum(ev > 1e-10 * ev.max())) == rows[0][1] == 4096


def kuhn_hat_integrals(l: int, edge: float) -> np.ndarray:
    """int phi_k over the level-l Kuhn lattice of a cube of edge `edge` (the
    6-tetrahedron coarse mesh refined l times) for every vertex k in
    lexicographic order, last axis slowest.  Each of the cubes of side
    h = edge / 2^l holds 6 tetrahedra of volume h^3 / 6 around its main
    diagonal: its two diagonal corners touch all 6, the other corners 2; a
    hat function integrates to a quarter of the volume of every tetrahedron
    it lives on, so int phi_k = h^3 n_k / 24 with n_k the tetrahedra around k."""
    m = 2 ** l
    h = edge / m
    i = np.arange(m + 1)
    K, J, I = np.meshgrid(i, i, i, indexing="ij")
    n = np.zeros(K.shape)
    for o in [(a, b, c) for a in (0, 1) for b in (0, 1) for c in (0, 1)]:
        ci, cj, ck = I - o[0], J - o[1], K - o[2]
        ok = (ci >= 0) & (ci < m) & (cj >= 0) & (cj < m) & (ck >= 0) & (ck < m)
        n += ok * (6 if o in ((0, 0, 0), (1, 1, 1)) else 2)
    return (h ** 3 * n / 24.0).ravel()


def test_kuhn_hat_integrals():
    """The closed form above against the oracle's projected mass rows (every
    level of an L = 3 hierarchy, both boxes of the d = 3 workload); the GPU
    tests use it at L = 7, where the oracle cannot assemble."""
    for lo, hi in ((0.0, 1.0), (-1.0, 1.0)):
        H = Hierarchy(W.cube_mesh(lo, hi, 1), 3)
        M = assemble_level(H.levels[3], Factor("vol"))
        for l in range(4):
            E = H.embed(3, l)
            ref = np.asarray((E.T @ M @ E).sum(axis=1)).ravel()
            assert np.allclose(kuhn_hat_integrals(l, hi - lo), ref, rtol=1e-13, atol=0), l
