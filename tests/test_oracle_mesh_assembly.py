"""Pins of the oracle's meshes, embeddings and factor matrices (CPU only).

Each check compares against something the mathematics fixes independently of
the oracle's own code: vertex counts of uniform refinement, partition of
unity, closed-form integrals of polynomials, Green's identity (Sect. 3) and
exactness of the Galerkin projection for nested spaces (Sect. 4.2).
"""
import numpy as np
import pytest
import scipy.sparse as sp

import sgdg_workloads as W
from oracle.assembly import Factor, assemble_level, assemble_load
from oracle.mesh import Hierarchy

pytestmark = pytest.mark.filterwarnings("ignore")


@pytest.mark.parametrize("L", [0, 1, 3])
def test_vertex_counts(L):
    h1 = Hierarchy(W.interval_mesh(0, 1, 4), L)
    assert [lv.n for lv in h1.levels] == [4 * 2 ** l + 1 for l in range(L + 1)]
    h2 = Hierarchy(W.square_mesh(0, 1, 2), L)
    assert [lv.n for lv in h2.levels] == [(2 ** (l + 1) + 1) ** 2 for l in range(L + 1)]
    assert [lv.cells.shape[0] for lv in h2.levels] == [8 * 4 ** l for l in range(L + 1)]
    hp = Hierarchy(W.interval_mesh(0, 1, 4, periodic=True), L)
    assert [lv.n for lv in hp.levels] == [4 * 2 ** l for l in range(L + 1)]
    hp2 = Hierarchy(W.square_mesh(0, 1, 2, periodic=True), L)
    assert [lv.n for lv in hp2.levels] == [(2 ** (l + 1)) ** 2 for l in range(L + 1)]


def test_canonical_order_lexicographic():
    h = Hierarchy(W.square_mesh(-1, 1, 2), 2)
    c = h.levels[2].coords
    m = 2 ** 3 + 1
    grid = np.linspace(-1, 1, m)
    # last axis slowest: row-major (y, x) lattice
    assert np.array_equal(c[:, 0], np.tile(grid, m))
    assert np.array_equal(c[:, 1], np.repeat(grid, m))


@pytest.mark.parametrize("mesh", [W.interval_mesh(0, 1, 4), W.square_mesh(-1, 1, 2),
                                  W.interval_mesh(0, 1, 4, periodic=True),
                                  W.square_mesh(0, 1, 2, periodic=True)])
def test_embedding_partition_of_unity_and_linear(mesh):
    h = Hierarchy(mesh, 3)
    for l in range(3):
        E = h.E[l]
        assert np.allclose(E @ np.ones(E.shape[1]), 1.0, atol=0, rtol=0)
        if not any(mesh.periodic):
            # P1 reproduces linear functions: E x_coarse = x_fine
            for ax in range(mesh.dim):
                assert np.array_equal(E @ h.levels[l].coords[:, ax], h.levels[l + 1].coords[:, ax])


@pytest.mark.parametrize("mesh,vol", [(W.interval_mesh(0, 1, 4), 1.0), (W.square_mesh(-1, 1, 2), 4.0),
                                      (W.square_mesh(0, 1, 2, periodic=True), 1.0)])
def test_mass_rowsums_and_total(mesh, vol):
    h = Hierarchy(mesh, 2)
    lev = h.levels[2]
    M = assemble_level(lev, Factor("vol"))
    one = assemble_load(lev, None)
    assert np.allclose(M @ np.ones(lev.n), one, rtol=1e-14, atol=1e-16)
    assert abs(M.sum() - vol) < 1e-13
    # int phi_k: interior vertex of a uniform mesh = |patch| / (d+1)
    if mesh.dim == 1 and not mesh.periodic[0]:
        hh = 1.0 / 16
        assert np.allclose(one[1:-1], hh) and np.allclose(one[[0, -1]], hh / 2)


def test_polynomial_weights_closed_forms():
    """1^T X(w) 1 = int w; x^T-moments of the derivative factors."""
    v2 = lambda p: p[:, 0] * p[:, 1]
    sq = lambda p: p[:, 0] ** 2
    h = Hierarchy(W.square_mesh(-1, 1, 2), 2)
    lev = h.levels[2]
    one = np.ones(lev.n)
    X = assemble_level(lev, Factor("vol", 1.0, (sq,)))
    assert abs(one @ X @ one - 4.0 / 3.0) < 1e-13           # int_{[-1,1]^2} v1^2 = 2/3 * 2
    X = assemble_level(lev, Factor("vol", 1.0, (sq, sq)))
    assert abs(one @ X @ one - 4.0 / 5.0) < 1e-13           # int v1^4 = 2/5 * 2
    for p in (1, 2):
        D = assemble_level(lev, Factor("vol", 1.0, (), 0, p))   # int d_p phi_j phi_i
        assert np.allclose(D @ one, 0.0, atol=1e-14)
        # trial = coordinate x_p: d_p x_p = 1 -> row sums = int phi_i
        assert np.allclose(D @ lev.coords[:, p - 1], assemble_load(lev, None), atol=1e-14)
        S = assemble_level(lev, Factor("vol", 1.0, (), p, p))   # stiffness part
        assert abs(lev.coords[:, p - 1] @ S @ lev.coords[:, p - 1] - 4.0) < 1e-13


@pytest.mark.parametrize("mesh", [W.interval_mesh(0, 1, 4), W.square_mesh(-1, 1, 2)])
def test_green_identity(mesh):
    """(d_p phi_j, phi_i) + (phi_j, d_p phi_i) = int_{dOmega} n_p phi_j phi_i (Sect. 3)."""
    h = Hierarchy(mesh, 2)
    lev = h.levels[2]
    for p in range(1, mesh.dim + 1):
        D = assemble_level(lev, Factor("vol", 1.0, (), 0, p))
        G = sum(side * assemble_level(lev, Factor("face", 1.0, face=(p - 1, side))) for side in (-1, 1))
        assert abs(D + D.T - G).max() < 1e-14


def test_galerkin_projection_is_coarse_assembly():
    """E^T X_fine E = X_coarse for polynomial weights (nested spaces, exact quadrature)."""
    v1 = lambda p: p[:, 0]
    h = Hierarchy(W.square_mesh(-1, 1, 2), 2)
    for f in [Factor("vol"), Factor("vol", 1.0, (v1,), 0, 2), Factor("vol", 1.0, (v1, v1), 1, 2),
              Factor("face", 1.0, (v1,), face=(1, -1))]:
        Xf = assemble_level(h.levels[2], f)
        Xc = assemble_level(h.levels[0], f)
        E = h.embed(2, 0)
        assert abs(E.T @ Xf @ E - Xc).max() < 1e-14


def test_sign_split_faces_sum():
    """Splitting a face integral by the sign of a weight that changes sign on a
    mesh line reproduces the unsplit integral."""
    h = Hierarchy(W.square_mesh(0, 1, 2), 2)
    lev = h.levels[2]
    E1 = lambda p: np.sin(2 * np.pi * p[:, 1])
    full = assemble_level(lev, Factor("vol", 0.5, (E1,)))
    parts = [assemble_level(lev, Factor("vol", 0.5, (E1,), restrict=((E1, 0.5, s),))) for s in (1, -1)]
    assert abs(parts[0] + parts[1] - full).max() < 1e-15
    assert parts[0].nnz > 0 and parts[1].nnz > 0
