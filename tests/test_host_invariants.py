"""Invariants of the library's own host code (through sgdg_inspect_*, CPU
only), independent of the oracle:

* E 1 = 1: every row of every embedding sums to one, and E carries linear
  functions exactly (P1 nesting, Sect. 2).
* Galerkin consistency (Sect. 4.2): the mass and stiffness factors projected
  from level L to level l equal the factors assembled directly on a
  hierarchy refined only to l.
* Mass row sums: sum_j M_ij = int phi_i (the library's load of 1), total
  |Omega|.
* Green's identity (Sect. 3, stability): D_p + D_p^T equals the difference of
  the face masses on the two sides of axis p (non-periodic box).
* Time couplings (Eq. 10 with the Legendre basis): for beta = 0 the single
  term has tau = T_t + G_t + sigma M_t with M_t = dt diag(1, 1/3),
  T_t = [[0, 2], [0, 0]], G_t = [[1, -1], [-1, 1]] in closed form, and one
  strip of a mode then advances by the Radau IIA stability function.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2204_05988_gb300 as P
import sgdg_workloads as W

MESHES = [W.interval_mesh(0.0, 2.0, 4), W.interval_mesh(0.0, 1.0, 4, periodic=True), W.square_mesh(-1.0, 1.0, 2),
          W.square_mesh(0.0, 1.0, 4, periodic=True), W.cube_mesh(0.0, 1.0, 1)]
IDS = ["d1", "d1_per", "d2", "d2_per", "d3"]


def _csr(t, ncols):
    rp, cl, vl = t
    return sp.csr_matrix((vl, cl, rp), shape=(len(rp) - 1, ncols))


def _problem(mesh):
    """A problem whose only use is to carry the mesh and constant coefficients."""
    d = mesh.dim
    return W.Problem(name="host", d=d, mesh_x=mesh, mesh_v=mesh, L=0, r=1, dt=0.1, delta=0.0, n_strips=1,
                     beta=[W.Product(0.0)] * (2 * d), sigma=W.Product(0.0), u0=[])


@pytest.mark.parametrize("mesh", MESHES, ids=IDS)
def test_embeddings_partition_of_unity_and_linear(mesh):
    L = 2 if mesh.dim < 3 else 1
    f = lambda X: 0.25 + X @ np.arange(1.0, mesh.dim + 1.0)
    for l in range(L):
        c0, c1 = P.inspect_level(mesh, L, l), P.inspect_level(mesh, L, l + 1)
        E = _csr(P.inspect_embedding(mesh, L, l), c0.shape[0])
        assert np.abs(E @ np.ones(c0.shape[0]) - 1.0).max() < 1e-15
        if not any(mesh.periodic):
            assert np.abs(E @ f(c0) - f(c1)).max() < 1e-13


@pytest.mark.parametrize("mesh", MESHES, ids=IDS)
def test_projection_equals_direct_assembly(mesh):
    prob = _problem(mesh)
    L = 2 if mesh.dim < 3 else 1
    for spec in ({}, {"test": 1, "trial": 1}, {"test": 0, "trial": mesh.dim}):
        for l in range(L):
            n = P.inspect_level(mesh, L, l).shape[0]
            projected = _csr(P.inspect_factor(prob, 0, L, l, **spec), n)
            direct = _csr(P.inspect_factor(prob, 0, l, l, **spec), n)
            assert abs(projected - direct).max() <= 1e-13 * abs(direct).max(), (spec, l)


@pytest.mark.parametrize("mesh", MESHES, ids=IDS)
def test_mass_row_sums_and_total(mesh):
    prob = _problem(mesh)
    L = 1
    n = P.inspect_level(mesh, L, L).shape[0]
    M = _csr(P.inspect_factor(prob, 0, L, L), n)
    ones = P.inspect_load(mesh, L, L, (), 0)
    assert np.abs(M @ np.ones(n) - ones).max() < 1e-15
    assert abs(M.sum() - np.prod(np.array(mesh.hi) - np.array(mesh.lo))) < 1e-13


@pytest.mark.parametrize("mesh", [MESHES[0], MESHES[2], MESHES[4]], ids=["d1", "d2", "d3"])
def test_green_identity(mesh):
    prob = _problem(mesh)
    L = 1
    n = P.inspect_level(mesh, L, L).shape[0]
    for p in range(1, mesh.dim + 1):
        D = _csr(P.inspect_factor(prob, 0, L, L, test=0, trial=p), n)          # int d_p phi_j phi_i
        faces = sum(side * _csr(P.inspect_factor(prob, 0, L, L, kind=1, face=(p - 1, side)), n)
                    for side in (-1, 1))
        assert abs(D + D.T - faces).max() < 1e-13, p


def test_time_couplings_closed_forms():
    dt, sigma = 0.05, 0.7
    prob = W.free_streaming_1d(L=1, n_strips=1)
    prob.beta = [W.Product(0.0), W.Product(0.0)]
    prob.dt, prob.delta = dt, 0.0
    prob.sigma = W.Product(sigma)
    terms = P.inspect_terms(prob)
    Mt = dt * np.diag([1.0, 1.0 / 3.0])
    Tt = np.array([[0.0, 2.0], [0.0, 0.0]])
    Gt = np.array([[1.0, -1.0], [-1.0, 1.0]])
    assert len(terms) == 1
    tau, xs, vs = terms[0]
    assert xs["test"] == xs["trial"] == vs["test"] == vs["trial"] == 0 and not xs["weight"] and not vs["weight"]
    assert np.abs(tau - (Tt + Gt + sigma * Mt)).max() < 1e-15


@pytest.mark.parametrize("sigma_dt", [0.01, 0.5, 2.0, 40.0])
def test_dg1_strip_is_radau_iia(sigma_dt):
    """With beta = 0 and delta = 0 the spatial factor is the mass matrix, so
    every mode follows the 2 x 2 strip system tau c = eta(t_{j-1}^+) U^-:
    the end value c_0 + c_1 over U^- is the stability function of DG(1) in
    time, the (1, 2) Pade approximant of exp(z) that 2-stage Radau IIA also
    has, R(z) = (1 + z/3) / (1 - 2z/3 + z^2/6), z = -sigma dt."""
    dt = 0.1
    prob = W.free_streaming_1d(L=1, n_strips=1)
    prob.beta = [W.Product(0.0), W.Product(0.0)]
    prob.dt, prob.delta = dt, 0.0
    prob.sigma = W.Product(sigma_dt / dt)
    (tau, _, _), = P.inspect_terms(prob)
    c = np.linalg.solve(tau, np.array([1.0, -1.0]))     # eta_s(t_{j-1}^+) = (1, -1)
    z = -sigma_dt
    R = (1.0 + z / 3.0) / (1.0 - 2.0 * z / 3.0 + z * z / 6.0)
    assert abs((c[0] + c[1]) - R) < 1e-14 * max(1.0, abs(R)), (sigma_dt, c[0] + c[1], R)
