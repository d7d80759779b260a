"""The library's host-side spaces and factors against the oracle, on the CPU
(sgdg_inspect_level / _embedding / _factor: the code sgdg_create runs,
without a handle or a device).

* Levels: the vertex coordinates of every level, in the canonical order of
  the storage layout, equal the oracle's (d = 1, 2, 3; periodic and not).
* Embeddings E_{l+1 <- l} (Sect. 4.2) equal the oracle's, entry for entry.
* Kronecker factors (Sect. 4.2): mass, derivative pairings, weights by the
  coefficient functions of the workloads (linear v, sin/cos of x), products
  of two weights, sign restrictions (the inflow splitting of Sect. 5.2) and
  boundary faces on every box side, on both sides of the phase space,
  assembled on level L and projected to every coarser level, agree with
  the oracle's independent assembly and projection to 1e-13 of the
  factor's largest entry.  Both use collapsed Gauss rules with 4 points per
  direction, written independently.
* The factor-transfer products of the sweep (sgdg_inspect_product:
  R_l X_{l+1} and X_l E_{l-1}) equal the oracle's projected factors times
  its embeddings, to 1e-13.
* Load vectors of the source terms (sgdg_inspect_load; a product of two
  functions, its value and derivative pairings) on every level, d = 1, 2, 3.
* The Kronecker term table (sgdg_inspect_terms: time couplings of the
  strip, δ placement, inflow splitting, time-factor gates) with the factors
  forms the same finest full-grid operator sum_k X_k (x) V_k (x) tau_k as the
  oracle's block formula, to 1e-13 (d = 1, 2, 3; with and without inflow
  boundaries; time-dependent strips across sign changes; time rules of 1 to
  8 Gauss points per strip).
* Bad requests give SGDG_EINVAL.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2204_05988_gb300 as P
import sgdg_workloads as W
from oracle.assembly import Factor, FactorStore
from oracle.mesh import Hierarchy


def _csr(t, n):
    rp, cl, vl = t
    return sp.csr_matrix((vl, cl, rp), shape=(len(rp) - 1, n))


MESHES = [W.interval_mesh(0.0, 1.0, 4), W.interval_mesh(-1.0, 1.0, 4, periodic=True), W.square_mesh(0.0, 1.0, 2),
          W.square_mesh(-1.0, 1.0, 4, periodic=True), W.cube_mesh(0.0, 1.0, 1)]


@pytest.mark.parametrize("mesh", MESHES, ids=lambda m: f"d{m.dim}{'_per' if any(m.periodic) else ''}")
def test_levels_and_embeddings_equal_the_oracle(mesh):
    L = 2 if mesh.dim < 3 else 1
    H = Hierarchy(mesh, L)
    for l in range(L + 1):
        c = P.inspect_level(mesh, L, l)
        assert c.shape == H.levels[l].coords.shape and np.array_equal(c, H.levels[l].coords), l
    for l in range(L):
        E = _csr(P.inspect_embedding(mesh, L, l), H.levels[l].n)
        assert (E != H.E[l]).nnz == 0, l


def _oracle_factor(prob, side, spec):
    d = prob.d
    fn = lambda i: (prob.sigma if i == 2 * d else prob.beta[i]).__dict__["fx" if side == 0 else "fv"]
    kind = "face" if spec.get("kind", 0) == 1 else "vol"
    return Factor(kind, 1.0, tuple(fn(i) for i in spec.get("weight", ())), spec.get("test", 0),
                  spec.get("trial", 0), tuple((fn(i), 1.0, s) for i, s in spec.get("restrict", ())),
                  spec.get("face", (-1, 0)))


def _specs(prob, side):
    """Factor specs with weights and restrictions by the functions this side has."""
    d = prob.d
    have = [p for p in range(2 * d) if (prob.beta[p].fx if side == 0 else prob.beta[p].fv) is not None]
    out = [{}]
    for p in range(1, d + 1):
        out += [{"test": p, "trial": p}, {"test": 0, "trial": p}, {"test": p, "trial": 0}]
    if d >= 2:
        out.append({"test": 1, "trial": 2})
    for a in have:
        out += [{"weight": (a,)}, {"weight": (a,), "test": 0, "trial": 1}, {"weight": (a,), "restrict": ((a, 1),)},
                {"weight": (a,), "restrict": ((a, -1),)}]
        for b in have:
            if b >= a:
                out.append({"weight": (a, b), "test": 1, "trial": d})
        for ax in range(d):
            for sd in (-1, 1):
                out.append({"kind": 1, "weight": (a,), "restrict": ((a, -sd),), "face": (ax, sd)})
    for ax in range(d):
        for sd in (-1, 1):
            out.append({"kind": 1, "face": (ax, sd)})
    return out


def _map_ids(prob, spec):
    """Oracle function index 2d (sigma) is id 6 in the C ABI."""
    d = prob.d
    m = lambda i: 6 if i == 2 * d else i
    out = dict(spec)
    if "weight" in spec:
        out["weight"] = tuple(m(i) for i in spec["weight"])
    if "restrict" in spec:
        out["restrict"] = tuple((m(i), s) for i, s in spec["restrict"])
    return out


@pytest.mark.parametrize("case", ["d1_inflow", "d2_transport", "d3_transport"])
def test_factors_equal_the_oracle(case):
    prob = {"d1_inflow": lambda: W.inflow_manufactured_1d(L=3), "d2_transport": lambda: W.transport_2d(L=2),
            "d3_transport": lambda: W.transport_3d(L=1)}[case]()
    L = prob.L
    for side, mesh in ((0, prob.mesh_x), (1, prob.mesh_v)):
        H = Hierarchy(mesh, L)
        fs = FactorStore(H)
        specs = _specs(prob, side)
        if prob.sigma.coef != 0.0 and (prob.sigma.fx if side == 0 else prob.sigma.fv) is not None:
            specs.append({"weight": (2 * prob.d,)})
        for spec in specs:
            f = _oracle_factor(prob, side, spec)
            cs = _map_ids(prob, spec)
            for level in range(L, -1, -1):
                A = _csr(P.inspect_factor(prob, side, L, level, kind=cs.get("kind", 0), test=cs.get("test", 0),
                                          trial=cs.get("trial", 0), weight=cs.get("weight", ()),
                                          restrict=cs.get("restrict", ()), face=cs.get("face", (-1, 0))),
                         H.levels[level].n)
                B = fs.proj(f, level, level)
                scale = max(abs(B).max(), 1e-300)
                assert abs(A - B).max() <= 1e-13 * scale, (case, side, spec, level, abs(A - B).max(), scale)


def test_bad_requests_are_refused():
    prob = W.transport_2d(L=1)
    with pytest.raises(P.SgdgError) as e:
        P.inspect_level(prob.mesh_x, 2, 3)
    assert e.value.code == 1
    with pytest.raises(P.SgdgError):
        P.inspect_embedding(prob.mesh_x, 2, 2)                 # no E out of the finest level
    with pytest.raises(P.SgdgError):
        P.inspect_factor(prob, 0, 1, 1, weight=(0,))           # beta_0 = v1 has no x function
    with pytest.raises(P.SgdgError):
        P.inspect_factor(prob, 1, 1, 1, kind=1, face=(2, 1))   # axis 2 on a 2-D mesh
    with pytest.raises(P.SgdgError):
        P.inspect_factor(prob, 0, 1, 1, test=3)
    bad = W.CoarseMesh(coords=np.array([[0.0], [0.5], [0.5], [1.0]]), cells=np.array([[0, 1], [2, 3]], dtype=np.int32),
                       lo=(0.0,), hi=(1.0,), periodic=(False,))
    with pytest.raises(P.SgdgError):
        P.inspect_level(bad, 1, 0)


def _library_operator(prob, t0, time_quad=0):
    """sum_k X_k (x) V_k (x) tau_k on the finest full grid (L, L), from the
    library's term table and factors."""
    L = prob.L
    cache = {}

    def fac(side, spec):
        key = (side, repr(sorted(spec.items())))
        if key not in cache:
            n = P.inspect_level(prob.mesh_x if side == 0 else prob.mesh_v, L, L).shape[0]
            cache[key] = _csr(P.inspect_factor(prob, side, L, L, **spec), n)
        return cache[key]

    A = None
    for tau, xs, vs in P.inspect_terms(prob, t0, time_quad):
        K = sp.kron(fac(0, xs), sp.kron(fac(1, vs), sp.csr_matrix(tau)))
        A = K if A is None else A + K
    return A.tocsr()


def _oracle_operator(prob, t0, m=3):
    from oracle.operator import SparseGridOperator, is_time_dependent, kron_terms
    op = SparseGridOperator(prob)
    terms = kron_terms(prob, t0, m) if is_time_dependent(prob) else op.terms
    A = None
    for tau, X, V in terms:
        K = sp.kron(op.fx.fine(X), sp.kron(op.fv.fine(V), sp.csr_matrix(tau)))
        A = K if A is None else A + K
    return A.tocsr()


@pytest.mark.parametrize("case,t0", [
    ("transport_2d", 0.0), ("free_streaming_1d", 0.0), ("inflow_manufactured_1d", 0.0), ("transport_3d", 0.0),
    ("time_dependent_1d", 0.5), ("time_dependent_2d", 0.25), ("inflow_time_dependent_1d", 0.25),
    ("inflow_time_dependent_2d", 0.25)])
def test_term_table_gives_the_oracle_operator(case, t0):
    """The library's Kronecker terms (time couplings of the strip at t0,
    inflow splitting, time-factor gates) with its factors form the same
    finest full-grid operator as the oracle's block formula (Sect. 4.2); the
    time-dependent strips contain a sign change of a beta component."""
    make = {"transport_2d": lambda: W.transport_2d(L=1), "free_streaming_1d": lambda: W.free_streaming_1d(L=2),
            "inflow_manufactured_1d": lambda: W.inflow_manufactured_1d(L=2),
            "transport_3d": lambda: W.transport_3d(L=0), "time_dependent_1d": lambda: W.time_dependent_1d(L=2),
            "time_dependent_2d": lambda: W.time_dependent_2d(L=1),
            "inflow_time_dependent_1d": lambda: W.inflow_time_dependent_1d(L=2),
            "inflow_time_dependent_2d": lambda: W.inflow_time_dependent_2d(L=1)}
    prob = make[case]()
    A, B = _library_operator(prob, t0), _oracle_operator(prob, t0)
    assert A.shape == B.shape
    assert abs(A - B).max() <= 1e-13 * abs(B).max(), (case, abs(A - B).max(), abs(B).max())


def test_term_table_comparison_sees_the_strip_time():
    """The comparison is sensitive to the time couplings: the library's terms
    of the next strip (t0 + dt) differ from the oracle's operator of the strip
    at t0, which contains a sign change of a time factor."""
    prob = W.time_dependent_1d(L=2)
    A, B = _library_operator(prob, 0.5 + prob.dt), _oracle_operator(prob, 0.5)
    assert abs(A - B).max() > 1e-6 * abs(B).max()


@pytest.mark.parametrize("mesh", [W.interval_mesh(0.0, 1.0, 4), W.square_mesh(-1.0, 1.0, 2), W.cube_mesh(0.0, 1.0, 1)],
                         ids=["d1", "d2", "d3"])
def test_load_vectors_equal_the_oracle(mesh):
    """The spatial factors of the source terms (Sect. 2, b_j): loads of a
    product of functions and of its derivative pairing, on every level."""
    from oracle.assembly import assemble_load, assemble_load_grad
    L = 2 if mesh.dim < 3 else 1
    H = Hierarchy(mesh, L)
    f1 = lambda p: np.cos(np.pi * p[:, 0]) + 0.5
    f2 = lambda p: 1.0 + p[:, -1] ** 2
    prod = lambda p: f1(p) * f2(p)
    for level in range(L + 1):
        E = H.embed(L, level)
        ref0 = E.T @ assemble_load(H.levels[L], prod)
        got0 = P.inspect_load(mesh, L, level, (f1, f2), 0)
        assert np.abs(got0 - ref0).max() <= 1e-13 * np.abs(ref0).max(), level
        one = P.inspect_load(mesh, L, level, (), 0)
        assert abs(one.sum() - np.prod(np.array(mesh.hi) - np.array(mesh.lo))) < 1e-12
        for ax in range(mesh.dim):
            ref = E.T @ assemble_load_grad(H.levels[L], prod, ax)
            got = P.inspect_load(mesh, L, level, (f1, f2), ax + 1)
            assert np.abs(got - ref).max() <= 1e-13 * max(np.abs(ref).max(), 1e-300), (level, ax)


@pytest.mark.parametrize("case", ["d1_inflow", "d2_transport", "d3_transport"])
def test_transfer_products_equal_the_oracle(case):
    """The factor-transfer products the sweep applies (sgdg_inspect_product):
    R_l X_{l+1} = E_l^T X_{l+1} and X_l E_{l-1}, for the mass, a derivative
    pairing and a weighted factor, against the oracle's projected factors
    times its embeddings."""
    prob = {"d1_inflow": lambda: W.inflow_manufactured_1d(L=3), "d2_transport": lambda: W.transport_2d(L=2),
            "d3_transport": lambda: W.transport_3d(L=1)}[case]()
    L = prob.L
    for side, mesh in ((0, prob.mesh_x), (1, prob.mesh_v)):
        H = Hierarchy(mesh, L)
        fs = FactorStore(H)
        have = [p for p in range(2 * prob.d) if (prob.beta[p].fx if side == 0 else prob.beta[p].fv) is not None]
        specs = [{}, {"test": 0, "trial": 1}] + [{"weight": (have[0],), "test": 1, "trial": 0}]
        for spec in specs:
            f = _oracle_factor(prob, side, spec)
            for level in range(L + 1):
                if level < L:
                    A = _csr(P.inspect_factor(prob, side, L, level, product=0, **spec), H.levels[level + 1].n)
                    B = (H.E[level].T @ fs.proj(f, level + 1, level + 1)).tocsr()
                    assert abs(A - B).max() <= 1e-13 * abs(B).max(), (case, side, spec, level, "RX")
                if level >= 1:
                    A = _csr(P.inspect_factor(prob, side, L, level, product=1, **spec), H.levels[level - 1].n)
                    B = (fs.proj(f, level, level) @ H.E[level - 1]).tocsr()
                    assert abs(A - B).max() <= 1e-13 * abs(B).max(), (case, side, spec, level, "XE")


@pytest.mark.parametrize("m", [1, 2, 5, 8])
def test_time_quadrature_rules_equal_the_oracle(m):
    """Strips with time factors under m-point rules (the library's nodes by
    Newton's method on P_m, the oracle's from numpy's leggauss): the same
    operator, on a strip across a sign change of the field."""
    prob = W.time_dependent_1d(L=2)
    A, B = _library_operator(prob, 0.5, m), _oracle_operator(prob, 0.5, m)
    assert abs(A - B).max() <= 1e-13 * abs(B).max(), (m, abs(A - B).max())
    if m == 1:
        C = _oracle_operator(prob, 0.5, 3)
        assert abs(A - C).max() > 1e-6 * abs(C).max()     # the rule matters on this strip


def test_non_finite_coefficient_values_are_refused():
    """A coefficient function of the operator that returns NaN or Inf
    anywhere (a weight at a quadrature point, a restriction at a centroid, a
    face weight) makes the assembly fail with SGDG_EINVAL instead of filling
    the factors with NaN; sgdg_create runs the same code.  Data loads (u0,
    sources) pass NaN on: the solver's NaN check reports them (SGDG_ENAN)."""
    prob = W.transport_2d(L=1)
    bad = lambda p: np.where(p[:, 0] > 0.7, np.nan, p[:, 0])
    inf = lambda p: np.where(p[:, 1] < -0.7, np.inf, 1.0 + p[:, 1])
    prob.beta[0] = W.Product(1.0, None, bad)
    prob.beta[1] = W.Product(1.0, None, inf)
    for kw in ({"weight": (0,)}, {"weight": (1,), "test": 1, "trial": 0}, {"restrict": ((0, 1),)},
               {"kind": 1, "weight": (1,), "face": (1, -1)}):
        with pytest.raises(P.SgdgError) as e:
            P.inspect_factor(prob, 1, 1, 1, **kw)
        assert e.value.code == 1 and "NaN or Inf" in str(e.value), kw
    assert np.isnan(P.inspect_load(prob.mesh_v, 1, 0, (bad,), 0)).any()
    P.inspect_factor(W.transport_2d(L=1), 1, 1, 1, weight=(0,))   # the finite original passes
