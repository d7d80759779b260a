"""GPU parity with time-dependent beta and sigma (Sect. 4.2: the block
formula as a Gauss sum over every strip's time points, the inflow boundary
following the sign of the time factors).

The library recomputes the 2 x 2 time couplings of its Kronecker terms per
strip; applies use the operator of the strip that starts at the handle's
current time, which advances by dt with every strip.  Compared with the
oracle's time-dependent block formula (pinned against the brute-force
space-time weak form in test_oracle_time): applies 1e-12 (FP64) and 1e-5
(FP32) relative, per grid as well; strip solutions 1e-8 on the canonical
nodal values.  Strips cross the times where the v-component of beta changes
sign (t = 0.52 in d = 1, t = 0.26 in d = 2).
"""
import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def P():
    import paper_2204_05988_gb300 as P
    P.load_library()
    return P


def _apply(P, s, u, prec):
    dt = torch.float64 if prec == "fp64" else torch.float32
    ud = torch.tensor(u, dtype=dt, device="cuda")
    yd = torch.full_like(ud, float("nan"))
    s.apply_operator(ud, yd, P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32)
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


@pytest.mark.parametrize("case", ["d1", "d2"])
def test_apply_follows_the_strip_time(P, case):
    """Applies before any strip (strip (0, dt)) and after k strips (strip
    (k dt, (k + 1) dt), one across the sign change) against the oracle."""
    from oracle.operator import SparseGridOperator
    prob = W.time_dependent_1d(L=3) if case == "d1" else W.time_dependent_2d(L=2)
    k_strips = 4 if case == "d1" else 4
    op = SparseGridOperator(prob)
    s = P.Solver(prob, rtol=1e-10, restart=30, inner_its=30, inner_rtol=1e-4)
    u = W.uniform_vector(op.size, seed=61)
    for prec in ("fp64", "fp32"):
        ref = op.apply(u)
        y = _apply(P, s, u, prec)
        assert _rel(y, ref) < (1e-12 if prec == "fp64" else 1e-5), prec
    s.set_initial()
    for _ in range(k_strips):
        s.advance_strip()
    op.set_time(k_strips * prob.dt)
    ref = op.apply(u)
    for prec in ("fp64", "fp32"):
        tol = 1e-12 if prec == "fp64" else 1e-5
        y = _apply(P, s, u, prec)
        assert _rel(y, ref) < tol, prec
        for i in range(len(op.grids)):
            a, b = y[op.offsets[i]:op.offsets[i + 1]], ref[op.offsets[i]:op.offsets[i + 1]]
            assert np.abs(a - b).max() < tol * np.abs(b).max(), (prec, i)
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_strips_with_time_dependent_coefficients(P, prec):
    """Six d = 1 strips (t from 0 to 0.75, across the sign change of the
    field) against the oracle's strip solutions."""
    from oracle.solver import StripSolver, nodal_values
    prob = W.time_dependent_1d(L=3, n_strips=6)
    ref = StripSolver(prob, tol=1e-12)
    ends = ref.run()
    s = P.Solver(prob, precision=P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32, rtol=1e-11,
                 restart=30, inner_its=30, inner_rtol=1e-4)
    s.set_initial()
    for j in range(prob.n_strips):
        st = s.advance_strip()
        assert st.status == 0 and st.rel_residual <= 1e-11, j
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        assert _rel(nodal_values(ref.op, U, R=1), nodal_values(ref.op, ends[j], R=1)) < 1e-8, j
    s.close()


def test_strips_d2_time_dependent(P):
    from oracle.solver import StripSolver, nodal_values
    prob = W.time_dependent_2d(L=2, n_strips=5)
    ref = StripSolver(prob, tol=1e-12)
    ends = ref.run()
    s = P.Solver(prob, rtol=1e-11, restart=30, inner_its=30, inner_rtol=1e-4)
    s.set_initial()
    for j in range(prob.n_strips):
        st = s.advance_strip()
        assert st.status == 0, j
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        assert _rel(nodal_values(ref.op, U, R=1), nodal_values(ref.op, ends[j], R=1)) < 1e-8, j
    s.close()


def test_batch_graph_recaptures_when_the_time_moves(P):
    """A batch graph captured at t = 0 is not replayed with stale couplings
    after a member advanced: the batch apply equals the member's own apply
    at its new time."""
    prob = W.time_dependent_1d(L=3)
    a = P.Solver(prob, rtol=1e-10, restart=30, inner_its=30, inner_rtol=1e-4)
    b = P.Solver(W.free_streaming_1d(L=3), rtol=1e-10)
    B = P.Batch([a, b])
    ua = torch.tensor(W.uniform_vector(a.n_coeffs, seed=62), device="cuda")
    ub = torch.tensor(W.uniform_vector(b.n_coeffs, seed=63), device="cuda")
    ya, yb = torch.empty_like(ua), torch.empty_like(ub)
    B.apply([ua, ub], [ya, yb], P.SGDG_FP64)
    y0 = ya.clone()
    a.set_initial()
    a.advance_strip()
    a.advance_strip()
    B.apply([ua, ub], [ya, yb], P.SGDG_FP64)
    ref = torch.empty_like(ua)
    a.apply_operator(ua, ref, P.SGDG_FP64)
    torch.cuda.synchronize()
    assert torch.equal(ya, ref)
    assert not torch.equal(ya, y0)
    B.close()
    a.close()
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_time_dependent_inflow_and_sources(P, prec):
    """Sources and inflow data with a time factor in beta (beta_v changes sign
    at t = 1/3, inside the third strip): strip solutions against the oracle
    at 1e-8, and the manufactured solution reproduced at every node."""
    from oracle.solver import StripSolver, nodal_values
    prob = W.inflow_time_dependent_1d(L=3)
    ref = StripSolver(prob, tol=1e-12)
    ends = ref.run()
    s = P.Solver(prob, precision=P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32, rtol=1e-11,
                 restart=30, inner_its=30, inner_rtol=1e-4)
    s.set_initial()
    for j in range(prob.n_strips):
        st = s.advance_strip()
        assert st.status == 0 and st.rel_residual <= 1e-11, j
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        got = nodal_values(ref.op, U, R=1)
        assert _rel(got, nodal_values(ref.op, ends[j], R=1)) < 1e-8, j
        exact = []
        for (l1, l2) in ref.op.grids:
            x, v = ref.op.hx.levels[l1].coords[:, 0], ref.op.hv.levels[l2].coords[:, 0]
            exact.append(prob.exact((j + 1) * prob.dt, x[:, None], v[None, :]).ravel())
        exact = np.concatenate(exact)
        assert np.abs(got - exact).max() < 1e-8 * np.abs(exact).max(), j
    s.close()


def test_time_factors_with_vlasov_poisson_are_rejected(P):
    prob = W.landau_4d(L=2)
    prob.sigma = W.Product(0.1, None, None, lambda t: 1.0 + np.asarray(t))
    with pytest.raises(P.SgdgError):
        P.Solver(prob, vlasov_poisson=True)
