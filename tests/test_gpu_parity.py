"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (relative l2 over the output vector):
  * operator, mass and diagonal-block applies: 1e-12 in FP64, 1e-5 in FP32
    (apply outputs are unique - rows are test functions); the operator and
    mass applies are also checked grid by grid at the same tolerances, as
    max |y_l - ref_l| / max |ref_l| on every component grid l, so that a
    wrong boundary row or ragged tile edge on one grid is not diluted by the
    other grids' correct entries;
  * strip solutions: 1e-8 on the canonical nodal values (the spanning-set
    coefficients are not unique, Sect. 4.1), both sides solved tightly.
Inputs are seeded U[-1, 1] vectors from sgdg_workloads.
"""
import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _per_grid(op, y, ref, tol):
    """max-abs error over each component grid, scaled by that grid's largest
    reference value; every grid within tol."""
    for i in range(len(op.grids)):
        a, b = y[op.offsets[i]:op.offsets[i + 1]], ref[op.offsets[i]:op.offsets[i + 1]]
        err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
        assert err < tol, (op.grids[i], err)


@pytest.fixture(scope="module")
def P():
    import paper_2204_05988_gb300 as P
    P.load_library()
    return P


_CASES = {
    "d1_L6": lambda: W.free_streaming_1d(L=6),
    "d1_L0": lambda: W.free_streaming_1d(L=0),
    "d2_L3_sigma": lambda: W.transport_2d(L=3, sigma=0.1),
    "d2_L2_nosigma": lambda: W.transport_2d(L=2, sigma=0.0),
    "d1_periodic_L3": lambda: W.periodic_advection_1d(L=3),
}


@pytest.fixture(scope="module")
def setups(P):
    from oracle.operator import SparseGridOperator
    cache = {}

    def get(name):
        if name not in cache:
            prob = _CASES[name]()
            cache[name] = (prob, P.Solver(prob), SparseGridOperator(prob))
        return cache[name]
    return get


@pytest.mark.parametrize("name", list(_CASES))
def test_layout_matches_oracle(setups, name):
    prob, s, op = setups(name)
    assert s.n_coeffs == op.size
    assert s.shapes == [tuple(x) for x in op.shape]


@pytest.mark.parametrize("name", list(_CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_operator_parity(P, setups, name, prec):
    prob, s, op = setups(name)
    u = W.uniform_vector(op.size, seed=11)
    ref = op.apply(u)
    dt = torch.float64 if prec == "fp64" else torch.float32
    ud = torch.tensor(u, dtype=dt, device="cuda")
    yd = torch.full_like(ud, float("nan"))
    s.apply_operator(ud, yd, P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32)
    torch.cuda.synchronize()
    y = yd.double().cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert _rel(y, ref) < tol
    _per_grid(op, y, ref, tol)


@pytest.mark.parametrize("name", ["d1_L6", "d2_L3_sigma", "d1_L0"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_host_buffer_apply(P, setups, name, prec):
    """The host-buffer apply (grid-by-grid copies and conversions overlapped
    with the sweep) returns what the device-buffer apply returns, bit for
    bit, and the oracle's apply within the precision's tolerance."""
    prob, s, op = setups(name)
    u = W.uniform_vector(op.size, seed=13)
    ref = op.apply(u)
    pr = P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32
    hu = torch.tensor(u, dtype=torch.float64).pin_memory()
    hy = torch.full((op.size,), float("nan"), dtype=torch.float64).pin_memory()
    s.apply_operator_host(hu, hy, pr)
    dt = torch.float64 if prec == "fp64" else torch.float32
    ud = torch.tensor(u, dtype=torch.float64, device="cuda").to(dt)
    yd = torch.empty_like(ud)
    s.apply_operator(ud, yd, pr)
    torch.cuda.synchronize()
    assert torch.equal(hy, yd.double().cpu())
    assert _rel(hy.numpy(), ref) < (1e-12 if prec == "fp64" else 1e-5)


@pytest.mark.parametrize("name", ["d1_L6", "d2_L3_sigma"])
def test_apply_mass_parity(P, setups, name):
    prob, s, op = setups(name)
    u = W.uniform_vector(op.size, seed=12)
    ref = op.apply_mass(u)
    ud = torch.tensor(u, device="cuda")
    yd = torch.empty_like(ud)
    s.apply_mass(ud, yd, P.SGDG_FP64)
    torch.cuda.synchronize()
    assert _rel(yd.cpu().numpy(), ref) < 1e-12
    _per_grid(op, yd.cpu().numpy(), ref, 1e-12)


@pytest.mark.parametrize("name", ["d1_L6", "d2_L3_sigma"])
def test_apply_diag_parity(P, setups, name):
    prob, s, op = setups(name)
    L = prob.L
    for (l1, l2) in [(0, L), (L, 0), (L // 2, L - L // 2), (0, L - 1), (L - 1, 0)]:
        n1, n2 = op.grid_shape(l1, l2)
        u = W.uniform_vector(n1 * n2 * 2, seed=13 + l1)
        ref = op.apply_diag(l1, l2, u.reshape(n1, n2, 2)).ravel()
        ud = torch.tensor(u, device="cuda")
        yd = torch.empty_like(ud)
        s.apply_diag(l1, l2, ud, yd, P.SGDG_FP64)
        torch.cuda.synchronize()
        assert _rel(yd.cpu().numpy(), ref) < 1e-12, (l1, l2)


def test_apply_rejects_bad_levels(P, setups):
    prob, s, op = setups("d1_L6")
    ud = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(P.SgdgError):
        s.apply_diag(0, 0, ud, ud, P.SGDG_FP64)


def test_ct_preconditioner_parity(P):
    """Algorithm 1's preconditioner with (nearly) exact component solves."""
    from oracle.operator import SparseGridOperator
    from oracle.solver import ComponentSolver, ct_precondition
    prob = W.free_streaming_1d(L=3)
    s = P.Solver(prob, inner_its=60, inner_rtol=1e-13, cheb_steps=12)
    op = SparseGridOperator(prob)
    comp = ComponentSolver(op, tol=1e-13)
    r = W.uniform_vector(op.size, seed=21)
    ref = ct_precondition(op, comp, r)
    rd = torch.tensor(r, device="cuda")
    zd = torch.empty_like(rd)
    s.ct_precondition(rd, zd)
    torch.cuda.synchronize()
    assert _rel(zd.cpu().numpy(), ref) < 1e-9


def _nodal(P, s, U):
    Ud = torch.tensor(U, device="cuda")
    out = torch.empty_like(Ud)
    s.eval_nodal(Ud, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_eval_nodal_parity(P, setups):
    from oracle.solver import nodal_values
    prob, s, op = setups("d2_L3_sigma")
    U = W.uniform_vector(op.size // 2, seed=31)
    ref = nodal_values(op, U, R=1)
    assert _rel(_nodal(P, s, U), ref) < 1e-13


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_strip_solution_parity_free_streaming(P, prec):
    """Config d=1, L=6 (free streaming): the first strips agree with the
    oracle's strips on the canonical nodal values within 1e-8."""
    from oracle.solver import StripSolver, nodal_values
    prob = W.free_streaming_1d(L=6, n_strips=2)
    ref = StripSolver(prob, tol=1e-12)
    ends_ref = ref.run()
    s = P.Solver(prob, precision=P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32, rtol=1e-11,
                 restart=30, inner_its=30, inner_rtol=1e-4)
    s.set_initial()
    for j in range(2):
        st = s.advance_strip()
        assert st.rel_residual <= 1e-11
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        a = nodal_values(ref.op, U, R=1)
        b = nodal_values(ref.op, ends_ref[j], R=1)
        assert _rel(a, b) < 1e-8, j


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_richardson_outer_iteration(P, prec):
    """Algorithm 1's outer iteration, u <- u + P_CT(b - A u), on the GPU:
    it reaches the true-residual tolerance and the oracle's strip solution
    (1e-8 on the nodal values), and takes at least as many outer steps as
    FGMRES with the same preconditioner."""
    from oracle.solver import StripSolver, nodal_values
    prob = W.free_streaming_1d(L=3, n_strips=1)
    ref = StripSolver(prob, tol=1e-12)
    end_ref = ref.run()[0]
    its = {}
    for method in (P.SGDG_OUTER_RICHARDSON, P.SGDG_OUTER_FGMRES):
        s = P.Solver(prob, precision=P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32, rtol=1e-11,
                     max_outer=300, inner_its=60, inner_rtol=1e-12, cheb_steps=12, outer_method=method)
        s.set_initial()
        st = s.advance_strip()
        assert st.status == 0 and st.rel_residual <= 1e-11, (method, st.rel_residual)
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        assert _rel(nodal_values(ref.op, U, R=1), nodal_values(ref.op, end_ref, R=1)) < 1e-8, method
        its[method] = st.outer_its
        s.close()
    assert its[P.SGDG_OUTER_RICHARDSON] >= its[P.SGDG_OUTER_FGMRES], its


def test_strip_d2_converges_to_tolerance(P):
    prob = W.transport_2d(L=3, sigma=0.1, n_strips=2)
    s = P.Solver(prob, rtol=1e-8, precision=P.SGDG_MIXED_FP32)
    s.set_initial()
    for _ in range(2):
        st = s.advance_strip()
        assert st.rel_residual <= 1e-8 and st.outer_its < 60


def test_config1_run_to_end_time(P):
    """The d = 1 free-streaming configuration (L = 6, dt = 1/32) run through
    all 16 strips to T = 0.5 in FP64: the unique nodal values of U^-(T)
    match the oracle's end state (tests/golden/config1_end_L6.txt, written
    by make_config1_end.py from the oracle's strip solver) within 1e-8 at
    the sampled nodes and in the l2 norm over all nodes.  The oracle's error
    against the exact solution u0(x - v t, v), recorded beside it, is the
    discretisation error both share (3.0e-3 at L = 6)."""
    import os
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "config1_end_L6.txt")
    head, idx, val = {}, [], []
    with open(path) as f:
        for line in f:
            if line.startswith("# ") and len(line.split()) == 3:
                head[line.split()[1]] = float(line.split()[2])
            elif not line.startswith("#"):
                i, v = line.split()
                idx.append(int(i))
                val.append(float(v))
    prob = W.free_streaming_1d(L=6)
    s = P.Solver(prob, rtol=1e-11, restart=30, inner_its=30, inner_rtol=1e-4)
    s.set_initial()
    for j in range(prob.n_strips):
        st = s.advance_strip()
        assert st.rel_residual <= 1e-11, j
    U = np.empty(s.n_spatial)
    s.get_end_value(U, on_device=False)
    nod = _nodal(P, s, U)
    assert nod.size == int(head["n_nodal"])
    assert _rel(nod[idx], np.array(val)) < 1e-8
    assert abs(np.linalg.norm(nod) - head["nodal_l2"]) < 1e-8 * head["nodal_l2"]
    assert 1e-3 < head["exact_rel_l2_error_finest_grid"] < 1e-2
    s.close()
