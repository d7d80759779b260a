"""GPU parity at d = 3 (6-D phase space): Kuhn cube meshes refined after Bey,
15-entry P1 rows, branch B of the sweep through full-size states (the
restriction-factor products would have 65-entry rows).  The CUDA path is
called through the C ABI and compared with the FP64 oracle.

Tolerances as for d = 1, 2 (test_gpu_parity): applies 1e-12 relative in FP64
and 1e-5 in FP32, per grid as well as over the vector; strip solutions 1e-8
on the canonical nodal values.

At the full size of the d = 3 workload (L = 7, 130,648,356 coefficients) the
oracle cannot assemble the finest factors (12.6 M tetrahedra).  There the
mass apply is checked element by element against a closed form, and the
FP32 operator apply against the FP64 one:
  * every hat function of a level-l Kuhn lattice (h = box edge / 2^l)
    integrates to h^3 n / 24, where n counts the tetrahedra around the vertex
    (6 in a cube whose main diagonal starts or ends at the vertex, 2 in the
    other cubes it is a corner of); with u = 1 on every grid the function is
    L + 1 everywhere, so (Id_t (x) M_sg) u at row (l, k1, k2, s) is
    (L + 1) int phi_k1 int psi_k2.
"""
import numpy as np
import pytest

import sgdg_workloads as W
from test_oracle_3d import kuhn_hat_integrals

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _per_grid(offsets, y, ref, tol):
    for i in range(len(offsets) - 1):
        a, b = y[offsets[i]:offsets[i + 1]], ref[offsets[i]:offsets[i + 1]]
        err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
        assert err < tol, (i, err)


@pytest.fixture(scope="module")
def P():
    import paper_2204_05988_gb300 as P
    P.load_library()
    return P


@pytest.fixture(scope="module")
def setups(P):
    from oracle.operator import SparseGridOperator
    cache = {}

    def get(L):
        if L not in cache:
            prob = W.transport_3d(L=L)
            cache[L] = (prob, P.Solver(prob), SparseGridOperator(prob))
        return cache[L]
    return get


@pytest.mark.parametrize("L", [0, 1, 3])
def test_layout_matches_oracle(setups, L):
    prob, s, op = setups(L)
    assert s.n_coeffs == op.size
    assert s.shapes == [tuple(x) for x in op.shape]


@pytest.mark.parametrize("L", [0, 1, 3])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_operator_parity_3d(P, setups, L, prec):
    prob, s, op = setups(L)
    u = W.uniform_vector(op.size, seed=41 + L)
    ref = op.apply(u)
    dt = torch.float64 if prec == "fp64" else torch.float32
    ud = torch.tensor(u, dtype=dt, device="cuda")
    yd = torch.full_like(ud, float("nan"))
    s.apply_operator(ud, yd, P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32)
    torch.cuda.synchronize()
    y = yd.double().cpu().numpy()
    tol = 1e-12 if prec == "fp64" else 1e-5
    assert _rel(y, ref) < tol
    _per_grid(op.offsets, y, ref, tol)


def test_apply_operator_bf16_3d(P, setups):
    """BF16 storage on the bfloat16-rounded input, at the bound of the
    root-sum-square of the roundings, sqrt(2L + 2) 2^-8 (test_gpu_bf16)."""
    L = 3
    prob, s, op = setups(L)
    u = W.round_to_bf16(W.uniform_vector(op.size, seed=47))
    ref = op.apply(u)
    ud = torch.tensor(u, device="cuda").to(torch.bfloat16)
    yd = torch.empty_like(ud)
    s.apply_operator(ud, yd, P.SGDG_BF16_STORE)
    torch.cuda.synchronize()
    assert _rel(yd.double().cpu().numpy(), ref) < np.sqrt(2 * L + 2) * 2.0 ** -8


def test_apply_mass_and_diag_3d(P, setups):
    L = 3
    prob, s, op = setups(L)
    u = W.uniform_vector(op.size, seed=43)
    ref = op.apply_mass(u)
    ud = torch.tensor(u, device="cuda")
    yd = torch.empty_like(ud)
    s.apply_mass(ud, yd, P.SGDG_FP64)
    torch.cuda.synchronize()
    y = yd.cpu().numpy()
    assert _rel(y, ref) < 1e-12
    _per_grid(op.offsets, y, ref, 1e-12)
    for (l1, l2) in [(0, L), (L, 0), (1, 2), (2, 0)]:
        n1, n2 = op.grid_shape(l1, l2)
        v = W.uniform_vector(n1 * n2 * 2, seed=44 + l1)
        rd = op.apply_diag(l1, l2, v.reshape(n1, n2, 2)).ravel()
        vd = torch.tensor(v, device="cuda")
        wd = torch.empty_like(vd)
        s.apply_diag(l1, l2, vd, wd, P.SGDG_FP64)
        torch.cuda.synchronize()
        assert _rel(wd.cpu().numpy(), rd) < 1e-12, (l1, l2)


def test_ct_preconditioner_3d(P):
    """Algorithm 1's preconditioner with (nearly) exact component solves."""
    from oracle.operator import SparseGridOperator
    from oracle.solver import ComponentSolver, ct_precondition
    prob = W.transport_3d(L=2)
    s = P.Solver(prob, inner_its=60, inner_rtol=1e-13, cheb_steps=16)
    op = SparseGridOperator(prob)
    comp = ComponentSolver(op, tol=1e-13)
    r = W.uniform_vector(op.size, seed=45)
    ref = ct_precondition(op, comp, r)
    rd = torch.tensor(r, device="cuda")
    zd = torch.empty_like(rd)
    s.ct_precondition(rd, zd)
    torch.cuda.synchronize()
    assert _rel(zd.cpu().numpy(), ref) < 1e-9
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_strip_parity_3d(P, prec):
    """The first strip of the d = 3 workload at L = 2 against the oracle's
    strip solution, 1e-8 on the canonical nodal values."""
    from oracle.solver import StripSolver, nodal_values
    prob = W.transport_3d(L=2, n_strips=1)
    ref = StripSolver(prob, tol=1e-12)
    end_ref = ref.run()[0]
    s = P.Solver(prob, precision=P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32, rtol=1e-11,
                 restart=30, inner_its=30, inner_rtol=1e-4)
    s.set_initial()
    st = s.advance_strip()
    assert st.status == 0 and st.rel_residual <= 1e-11
    U = np.empty(s.n_spatial)
    s.get_end_value(U, on_device=False)
    assert _rel(nodal_values(ref.op, U, R=1), nodal_values(ref.op, end_ref, R=1)) < 1e-8
    s.close()


@pytest.fixture(scope="module")
def full3d(P):
    L = 7
    s = P.Solver(W.transport_3d(L=L))
    yield L, s
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_mass_closed_form_at_full_size(P, full3d, prec):
    L, s = full3d
    dt = torch.float64 if prec == "fp64" else torch.float32
    ud = torch.ones(s.n_coeffs, dtype=dt, device="cuda")
    yd = torch.full_like(ud, float("nan"))
    s.apply_mass(ud, yd, P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "fp64" else 1e-5
    for i, ((n1, n2), off) in enumerate(zip(s.shapes, s.offsets)):
        ref = (L + 1) * np.outer(kuhn_hat_integrals(i, 1.0), kuhn_hat_integrals(L - i, 2.0))
        got = yd[off:off + 2 * n1 * n2].view(n1, n2, 2).double().cpu().numpy()
        for t in range(2):
            err = np.abs(got[:, :, t] - ref).max() / ref.max()
            assert err < tol, (i, t, err)


def test_fp32_apply_against_fp64_at_full_size(P, full3d):
    L, s = full3d
    u = torch.tensor(W.uniform_vector(s.n_coeffs, seed=49), device="cuda")
    y64 = torch.full_like(u, float("nan"))
    s.apply_operator(u, y64, P.SGDG_FP64)
    u32 = u.float()
    y32 = torch.full_like(u32, float("nan"))
    s.autotune(u32, y32, P.SGDG_MIXED_FP32)
    y32.fill_(float("nan"))
    s.apply_operator(u32, y32, P.SGDG_MIXED_FP32)
    torch.cuda.synchronize()
    assert torch.isfinite(y64).all() and torch.isfinite(y32).all()
    a, b = y32.double(), y64
    assert float(torch.linalg.norm(a - b) / torch.linalg.norm(b)) < 1e-5
    for (n1, n2), off in zip(s.shapes, s.offsets):
        ga, gb = a[off:off + 2 * n1 * n2], b[off:off + 2 * n1 * n2]
        assert float((ga - gb).abs().max() / gb.abs().max()) < 1e-5
