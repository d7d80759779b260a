"""BF16-storage applies (SGDG_BF16_STORE) against the FP64 oracle (GPU).

The variant stores every grid array of the sweep - the input u, the chain
states S_b, Z_b, Q and the output y - in bfloat16 (8 significant bits, round
to nearest even) and computes in FP32 with FP32 matrix values.  Tolerance,
from the arithmetic: the input is given exactly (values already in bfloat16
on both sides, `round_to_bf16`), FP32 arithmetic adds ~1e-7, and each stored
value carries one relative rounding of at most u_b = 2^-8.  Along the sweep
an output collects at most k = 2L + 2 successive roundings (branch A on grid
i: S_{b,0}, then Z_{b,k} and S_{b,k} per step, 2i + 1 stores; the final
update along dim 1 and the accumulating final along dim 2 add two more).
The worst case k u_b (0.078 at L = 9) is far above what is seen (2.3e-3 to
3.0e-3 at L = 0..6, 2.5e-3 at L = 9): roundings of independent values are
unbiased and add in quadrature, so the test bound is twice the root-sum-square
of k roundings of size u_b / 2, sqrt(2L + 2) u_b (5.5e-3 at L = 0, 1.75e-2
at L = 9), a few times the measured error: a regression by more than that
factor fails.  A diagonal block (no transfers) has two roundings, S_b and
y: sqrt(2) u_b.  Grid by grid, the max-abs error over a component grid
scaled by its largest reference value, allowed twice the l2 bound.
"""
import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U_B = 2.0 ** -8


def bf16_tol(L: int) -> float:
    return np.sqrt(2 * L + 2) * U_B


def _per_grid(op, y, ref, tol):
    for i in range(len(op.grids)):
        a, b = y[op.offsets[i]:op.offsets[i + 1]], ref[op.offsets[i]:op.offsets[i + 1]]
        err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
        assert err < tol, (op.grids[i], err)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _bf16(x: np.ndarray):
    """Device bfloat16 copy of values that are already bfloat16 (exact)."""
    return torch.tensor(x, dtype=torch.float64, device="cuda").to(torch.bfloat16)


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
def test_bf16_apply_operator_parity(P, setups, name):
    prob, s, op = setups(name)
    ub = W.round_to_bf16(W.uniform_vector(op.size, seed=11))
    ref = op.apply(ub)
    ud = _bf16(ub)
    yd = torch.full_like(ud, float("nan"))
    s.apply_operator(ud, yd, P.SGDG_BF16_STORE)
    torch.cuda.synchronize()
    y = yd.double().cpu().numpy()
    assert np.all(np.isfinite(y))
    assert _rel(y, ref) < bf16_tol(prob.L)
    _per_grid(op, y, ref, 2 * bf16_tol(prob.L))


@pytest.mark.parametrize("name", ["d1_L6", "d2_L3_sigma"])
def test_bf16_apply_mass_parity(P, setups, name):
    prob, s, op = setups(name)
    ub = W.round_to_bf16(W.uniform_vector(op.size, seed=12))
    ref = op.apply_mass(ub)
    ud = _bf16(ub)
    yd = torch.empty_like(ud)
    s.apply_mass(ud, yd, P.SGDG_BF16_STORE)
    torch.cuda.synchronize()
    assert _rel(yd.double().cpu().numpy(), ref) < bf16_tol(prob.L)


@pytest.mark.parametrize("name", ["d1_L6", "d2_L3_sigma"])
def test_bf16_apply_diag_parity(P, setups, name):
    prob, s, op = setups(name)
    L = prob.L
    for (l1, l2) in [(0, L), (L, 0), (L // 2, L - L // 2), (0, L - 1)]:
        n1, n2 = op.grid_shape(l1, l2)
        ub = W.round_to_bf16(W.uniform_vector(n1 * n2 * 2, seed=13 + l1))
        ref = op.apply_diag(l1, l2, ub.reshape(n1, n2, 2)).ravel()
        ud = _bf16(ub)
        yd = torch.empty_like(ud)
        s.apply_diag(l1, l2, ud, yd, P.SGDG_BF16_STORE)
        torch.cuda.synchronize()
        assert _rel(yd.double().cpu().numpy(), ref) < np.sqrt(2.0) * U_B, (l1, l2)


@pytest.mark.parametrize("name", ["d1_L6", "d2_L3_sigma"])
def test_bf16_host_buffer_apply(P, setups, name):
    """The host-buffer apply rounds the FP64 input to bfloat16 on the device;
    for input already in bfloat16 it returns the device apply's values."""
    prob, s, op = setups(name)
    ub = W.round_to_bf16(W.uniform_vector(op.size, seed=14))
    hu = torch.tensor(ub, dtype=torch.float64).pin_memory()
    hy = torch.full((op.size,), float("nan"), dtype=torch.float64).pin_memory()
    s.apply_operator_host(hu, hy, P.SGDG_BF16_STORE)
    ud = _bf16(ub)
    yd = torch.empty_like(ud)
    s.apply_operator(ud, yd, P.SGDG_BF16_STORE)
    torch.cuda.synchronize()
    assert torch.equal(hy, yd.double().cpu())


def test_bf16_batch_graph_and_autotune(P):
    """Batch graph replays and the autotuner's launch shapes give the plain
    BF16 applies' values bit for bit."""
    probs = [W.transport_2d(L=3, sigma=0.1), W.transport_2d(L=4, sigma=0.0), W.free_streaming_1d(L=5)]
    solvers = [P.Solver(pr) for pr in probs]
    us = [_bf16(W.round_to_bf16(W.uniform_vector(s.n_coeffs, seed=40 + k))) for k, s in enumerate(solvers)]
    refs = []
    for s, u in zip(solvers, us):
        y = torch.empty_like(u)
        s.apply_operator(u, y, P.SGDG_BF16_STORE)
        refs.append(y.clone())
    b = P.Batch(solvers)
    ys = [torch.empty_like(u) for u in us]
    for rep in range(2):
        b.apply(us, ys, P.SGDG_BF16_STORE)
        torch.cuda.synchronize()
        for y, r in zip(ys, refs):
            assert torch.equal(y, r), rep
    b.close()
    s, u = solvers[1], us[1]
    tmp, y1 = torch.empty_like(u), torch.empty_like(u)
    s.autotune(u, tmp, P.SGDG_BF16_STORE)
    s.apply_operator(u, y1, P.SGDG_BF16_STORE)
    torch.cuda.synchronize()
    assert torch.equal(y1, refs[1])


def test_bf16_is_not_a_solver_precision(P):
    with pytest.raises(P.SgdgError):
        P.Solver(W.free_streaming_1d(L=2), precision=P.SGDG_BF16_STORE)
