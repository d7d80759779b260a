"""The fused branch-A sweep (GPU): per tile, S_b in shared memory, folded into
y and restricted there (sgdg_set_sweep_variant 0) against the unfused
kernels (variant 1, the default) and the oracle.

Both variants compute the same operator with the same sums in FP32 and FP64.
Tolerances: FP64 1e-12 relative against the oracle and 1e-13 between the
variants (max-abs per grid over the grid's largest value); FP32
1e-5 against the oracle; BF16 storage as in test_gpu_bf16 (the fused kernel
keeps S_b in FP32 in shared memory, one rounding fewer per step).  Cases span
1-D, 2-D and periodic meshes, and a d = 2, L = 6 problem whose grids are cut
into many tiles of several shapes (ragged patches at the mesh boundary).
"""
import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

_CASES = {
    "d1_L6": lambda: W.free_streaming_1d(L=6),
    "d2_L3_sigma": lambda: W.transport_2d(L=3, sigma=0.1),
    "d1_periodic_L3": lambda: W.periodic_advection_1d(L=3),
    "d2_landau_L4": lambda: W.landau_4d(L=4),
}


@pytest.fixture(scope="module")
def P():
    import paper_2204_05988_gb300 as P
    P.load_library()
    return P


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _per_grid(offs, y, ref, tol):
    for i in range(len(offs) - 1):
        a, b = y[offs[i]:offs[i + 1]], ref[offs[i]:offs[i + 1]]
        err = np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)
        assert err < tol, (i, err)


def _apply(P, s, u, prec, variant):
    dt = {P.SGDG_FP64: torch.float64, P.SGDG_MIXED_FP32: torch.float32, P.SGDG_BF16_STORE: torch.bfloat16}[prec]
    ud = torch.tensor(u, dtype=torch.float64, device="cuda").to(dt)
    yd = torch.full_like(ud, float("nan"))
    s.set_sweep_variant(variant)
    s.apply_operator(ud, yd, prec)
    torch.cuda.synchronize()
    return yd.double().cpu().numpy()


@pytest.mark.parametrize("name", list(_CASES))
def test_fused_matches_oracle_and_unfused(P, name):
    from oracle.operator import SparseGridOperator
    prob = _CASES[name]()
    s = P.Solver(prob, vlasov_poisson=name.startswith("d2_landau"))
    op = SparseGridOperator(prob)
    u = W.uniform_vector(op.size, seed=17)
    ref = op.apply(u)
    offs = op.offsets
    y_f = _apply(P, s, u, P.SGDG_FP64, 0)
    y_u = _apply(P, s, u, P.SGDG_FP64, 1)
    assert np.all(np.isfinite(y_f))
    assert _rel(y_f, ref) < 1e-12
    _per_grid(offs, y_f, ref, 1e-12)
    _per_grid(offs, y_f, y_u, 1e-13)
    y32 = _apply(P, s, u, P.SGDG_MIXED_FP32, 0)
    assert _rel(y32, ref) < 1e-5
    _per_grid(offs, y32, ref, 1e-5)
    ub = W.round_to_bf16(u)
    yb = _apply(P, s, ub, P.SGDG_BF16_STORE, 0)
    refb = op.apply(ub)
    assert _rel(yb, refb) < np.sqrt(2 * prob.L + 2) * 2.0 ** -8
    s.close()


def test_fused_many_tiles_d2_L6(P):
    """d = 2, L = 6 (3.3 M coefficients): the fused and unfused sweeps agree
    grid by grid (FP64 1e-13, FP32 2e-6 of each grid's largest value), and
    the fused apply runs one branch-A launch per grid and no unfused
    branch-A kernel."""
    prob = W.transport_2d(L=6, sigma=0.1)
    s = P.Solver(prob)
    u = W.uniform_vector(s.n_coeffs, seed=23)
    offs = np.concatenate([[0], np.cumsum([2 * a * b for a, b in s.shapes])])
    for prec, tol in ((P.SGDG_FP64, 1e-13), (P.SGDG_MIXED_FP32, 2e-6)):
        y_u = _apply(P, s, u, prec, 1)
        s.profile(True)
        y_f = _apply(P, s, u, prec, 0)
        st = s.kernel_stats()
        s.profile(False)
        assert st["fused_a"]["launches"] == prob.L + 1
        assert st["s_chain"]["launches"] == 0 and st["restrict_dim2"]["launches"] == 0
        _per_grid(offs, y_f, y_u, tol)
    s.close()
