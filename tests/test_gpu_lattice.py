"""The lattice kernels of 2-D x levels (sweep variant 1, the default) against
the generic kernels (variant 2) and the oracle.

On x levels that are structured lattices (the transport workloads' meshes:
non-periodic, every cell cut along the (1, 1) diagonal) the pattern rows are
held in stencil-slot order; the final update along dim 1 slides a register
window along the lattice rows, and the mode-A chain step (FP32 and BF16
storage) runs along them too, reusing each thread's factor row and a window
of the coarse states it prolongs.  The autotuner picks them per launch site where
they are faster (launch-shape bit 7); the tests pin them.  Both paths form
the same sums in the same order;
they are compared at 1e-14 (FP64) and 1e-6 (FP32) relative, and the default
path against the oracle at the parity tolerances (1e-12, 1e-5).  A periodic
x mesh (the Landau workload) is not a lattice in this sense (its rows wrap)
and keeps the generic layout.
"""
import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import paper_2204_05988_gb300 as P
    P.load_library()
    return P


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_lattice_levels_detected(P):
    s = P.Solver(W.transport_2d(L=3, sigma=0.1))
    assert s.info.lattice_x_levels == 4
    s.close()
    s = P.Solver(W.landau_4d(L=3), vlasov_poisson=True)
    assert s.info.lattice_x_levels == 0
    s.close()
    s = P.Solver(W.free_streaming_1d(L=3))
    assert s.info.lattice_x_levels == 0
    s.close()


@pytest.mark.parametrize("L", [2, 4])
def test_lattice_final_equals_generic_and_oracle(P, L):
    from oracle.operator import SparseGridOperator
    prob = W.transport_2d(L=L, sigma=0.1)
    op = SparseGridOperator(prob)
    s = P.Solver(prob)
    u = W.uniform_vector(op.size, seed=71)
    ref = op.apply(u)
    out = {}
    for variant in (1, 2):
        s.set_sweep_variant(variant)
        s.set_launch_shape(0x80 | 8)   # lattice kernels (variant 1) where the levels allow them
        for prec, dt in (("fp64", torch.float64), ("fp32", torch.float32)):
            ud = torch.tensor(u, device="cuda").to(dt)
            yd = torch.full_like(ud, float("nan"))
            s.apply_operator(ud, yd, P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32)
            torch.cuda.synchronize()
            out[(variant, prec)] = yd.double().cpu().numpy()
    assert _rel(out[(1, "fp64")], out[(2, "fp64")]) < 1e-14
    assert _rel(out[(1, "fp32")], out[(2, "fp32")]) < 1e-6
    assert _rel(out[(1, "fp64")], ref) < 1e-12
    assert _rel(out[(1, "fp32")], ref) < 1e-5
    for i in range(len(op.grids)):
        a, b = out[(1, "fp64")][op.offsets[i]:op.offsets[i + 1]], ref[op.offsets[i]:op.offsets[i + 1]]
        assert np.abs(a - b).max() < 1e-12 * np.abs(b).max(), i
    s.close()


def test_lattice_runs_of_4_and_8_agree(P):
    """Every run length (final: 4 or 8 vertices per thread, chain step: 2 or
    4) gives the same values, bit for bit."""
    prob = W.transport_2d(L=4, sigma=0.1)
    s = P.Solver(prob)
    u = torch.tensor(W.uniform_vector(s.n_coeffs, seed=72), device="cuda").float()
    ys = []
    for code in (1, 2, 4, 8):
        s.set_launch_shape(0x80 | code)
        y = torch.full_like(u, float("nan"))
        s.apply_operator(u, y, P.SGDG_MIXED_FP32)
        ys.append(y)
    torch.cuda.synchronize()
    for y in ys[1:]:
        assert torch.equal(ys[0], y)
    s.close()
