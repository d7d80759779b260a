"""Batching, CUDA-graph replay and the autotuner (GPU).

* a batch of instances of uneven L applied through one captured CUDA graph
  gives exactly the per-instance applies (same kernels, same order), on the
  first (capture) call and on replays;
* the batched concurrent strip advance reaches the same strip solutions as
  advancing each instance alone;
* autotuning changes only the thread mapping, never the arithmetic: applies
  before and after are identical, and still match the oracle.
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


def _batch_problems():
    return [W.transport_2d(L=3, sigma=0.1), W.transport_2d(L=4, sigma=0.0), W.free_streaming_1d(L=5)]


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batch_graph_apply_equals_single(P, prec):
    solvers = [P.Solver(pr) for pr in _batch_problems()]
    dt = torch.float64 if prec == "fp64" else torch.float32
    pc = P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32
    us = [torch.tensor(W.uniform_vector(s.n_coeffs, seed=40 + k), dtype=dt, device="cuda")
          for k, s in enumerate(solvers)]
    refs = []
    for s, u in zip(solvers, us):
        y = torch.empty_like(u)
        s.apply_operator(u, y, pc)
        refs.append(y.clone())
    b = P.Batch(solvers)
    ys = [torch.full_like(u, float("nan")) for u in us]
    for rep in range(3):          # capture, then replays
        for y in ys:
            y.fill_(float("nan"))
        b.apply(us, ys, pc)
        torch.cuda.synchronize()
        for y, r in zip(ys, refs):
            assert torch.equal(y, r), rep
    b.close()


def test_batch_advance_equals_single(P):
    probs = [W.free_streaming_1d(L=4, n_strips=1), W.transport_2d(L=3, sigma=0.1, n_strips=1)]
    alone = []
    for pr in probs:
        s = P.Solver(pr, rtol=1e-10)
        s.set_initial()
        s.advance_strip()
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        alone.append(U)
    solvers = [P.Solver(pr, rtol=1e-10) for pr in probs]
    for s in solvers:
        s.set_initial()
    b = P.Batch(solvers)
    stats = b.advance()
    for s, st, U0 in zip(solvers, stats, alone):
        assert st.rel_residual <= 1e-10
        U = np.empty(s.n_spatial)
        s.get_end_value(U, on_device=False)
        assert np.array_equal(U, U0)
    b.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_autotune_keeps_results(P, prec):
    from oracle.operator import SparseGridOperator
    prob = W.transport_2d(L=4, sigma=0.1)
    s = P.Solver(prob)
    dt = torch.float64 if prec == "fp64" else torch.float32
    pc = P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32
    u = torch.tensor(W.uniform_vector(s.n_coeffs, seed=5), dtype=dt, device="cuda")
    y0, y1, tmp = torch.empty_like(u), torch.empty_like(u), torch.empty_like(u)
    s.apply_operator(u, y0, pc)
    s.autotune(u, tmp, pc)
    s.apply_operator(u, y1, pc)
    torch.cuda.synchronize()
    assert torch.equal(y0, y1)
    ref = SparseGridOperator(prob).apply(u.double().cpu().numpy())
    err = np.linalg.norm(y1.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert err < (1e-12 if prec == "fp64" else 1e-5)


_SHAPES = [ch | tiled << 4 | pair << 5 | pf << 6
           for pf in (0, 1) for pair in (0, 1) for tiled in (0, 1) for ch in (1, 2, 3, 4, 8)]
_SHAPES += [ch | 1 << 7 for ch in (1, 2, 3, 4, 8)]   # the lattice kernels (2-D lattice x levels)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("case", ["d2_L4", "d1_L6"])
def test_every_launch_shape_gives_the_same_values(P, prec, case):
    """Every launch shape the autotuner can pick (rows per thread, block
    order, paired outputs, L2 prefetch hints, lattice kernels), and a ragged
    rows-per-thread,
    pinned on all sites at once:
    the values are those of the default shapes, bit for bit, and match the
    oracle."""
    from oracle.operator import SparseGridOperator
    prob = W.transport_2d(L=4, sigma=0.1) if case == "d2_L4" else W.free_streaming_1d(L=6)
    s = P.Solver(prob)
    u = W.uniform_vector(s.n_coeffs, seed=6)
    if prec == "bf16":
        u = W.round_to_bf16(u)
    dt = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[prec]
    pc = {"fp64": P.SGDG_FP64, "fp32": P.SGDG_MIXED_FP32, "bf16": P.SGDG_BF16_STORE}[prec]
    ud = torch.tensor(u, dtype=torch.float64, device="cuda").to(dt)
    y0 = torch.empty_like(ud)
    s.apply_operator(ud, y0, pc)
    ref = SparseGridOperator(prob).apply(u)
    tol = {"fp64": 1e-12, "fp32": 1e-5, "bf16": np.sqrt(2 * prob.L + 2) * 2.0 ** -8}[prec]
    for code in _SHAPES:
        s.set_launch_shape(code)
        y = torch.full_like(ud, float("nan"))
        s.apply_operator(ud, y, pc)
        torch.cuda.synchronize()
        assert torch.equal(y, y0), code
        err = np.linalg.norm(y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
        assert err < tol, (code, err)
    s.set_launch_shape(0)
    with pytest.raises(P.SgdgError):
        s.set_launch_shape(16)
    with pytest.raises(P.SgdgError):
        s.set_launch_shape(128)
    s.close()
