"""Learned warm start on the GPU.

* coarse full-grid values of sparse-grid functions match the oracle's
  (injection / prolongation are exact) and sgdg_add_coarse round-trips;
* the library's BF16 MLP gradients match the FP64 oracle MLP evaluated on the
  same (bf16-rounded) weights and inputs, within the bf16 tolerance;
* training on strip pairs from the plain solver lowers the loss; the trained
  network's guess (extrapolation + learned coarse correction, warm start 2)
  starts closer than the previous-solution guess and the solver still reaches
  the tolerance from every guess - the converged residual decides; the
  comparison with the extrapolation (the method without the network) is
  reported per strip.
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


def test_coarse_values_parity_and_roundtrip(P):
    from oracle.operator import SparseGridOperator
    from oracle.solver import coarse_values
    prob = W.landau_4d(L=4)
    op = SparseGridOperator(prob)
    s = P.Solver(prob, vlasov_poisson=True)
    u = W.uniform_vector(op.size, seed=9)
    for (lx, lv) in [(2, 2), (0, 4), (4, 1), (3, 3)]:
        nx, nv = op.hx.levels[lx].n, op.hv.levels[lv].n
        ref2 = coarse_values(op, u, 2, lx, lv)
        out = torch.empty(nx * nv * 2, dtype=torch.float64, device="cuda")
        s.coarse_values(torch.tensor(u, device="cuda"), 2, lx, lv, out)
        torch.cuda.synchronize()
        assert np.abs(out.cpu().numpy() - ref2).max() < 1e-12 * np.abs(ref2).max(), (lx, lv)
        U = u[: op.size // 2]
        ref1 = coarse_values(op, U, 1, lx, lv)
        out1 = torch.empty(nx * nv, dtype=torch.float64, device="cuda")
        s.coarse_values(torch.tensor(U, device="cuda"), 1, lx, lv, out1)
        torch.cuda.synchronize()
        assert np.abs(out1.cpu().numpy() - ref1).max() < 1e-12 * np.abs(ref1).max(), (lx, lv)
    # the view of a difference (the warm start's features and targets)
    a, b = W.uniform_vector(op.size, seed=10), W.uniform_vector(op.size, seed=11)
    ref = coarse_values(op, a - b, 2, 2, 2)
    out = torch.empty(ref.size, dtype=torch.float64, device="cuda")
    s.coarse_diff(torch.tensor(a, device="cuda"), torch.tensor(b, device="cuda"), 2, 2, 2, out)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()
    # round trip: a coarse function added to zero evaluates back to itself
    lx, lv = 2, 2
    nx, nv = op.hx.levels[lx].n, op.hv.levels[lv].n
    c = torch.tensor(W.uniform_vector(nx * nv * 2, seed=3), device="cuda")
    z = torch.zeros(op.size, dtype=torch.float64, device="cuda")
    s.add_coarse(c, lx, lv, z)
    back = torch.empty_like(c)
    s.coarse_values(z, 2, lx, lv, back)
    torch.cuda.synchronize()
    assert torch.allclose(back, c, rtol=0, atol=1e-14)


def test_mlp_gradients_match_oracle(P):
    from oracle.mlp import loss_and_grad, to_bf16
    n_in, w, n_out, B = 64, 32, 48, 20
    net = P.Mlp(n_in, w, n_out, max_batch=32, seed=5)
    net.set_scaling(0.5, 2.0)
    rng = np.random.default_rng(2)
    x = rng.normal(size=(B, n_in))
    t = rng.normal(size=(B, n_out)) * 0.3
    g, loss = net.gradients(torch.tensor(x, device="cuda"), torch.tensor(t, device="cuda"), B)
    p = net.get_params().astype(np.float64)
    # the GPU multiplies bf16 weights and bf16 (scaled) inputs
    from oracle.mlp import unpack
    pw = p.copy()
    o = 0
    for fi, fo in [(n_in, w), (w, w), (w, n_out)]:
        pw[o:o + fi * fo] = to_bf16(p[o:o + fi * fo])
        o += fi * fo + fo
    xs = to_bf16(x * 0.5) / 0.5
    loss_ref, g_ref = loss_and_grad(pw, xs, t, n_in, w, n_out, in_scale=0.5, out_scale=2.0)
    assert abs(loss - loss_ref) < 2e-2 * loss_ref
    assert np.linalg.norm(g - g_ref) < 3e-2 * np.linalg.norm(g_ref)


def test_training_and_learned_guess(P, record_property):
    """Train on strip pairs of the plain solver, then solve a held-out problem
    from three guesses: the previous solution, the extrapolation 2 u_{j-1} -
    u_{j-2} (the method without the network) and the learned guess
    (extrapolation + the network's coarse correction).  Asserted: training
    lowers the loss, every guess reaches the tolerance (the converged residual
    decides), and the learned guess starts closer than the previous solution.
    Reported against the extrapolation, per strip: the initial residual, the
    outer iterations and the time.  So far the network lowers the initial
    residual below the extrapolation's but does not lower the iteration count
    (at L = 6 on the Landau problem: 118 outer iterations against 83 for 16
    strips) - the gain over the method without it is not shown."""
    from paper_2204_05988_gb300 import warmstart as WS
    probs = [W.landau_4d(L=3, alpha=a, phase=ph, dt=0.25) for a, ph in [(0.01, 0.0), (0.02, 1.0), (0.015, 2.0)]]
    pairs = WS.collect(probs, n_strips=6, lx=2, lv=1)
    assert len(pairs.x) == 12
    net, losses = WS.train(pairs, width=64, steps=200, batch=8, lr=1e-3)
    assert np.mean(losses[-20:]) < 0.7 * np.mean(losses[:5])
    res = WS.evaluate(lambda: W.landau_4d(L=3, alpha=0.012, phase=0.5, dt=0.25), net, n_strips=5, lx=2, lv=1)
    for k in res:
        for its, r0, t, rel in res[k]:
            assert rel <= 1e-8, k
    # from strip 2 on the learned guess starts closer than the previous solution
    r_prev = np.mean([r[1] for r in res["previous"][2:]])
    r_learn = np.mean([r[1] for r in res["learned"][2:]])
    assert r_learn < r_prev, (r_learn, r_prev)
    # against the method without the network (extrapolation): reported
    for k in ("extrapolated", "learned"):
        record_property(f"{k}_initial_residual", [r[1] for r in res[k][2:]])
        record_property(f"{k}_outer_its", [r[0] for r in res[k][2:]])
        record_property(f"{k}_seconds", [round(r[2], 4) for r in res[k][2:]])
    print("learned vs extrapolated, strips 3-5: initial residual",
          [f"{a[1]:.2e}/{b[1]:.2e}" for a, b in zip(res["learned"][2:], res["extrapolated"][2:])],
          "outer its", [(a[0], b[0]) for a, b in zip(res["learned"][2:], res["extrapolated"][2:])])
