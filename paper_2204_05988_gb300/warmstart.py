"""Learned warm start for the strip solves (library-driven).

Non-learned guesses for strip j (kept as the fallback): the previous strip's
solution u_{j-1} (warm start 1) and its linear extrapolation
g_j = 2 u_{j-1} - u_{j-2} (warm start 3).  The learned guess adds a coarse
correction to g_j: a 3-layer MLP (the library's BF16 tensor-core kernels)
maps coarse features - the values of the last change u_{j-1} - u_{j-2} at
the nodes of the coarse full grid (lx, lv), both time coefficients - to the
values there of u_j - g_j (both time coefficients); the prediction is
added to g_j as a P1 function on component grid (lx, L-lx).  Every step runs
in the library: coarse views (sgdg_coarse_values / sgdg_add_coarse), the
extrapolation (sgdg_extrapolated_guess), the network (sgdg_mlp_*) and the
solve (sgdg_set_guess + warm start 2).  The converged residual decides: the
solver runs to the same tolerance from any guess.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field
from typing import List

from . import SGDG_MIXED_FP32, Mlp, Solver


@dataclass
class Pairs:
    x: List = field(default_factory=list)   # features (device tensors [n_in])
    y: List = field(default_factory=list)   # targets  (device tensors [n_out])


def coarse_dims(solver: Solver, lx: int, lv: int):
    L = solver.info.L
    nx = solver.shapes[lx][0]
    nv = {L - l: solver.shapes[l][1] for l in range(L + 1)}[lv]
    return nx, nv


def _solver(prob, kw):
    d = dict(precision=SGDG_MIXED_FP32, rtol=1e-8, inner_its=30, inner_rtol=1e-4)
    d.update(kw or {})
    return Solver(prob, vlasov_poisson=True, **d)


def features(solver: Solver, lx: int, lv: int, g):
    """coarse (g - u_{j-1}) (nx nv 2) for the next strip, g the extrapolated
    guess (g - u_{j-1} = u_{j-1} - u_{j-2}, the last change).  The end value
    U^-_{j-1} itself is left out: it is dominated by the part of the state
    that does not change (the Maxwellian of the Landau problem), which a
    single input scale would let swamp the changes."""
    import torch
    nx, nv = coarse_dims(solver, lx, lv)
    u = torch.empty(solver.n_coeffs, dtype=torch.float64, device="cuda")
    solver.get_solution(u, on_device=True)
    f = torch.empty(nx * nv * 2, dtype=torch.float64, device="cuda")
    solver.coarse_diff(g, u, 2, lx, lv, f)
    return f


def collect(problems, n_strips: int, lx: int = 2, lv: int = 2, solver_kw=None) -> Pairs:
    """Pairs (features before strip j, coarse values of u_j - g_j) from runs of
    the plain solver with the extrapolated guess, for strips j >= 2."""
    import torch
    pairs = Pairs()
    for prob in problems:
        s = _solver(prob, solver_kw)
        s.set_warm_start(3)
        s.set_initial()
        s.field_update(0)
        nx, nv = coarse_dims(s, lx, lv)
        g = torch.empty(s.n_coeffs, dtype=torch.float64, device="cuda")
        for j in range(n_strips):
            f = None
            if j >= 2:
                s.extrapolated_guess(g)
                f = features(s, lx, lv, g)
            s.advance_strip()
            if f is not None:
                u = torch.empty_like(g)
                s.get_solution(u, on_device=True)
                t = torch.empty(nx * nv * 2, dtype=torch.float64, device="cuda")
                s.coarse_diff(u, g, 2, lx, lv, t)
                pairs.x.append(f)
                pairs.y.append(t)
            s.field_update(0)
        s.close()
    return pairs


def train(pairs: Pairs, width: int = 256, steps: int = 400, batch: int = 32, lr: float = 1e-3, seed: int = 0):
    """Trains the MLP on the GPU with the library's forward/backward/Adam kernels."""
    import torch
    X = torch.stack(pairs.x)
    Y = torch.stack(pairs.y)
    n, n_in = X.shape
    n_out = Y.shape[1]
    net = Mlp(n_in, width, n_out, max_batch=batch, seed=seed)
    net.set_scaling(1.0 / float(X.abs().max()), 1.0 / float(Y.abs().max()))
    gen = torch.Generator(device="cpu").manual_seed(seed)
    losses = []
    for _ in range(steps):
        idx = torch.randperm(n, generator=gen)[:batch].cuda()
        xb = X.index_select(0, idx).contiguous()
        yb = Y.index_select(0, idx).contiguous()
        losses.append(net.train_step(xb, yb, xb.shape[0], lr))
    return net, losses


def set_learned_guess(solver: Solver, net: Mlp, lx: int, lv: int):
    """Extrapolated guess + MLP correction, installed as warm start 2."""
    import torch
    nx, nv = coarse_dims(solver, lx, lv)
    g = torch.empty(solver.n_coeffs, dtype=torch.float64, device="cuda")
    solver.extrapolated_guess(g)
    f = features(solver, lx, lv, g)
    corr = torch.empty(nx * nv * 2, dtype=torch.float64, device="cuda")
    net.forward(f, 1, corr)
    solver.add_coarse(corr, lx, lv, g)
    solver.set_guess(g)
    solver.set_warm_start(2)


def evaluate(problem_fn, net: Mlp, n_strips: int, lx: int = 2, lv: int = 2, solver_kw=None):
    """Three solvers in lockstep on the same problem: previous solution,
    extrapolation, learned.  Returns per strip (outer its, initial residual,
    seconds, final residual) for each."""
    names = ("previous", "extrapolated", "learned")
    sv = {k: _solver(problem_fn(), solver_kw) for k in names}
    sv["previous"].set_warm_start(1)
    sv["extrapolated"].set_warm_start(3)
    sv["learned"].set_warm_start(3)
    for s in sv.values():
        s.set_initial()
        s.field_update(0)
    res = {k: [] for k in names}
    for j in range(n_strips):
        for k in names:
            s = sv[k]
            t0 = time.perf_counter()
            if k == "learned" and j >= 2:
                set_learned_guess(s, net, lx, lv)
            st = s.advance_strip()
            dt = time.perf_counter() - t0
            res[k].append((st.outer_its, st.initial_rel_residual, dt, st.rel_residual))
            s.field_update(0)
    for s in sv.values():
        s.close()
    return res
