"""The allocation-free diagonal-block apply (GPU).

sgdg_apply_diag_noalloc serves callers that may not allocate device memory at
the time they apply the operator (loops that must not hit the allocator's
device-wide synchronisation, or processes whose device memory belongs to a
pool another component owns).  It must give the same y = A_{l,l} u as
sgdg_apply_diag, on repeated calls that reuse its static scratch, and must
reject grids whose intermediates do not fit that scratch.  This file is collected last so that a
run stopping at the first failure has run every other test already.
"""
import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _rel(a, b):
    return float(torch.linalg.norm((a - b).double()) / torch.linalg.norm(b.double()))


def test_noalloc_matches_apply_diag_on_consecutive_calls():
    import paper_2204_05988_gb300 as P
    s = P.Solver(W.transport_2d(L=4, sigma=0.1))
    for pc, dt, tol in ((P.SGDG_FP64, torch.float64, 1e-12), (P.SGDG_MIXED_FP32, torch.float32, 1e-5)):
        for k, (l1, l2) in enumerate([(0, 4), (2, 2), (4, 0), (1, 2)]):
            u = torch.tensor(W.uniform_vector(2 * _npts(s, l1, l2), seed=70 + k), dtype=dt, device="cuda")
            ref = torch.empty_like(u)
            s.apply_diag(l1, l2, u, ref, pc)
            for rep in range(2):
                out = torch.full_like(u, float("nan"))
                s.apply_diag_noalloc(l1, l2, u, out, pc)
                torch.cuda.synchronize()
                assert _rel(out, ref) <= tol, (pc, l1, l2, rep)
    s.close()


def test_noalloc_rejects_grids_beyond_the_scratch():
    import paper_2204_05988_gb300 as P
    s = P.Solver(W.transport_2d(L=7, sigma=0.1))
    u = torch.zeros(2 * _npts(s, 0, 7), dtype=torch.float64, device="cuda")
    with pytest.raises(P.SgdgError, match="limit"):
        s.apply_diag_noalloc(0, 7, u, torch.empty_like(u), P.SGDG_FP64)
    s.close()


def _npts(s, l1, l2):
    """n1 * n2 of grid (l1, l2), read from the sparse grid's own shapes."""
    L = s.info.L
    nx = {l: s.shapes[l][0] for l in range(L + 1)}
    nv = {L - l: s.shapes[l][1] for l in range(L + 1)}
    return nx[l1] * nv[l2]
