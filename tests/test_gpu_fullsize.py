"""Full-size parity: the d = 2, L = 9 operator apply (123,180,372 coefficients,
the size and launch shapes the benchmark times) against the oracle's outputs
at sampled positions (GPU).

The oracle cannot apply the whole operator at this size; its sampled apply
(`oracle.operator.apply_rows`, rows of the projected factors from the
finest-level matrices) wrote `tests/golden/apply_samples_transport2d_L9.txt`
through `tests/golden/make_apply_samples.py`.  Positions: the last row and
column of every grid (the ragged edges of any tiling) and one seeded interior
position per grid.  Tolerances as in the small-size parity tests: 1e-12 FP64,
1e-5 FP32 (after autotuning, the benchmark's launch shapes), and for BF16
storage sqrt(2L + 2) 2^-8 on the bfloat16-rounded input (derivation in
test_gpu_bf16).
"""
import os

import numpy as np
import pytest

import sgdg_workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

L = 9
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", f"apply_samples_transport2d_L{L}.txt")
INPUT_SEED = 29


def _golden():
    rows, y, yb = [], [], []
    with open(GOLDEN) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            p = line.split()
            rows.append((int(p[0]), int(p[1]), int(p[2])))
            y.append([float(p[3]), float(p[4])])
            yb.append([float(p[5]), float(p[6])])
    return rows, np.array(y), np.array(yb)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def fullsize():
    import paper_2204_05988_gb300 as P
    P.load_library()
    rows, y, yb = _golden()
    s = P.Solver(W.transport_2d(L=L, sigma=0.1))
    u = W.uniform_vector(s.n_coeffs, seed=INPUT_SEED)
    idx = []
    for (i, k1, k2) in rows:
        (n1, n2), off = s.shapes[i], s.offsets[i]
        assert 0 <= k1 < n1 and 0 <= k2 < n2
        base = off + (k1 * n2 + k2) * 2
        idx += [base, base + 1]
    yield P, s, u, torch.tensor(idx, device="cuda"), y.ravel(), yb.ravel()
    s.close()


def test_fp64_apply_at_full_size(fullsize):
    P, s, u, idx, y, _ = fullsize
    ud = torch.tensor(u, device="cuda")
    yd = torch.full_like(ud, float("nan"))
    s.apply_operator(ud, yd, P.SGDG_FP64)
    got = yd[idx].cpu().numpy()
    assert torch.isfinite(yd).all()
    assert _rel(got, y) < 1e-12


def test_fp32_autotuned_apply_at_full_size(fullsize):
    P, s, u, idx, y, _ = fullsize
    ud = torch.tensor(u, device="cuda").float()
    yd = torch.full_like(ud, float("nan"))
    s.autotune(ud, yd, P.SGDG_MIXED_FP32)
    yd.fill_(float("nan"))
    s.apply_operator(ud, yd, P.SGDG_MIXED_FP32)
    got = yd[idx].double().cpu().numpy()
    assert torch.isfinite(yd).all()
    assert _rel(got, y) < 1e-5


def test_bf16_autotuned_apply_at_full_size(fullsize):
    P, s, u, idx, _, yb = fullsize
    ud = torch.tensor(W.round_to_bf16(u), device="cuda").to(torch.bfloat16)
    yd = torch.full_like(ud, float("nan"))
    s.autotune(ud, yd, P.SGDG_BF16_STORE)
    yd.fill_(float("nan"))
    s.apply_operator(ud, yd, P.SGDG_BF16_STORE)
    got = yd[idx].double().cpu().numpy()
    assert torch.isfinite(yd).all()
    assert _rel(got, yb) < np.sqrt(2 * L + 2) * 2.0 ** -8
