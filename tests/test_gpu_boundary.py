"""The C ABI's state and failure paths (GPU).

* Checkpoint and restore at a strip boundary (the strip scheme of Sect. 2):
  a run interrupted after strip 2, restored into a fresh handle and continued,
  gives the strips an uninterrupted run gives, bit for bit - for the plain
  transport solver with the extrapolated warm start and for the
  Vlasov-Poisson solver whose field is iterated within each strip (Sect. 5.3).
  A checkpoint of another problem is refused; a corrupted or truncated one
  is refused (SGDG_EIO) before the handle's state changes.
* The device-memory budget: a handle whose set-up needs more than
  hbm_budget_bytes is refused with SGDG_ENOMEM; one that fits creates.
* Failures injected on the host: NaN initial data gives SGDG_ENAN; an outer
  iteration cap of 1 gives SGDG_ENOCONV with the statistics filled; a level
  beyond the supported range gives SGDG_EINVAL.
"""
import os

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


def _end(s):
    U = np.empty(s.n_spatial)
    s.get_end_value(U, on_device=False)
    return U


def _sol(s):
    u = np.empty(s.n_coeffs)
    s.get_solution(u, on_device=False)
    return u


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_checkpoint_resume_is_bit_identical(P, tmp_path, prec):
    prob = W.transport_2d(L=3, sigma=0.1, n_strips=4)
    pr = P.SGDG_FP64 if prec == "fp64" else P.SGDG_MIXED_FP32
    kw = dict(precision=pr, rtol=1e-9, restart=20, inner_its=12, inner_rtol=1e-2)
    a = P.Solver(prob, **kw)
    a.set_warm_start(3)
    a.set_initial()
    ends_a = []
    path = str(tmp_path / "strip2.ckpt")
    for j in range(4):
        a.advance_strip()
        ends_a.append(_end(a))
        if j == 1:
            a.checkpoint(path)
    sol_a = _sol(a)
    a.close()
    b = P.Solver(prob, **kw)
    b.restore(path)
    assert np.array_equal(_end(b), ends_a[1])
    for j in range(2, 4):
        b.advance_strip()
        assert np.array_equal(_end(b), ends_a[j]), j
    assert np.array_equal(_sol(b), sol_a)
    b.close()


def test_checkpoint_resume_vlasov_poisson(P, tmp_path):
    kw = dict(precision=P.SGDG_MIXED_FP32, rtol=1e-9, inner_its=30, inner_rtol=1e-4, vlasov_poisson=True)
    mk = lambda: W.landau_4d(L=3, dt=0.25, n_strips=4)
    a = P.Solver(mk(), **kw)
    a.set_initial()
    path = str(tmp_path / "vp.ckpt")
    ends, rhos = [], []
    for j in range(4):
        a.advance_strip_vp(tol=1e-6, max_fp=6)
        ends.append(_end(a))
        rhos.append(a.density_potential()[0].copy())
        if j == 1:
            a.checkpoint(path)
    a.close()
    b = P.Solver(mk(), **kw)
    b.restore(path)
    for j in range(2, 4):
        b.advance_strip_vp(tol=1e-6, max_fp=6)
        assert np.array_equal(_end(b), ends[j]), j
        assert np.array_equal(b.density_potential()[0], rhos[j]), j
    b.close()


def test_restore_refuses_another_problem(P, tmp_path):
    a = P.Solver(W.free_streaming_1d(L=3, n_strips=1))
    a.set_initial()
    a.advance_strip()
    path = str(tmp_path / "a.ckpt")
    a.checkpoint(path)
    a.close()
    other = W.free_streaming_1d(L=3, n_strips=1)
    other.dt = other.dt / 2                      # same sizes, another strip operator
    b = P.Solver(other)
    with pytest.raises(P.SgdgError) as e:
        b.restore(path)
    assert e.value.code == 1                      # SGDG_EINVAL
    with pytest.raises(P.SgdgError) as e:
        b.restore(str(tmp_path / "missing.ckpt"))
    assert e.value.code == 7                      # SGDG_EIO
    b.close()


def test_corrupted_checkpoint_leaves_the_handle_unchanged(P, tmp_path):
    """A checkpoint with one flipped payload byte, or cut short, is refused
    (SGDG_EIO) by sgdg_restore, and by sgdg_checkpoint_verify without a
    handle; the handle that refused it continues as if restore had not been
    called, bit for bit."""
    prob = W.free_streaming_1d(L=3, n_strips=3)
    a = P.Solver(prob, rtol=1e-10)
    a.set_initial()
    a.advance_strip()
    path = str(tmp_path / "a.ckpt")
    a.checkpoint(path)
    info = P.checkpoint_verify(path)
    assert info.n_coeffs == a.n_coeffs and info.strips_solved >= 1 and info.has_field == 0
    a.advance_strip()
    ref = _end(a)
    a.close()
    good = open(path, "rb").read()
    bad = bytearray(good)
    bad[len(bad) // 2] ^= 0x01                   # inside a state vector
    for name, data in (("flip", bytes(bad)), ("short", good[:-9])):
        p = str(tmp_path / f"{name}.ckpt")
        open(p, "wb").write(data)
        with pytest.raises(P.SgdgError) as e:
            P.checkpoint_verify(p)
        assert e.value.code == 7
        b = P.Solver(prob, rtol=1e-10)
        b.set_initial()
        b.advance_strip()
        with pytest.raises(P.SgdgError) as e:
            b.restore(p)
        assert e.value.code == 7                  # SGDG_EIO
        b.advance_strip()
        assert np.array_equal(_end(b), ref), name
        b.close()


def test_hbm_budget(P):
    prob = W.transport_2d(L=3, sigma=0.1)
    s = P.Solver(prob)
    held = int(s.info.device_bytes)
    s.close()
    with pytest.raises(P.SgdgError) as e:
        P.Solver(prob, hbm_budget_bytes=held // 2)
    assert e.value.code == 2                      # SGDG_ENOMEM
    ok = P.Solver(prob, hbm_budget_bytes=held + (1 << 20))
    assert ok.info.device_bytes <= held + (1 << 20)
    # the solver's workspace does not fit in what is left: the first strip fails cleanly
    ok.set_initial()
    with pytest.raises(P.SgdgError) as e:
        ok.advance_strip()
    assert e.value.code == 2
    ok.close()


def test_nan_initial_data_gives_enan(P):
    prob = W.free_streaming_1d(L=3, n_strips=1)
    prob.u0 = [W.Product(1.0, lambda p: np.full(p.shape[0], np.nan), None)]
    s = P.Solver(prob)
    s.set_initial()
    with pytest.raises(P.SgdgError) as e:
        s.advance_strip()
    assert e.value.code == 5                      # SGDG_ENAN
    s.close()


def test_outer_cap_gives_enoconv_with_stats(P):
    prob = W.transport_2d(L=3, sigma=0.1, n_strips=1)
    s = P.Solver(prob, rtol=1e-12, max_outer=1, inner_its=4, inner_rtol=1e-1)
    s.set_initial()
    st = s.advance_strip(check=False)
    assert st.status == 4                         # SGDG_ENOCONV
    assert st.outer_its == 1 and st.rel_residual > 1e-12 and st.applies >= 1
    assert np.isfinite(st.rel_residual) and st.seconds > 0
    s.close()


def test_level_out_of_range_gives_einval(P):
    prob = W.free_streaming_1d(L=3, n_strips=1)
    prob.L = 12
    with pytest.raises(P.SgdgError) as e:
        P.Solver(prob)
    assert e.value.code == 1
