"""Configurations sgdg_create refuses (SGDG_EINVAL) before it touches a
device, on the CPU: each case below is one wrong field of an otherwise valid
d = 1 problem, and the error names the field.  (Refusals that need the built
spaces, such as sources with vlasov_poisson, come after the device set-up
and are covered by the GPU tests.)"""
import dataclasses

import numpy as np
import pytest

import paper_2204_05988_gb300 as P
import sgdg_workloads as W

EINVAL = 1


def _refused(words, prob=None, **kw):
    prob = prob or W.free_streaming_1d(L=2, n_strips=1)
    with pytest.raises(P.SgdgError) as e:
        P.Solver(prob, **kw)
    assert e.value.code == EINVAL, str(e.value)
    assert words in str(e.value), str(e.value)


def test_levels_and_dimensions():
    _refused("level_L out of range", W.free_streaming_1d(L=12, n_strips=1))
    p = W.free_streaming_1d(L=2, n_strips=1)
    p.mesh_v = W.square_mesh(0.0, 1.0, 2)
    _refused("same dimension", p)


def test_time_step_delta_and_degree():
    p = W.free_streaming_1d(L=2, n_strips=1)
    _refused("dt must be > 0", dataclasses.replace(p, dt=0.0))
    _refused("dt must be > 0", dataclasses.replace(p, dt=float("nan")))
    _refused("delta >= 0", dataclasses.replace(p, delta=-1e-3))
    _refused("time_degree 1", dataclasses.replace(p, r=0))


def test_solver_settings():
    _refused("BF16 storage is an apply precision", precision=P.SGDG_BF16_STORE)
    _refused("unknown precision", precision=7)
    _refused("restart and inner_its", restart=0)
    _refused("restart and inner_its", restart=64)
    _refused("restart and inner_its", inner_its=0)
    _refused("unknown outer_method", outer_method=5)


def test_time_factors_with_the_field_update():
    p = W.landau_4d(L=1, n_strips=1)
    p.sigma = W.Product(0.1, None, None, lambda t: 1.0 + np.asarray(t))
    _refused("vlasov_poisson", p, vlasov_poisson=True)
