"""Python binding of libsgdg: the GB300 sparse-grid time-DG streamline-diffusion
transport library (C ABI in include/sgdg.h).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  The library must
have been built (``paper_2204_05988_gb300.build.build()``); importing the
binding without it raises - there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import List, Optional

from . import build  # noqa: F401  (in-tree build step)

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsgdg.so")

SGDG_FP64 = 0
SGDG_MIXED_FP32 = 1
SGDG_BF16_STORE = 2   # applies only: grid arrays in bfloat16, FP32 arithmetic
SGDG_OUTER_FGMRES = 0
SGDG_OUTER_RICHARDSON = 1   # Algorithm 1: u <- u + P_CT(b - A u)
STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ENOCONV", 5: "ENAN", 6: "ETIMEOUT", 7: "EIO"}

FN = C.CFUNCTYPE(None, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)


class Mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_vertices", C.c_int), ("coords", C.POINTER(C.c_double)),
                ("n_cells", C.c_int), ("cells", C.POINTER(C.c_int)), ("lo", C.POINTER(C.c_double)),
                ("hi", C.POINTER(C.c_double)), ("periodic", C.POINTER(C.c_int))]


class Product(C.Structure):
    _fields_ = [("coef", C.c_double), ("fx", FN), ("ux", C.c_void_p), ("fv", FN), ("uv", C.c_void_p)]


TFN = C.CFUNCTYPE(None, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double), C.c_void_p)


class Source(C.Structure):
    _fields_ = [("coef", C.c_double), ("fx", FN), ("ux", C.c_void_p), ("fv", FN), ("uv", C.c_void_p),
                ("ft", TFN), ("ut", C.c_void_p)]


class Coeffs(C.Structure):
    _fields_ = [("beta", Product * 6), ("sigma", Product), ("n_u0", C.c_int), ("u0", C.POINTER(Product)),
                ("n_f", C.c_int), ("f", C.POINTER(Source)), ("n_g", C.c_int), ("g", C.POINTER(Source)),
                ("beta_t", TFN * 6), ("beta_ut", C.c_void_p * 6), ("sigma_t", TFN), ("sigma_ut", C.c_void_p),
                ("time_quad", C.c_int)]


class Config(C.Structure):
    _fields_ = [("mesh_x", Mesh), ("mesh_v", Mesh), ("level_L", C.c_int), ("time_degree", C.c_int),
                ("dt", C.c_double), ("delta", C.c_double), ("precision", C.c_int), ("rtol", C.c_double),
                ("max_outer", C.c_int), ("restart", C.c_int), ("inner_its", C.c_int),
                ("inner_rtol", C.c_double), ("cheb_steps", C.c_int), ("device", C.c_int),
                ("vlasov_poisson", C.c_int), ("outer_method", C.c_int), ("hbm_budget_bytes", C.c_size_t)]


class Info(C.Structure):
    _fields_ = [("L", C.c_int), ("d", C.c_int), ("R", C.c_int), ("n_grids", C.c_int),
                ("n_spatial", C.c_longlong), ("n_coeffs", C.c_longlong), ("n_terms", C.c_int),
                ("n_x_factors", C.c_int), ("n_v_factors", C.c_int), ("device_bytes", C.c_double),
                ("nnz_x", C.c_longlong), ("nnz_v", C.c_longlong), ("rows_x", C.c_longlong),
                ("rows_v", C.c_longlong), ("lattice_x_levels", C.c_int)]


class StripStats(C.Structure):
    _fields_ = [("outer_its", C.c_int), ("inner_its_total", C.c_int), ("applies", C.c_int),
                ("rel_residual", C.c_double), ("initial_rel_residual", C.c_double), ("seconds", C.c_double),
                ("status", C.c_int)]


EXPORTS = {
    "sgdg_create": (C.c_int, [C.POINTER(Config), C.POINTER(Coeffs), C.POINTER(C.c_void_p)]),
    "sgdg_destroy": (None, [C.c_void_p]),
    "sgdg_last_error": (C.c_char_p, [C.c_void_p]),
    "sgdg_get_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "sgdg_grid_shape": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                  C.POINTER(C.c_longlong)]),
    "sgdg_apply_operator": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sgdg_apply_operator_host": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int]),
    "sgdg_apply_mass": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sgdg_apply_diag": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sgdg_apply_diag_noalloc": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                          C.c_void_p]),
    "sgdg_ct_precondition": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_set_initial": (C.c_int, [C.c_void_p]),
    "sgdg_advance_strip": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(StripStats)]),
    "sgdg_get_solution": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sgdg_get_end_value": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sgdg_eval_nodal": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "sgdg_kernel_stats": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sgdg_launch_count": (C.c_longlong, [C.c_void_p]),
    "sgdg_autotune": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "sgdg_set_launch_shape": (C.c_int, [C.c_void_p, C.c_int]),
    "sgdg_struct_sizes": (C.c_int, [C.POINTER(C.c_int), C.c_int]),
    "sgdg_checkpoint_verify": (C.c_int, [C.c_char_p, C.c_void_p]),
    "sgdg_validate_mesh": (C.c_int, [C.c_void_p]),
    "sgdg_inspect_level": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.c_void_p]),
    "sgdg_inspect_embedding": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                         C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_inspect_factor": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                      C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_inspect_product": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_int,
                                       C.POINTER(C.c_int), C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_inspect_load": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_int,
                                    C.c_void_p]),
    "sgdg_inspect_terms": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double,
                                     C.c_int, C.POINTER(C.c_int), C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_field_update": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double)]),
    "sgdg_resolve_strip": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_advance_strip_vp": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_void_p,
                                        C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "sgdg_set_warm_start": (C.c_int, [C.c_void_p, C.c_int]),
    "sgdg_set_guess": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sgdg_extrapolated_guess": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sgdg_finest_x": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_int)]),
    "sgdg_get_density_potential": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sgdg_set_field": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sgdg_get_field": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "sgdg_coarse_values": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "sgdg_coarse_diff": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                   C.c_void_p]),
    "sgdg_add_coarse": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "sgdg_mlp_create": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_ulonglong, C.POINTER(C.c_void_p)]),
    "sgdg_mlp_destroy": (None, [C.c_void_p]),
    "sgdg_mlp_set_scaling": (C.c_int, [C.c_void_p, C.c_double, C.c_double]),
    "sgdg_mlp_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "sgdg_mlp_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double,
                                      C.POINTER(C.c_double), C.c_void_p]),
    "sgdg_mlp_gradients": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p,
                                     C.POINTER(C.c_double)]),
    "sgdg_mlp_num_params": (C.c_longlong, [C.c_void_p]),
    "sgdg_mlp_get_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sgdg_mlp_set_params": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sgdg_batch_create": (C.c_int, [C.c_int, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p)]),
    "sgdg_batch_destroy": (None, [C.c_void_p]),
    "sgdg_batch_apply": (C.c_int, [C.c_void_p, C.POINTER(C.c_void_p), C.POINTER(C.c_void_p), C.c_int,
                                   C.c_void_p]),
    "sgdg_batch_advance": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sgdg_alu_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "sgdg_checkpoint": (C.c_int, [C.c_void_p, C.c_char_p]),
    "sgdg_copy_tuning": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sgdg_set_sweep_variant": (C.c_int, [C.c_void_p, C.c_int]),
    "sgdg_fused_plan_info": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "sgdg_set_vp_stop": (C.c_int, [C.c_void_p, C.c_int]),
    "sgdg_h1_norm": (C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    "sgdg_restore": (C.c_int, [C.c_void_p, C.c_char_p]),
}

KERNEL_KINDS = ("s_chain", "final_left", "restrict_dim1", "restrict_dim2", "fused_a", "chain_b", "reserved",
                "final_right")


class KernelStat(C.Structure):
    _fields_ = [("launches", C.c_longlong), ("ms", C.c_double), ("bytes", C.c_double), ("flops", C.c_double)]


class FactorSpec(C.Structure):
    _fields_ = [("kind", C.c_int), ("test", C.c_int), ("trial", C.c_int), ("n_weight", C.c_int),
                ("weight", C.c_int * 4), ("n_restrict", C.c_int), ("restrict_fn", C.c_int * 2),
                ("restrict_sign", C.c_int * 2), ("face_axis", C.c_int), ("face_side", C.c_int)]


class CheckpointInfo(C.Structure):
    _fields_ = [("problem_hash", C.c_ulonglong), ("n_coeffs", C.c_longlong), ("n_spatial", C.c_longlong),
                ("t_now", C.c_double), ("strips_solved", C.c_int), ("has_field", C.c_int)]

_lib = None


def load_library(path: str = LIB_PATH) -> C.CDLL:
    """Load libsgdg.so and declare its entry points; raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libsgdg.so not built ({path}); run paper_2204_05988_gb300.build.build()")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


class SgdgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"sgdg {STATUS.get(code, code)}: {msg}")
        self.code = code


def _ptr(t) -> int:
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return int(t)


def _stream(stream) -> Optional[int]:
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


class Solver:
    """One transport problem on the GPU (a handle of the C library).

    ``problem`` is an ``sgdg_workloads.Problem`` (coarse meshes, beta, sigma,
    u0 as products of callables); callables are evaluated by the library
    during construction only.
    """

    def __init__(self, problem, precision: int = SGDG_FP64, rtol: float = 1e-10, max_outer: int = 200,
                 restart: int = 30, inner_its: int = 20, inner_rtol: float = 1e-3, cheb_steps: int = 6,
                 device: int = 0, vlasov_poisson: bool = False, outer_method: int = SGDG_OUTER_FGMRES,
                 hbm_budget_bytes: int = 0):
        if getattr(problem, "order", 1) != 1 or getattr(problem, "element", "P") != "P":
            raise ValueError("the library builds continuous P1 spaces on simplices only (order 1, element 'P')")
        self.lib = load_library()
        self.problem = problem
        self._keep: List = []
        self._cb_error: List[str] = []
        cfg = Config()
        cfg.mesh_x = self._mesh(problem.mesh_x)
        cfg.mesh_v = self._mesh(problem.mesh_v)
        cfg.level_L = problem.L
        cfg.time_degree = problem.r
        cfg.dt = problem.dt
        cfg.delta = problem.delta
        cfg.precision = precision
        cfg.rtol = rtol
        cfg.max_outer = max_outer
        cfg.restart = restart
        cfg.inner_its = inner_its
        cfg.inner_rtol = inner_rtol
        cfg.cheb_steps = cheb_steps
        cfg.device = device
        cfg.vlasov_poisson = int(vlasov_poisson)
        cfg.outer_method = int(outer_method)
        cfg.hbm_budget_bytes = int(hbm_budget_bytes)
        co = Coeffs()
        d = problem.d
        for p in range(6):
            if p < 2 * d:
                co.beta[p] = self._product(problem.beta[p], d)
            else:
                co.beta[p] = Product(0.0, FN(), None, FN(), None)
        co.sigma = self._product(problem.sigma, d)
        u0 = (Product * max(1, len(problem.u0)))()
        for k, pr in enumerate(problem.u0):
            u0[k] = self._product(pr, d)
        co.n_u0 = len(problem.u0)
        co.u0 = u0
        srcs = getattr(problem, "f", None) or []
        fa = (Source * max(1, len(srcs)))()
        for k, sr in enumerate(srcs):
            fa[k] = Source(float(sr.coef), self._fn(sr.fx, d), None, self._fn(sr.fv, d), None, self._tfn(sr.ft),
                           None)
        co.n_f = len(srcs)
        co.f = fa
        gs = getattr(problem, "g", None) or []
        ga = (Source * max(1, len(gs)))()
        for k, sr in enumerate(gs):
            ga[k] = Source(float(sr.coef), self._fn(sr.fx, d), None, self._fn(sr.fv, d), None, self._tfn(sr.ft),
                           None)
        co.n_g = len(gs)
        co.g = ga
        for p in range(2 * d):
            co.beta_t[p] = self._tfn(getattr(problem.beta[p], "ft", None))
        co.sigma_t = self._tfn(getattr(problem.sigma, "ft", None))
        co.time_quad = 0
        self._keep += [cfg, co, u0, fa, ga]
        h = C.c_void_p()
        st = self.lib.sgdg_create(C.byref(cfg), C.byref(co), C.byref(h))
        if self._cb_error:
            if st == 0:
                self.lib.sgdg_destroy(h)
            raise RuntimeError("coefficient callback failed: " + self._cb_error[0])
        if st != 0:
            raise SgdgError(st, self.lib.sgdg_last_error(None).decode())
        self.h = h
        self.info = Info()
        self._check(self.lib.sgdg_get_info(self.h, C.byref(self.info)))
        self.shapes, self.offsets = [], []
        for l in range(self.info.n_grids):
            n1, n2, off = C.c_int(), C.c_int(), C.c_longlong()
            self._check(self.lib.sgdg_grid_shape(self.h, l, C.byref(n1), C.byref(n2), C.byref(off)))
            self.shapes.append((n1.value, n2.value))
            self.offsets.append(off.value)
        self.n_coeffs = self.info.n_coeffs
        self.n_spatial = self.info.n_spatial

    # -- marshalling helpers
    def _mesh(self, m) -> Mesh:
        return _mesh_struct(m, self._keep)

    def _fn(self, f, d):
        if f is None:
            return FN()
        errs = self._cb_error

        def cb(n, pts, out, user):
            try:
                p = np.ctypeslib.as_array(pts, shape=(n * d,)).reshape(n, d)
                o = np.ctypeslib.as_array(out, shape=(n,))
                o[:] = np.asarray(f(p), dtype=np.float64)
            except Exception as e:  # report after sgdg_create returns
                errs.append(repr(e))
                np.ctypeslib.as_array(out, shape=(n,))[:] = np.nan
        c = FN(cb)
        self._keep.append(c)
        return c

    def _tfn(self, f):
        if f is None:
            return TFN()
        errs = self._cb_error

        def cb(n, ts, out, user):
            try:
                t = np.ctypeslib.as_array(ts, shape=(n,))
                o = np.ctypeslib.as_array(out, shape=(n,))
                o[:] = np.broadcast_to(np.asarray(f(t.copy()), dtype=np.float64), (n,))
            except Exception as e:  # reported by the entry point that called it
                errs.append(repr(e))
                np.ctypeslib.as_array(out, shape=(n,))[:] = np.nan
        c = TFN(cb)
        self._keep.append(c)
        return c

    def _product(self, pr, d) -> Product:
        return Product(float(pr.coef), self._fn(pr.fx, d), None, self._fn(pr.fv, d), None)

    def _check(self, st):
        if st != 0:
            raise SgdgError(st, self.lib.sgdg_last_error(self.h).decode())

    # -- entry points (device arrays: torch CUDA tensors or raw pointers)
    def apply_operator(self, u, y, precision: int = SGDG_FP64, stream=None):
        self._check(self.lib.sgdg_apply_operator(self.h, _ptr(u), _ptr(y), precision, _stream(stream)))

    def apply_operator_host(self, u: np.ndarray, y: np.ndarray, precision: int = SGDG_FP64):
        self._check(self.lib.sgdg_apply_operator_host(self.h, _ptr(u), _ptr(y), precision))

    def apply_mass(self, u, y, precision: int = SGDG_FP64, stream=None):
        self._check(self.lib.sgdg_apply_mass(self.h, _ptr(u), _ptr(y), precision, _stream(stream)))

    def apply_diag(self, l1: int, l2: int, u, y, precision: int = SGDG_FP64, stream=None):
        self._check(self.lib.sgdg_apply_diag(self.h, l1, l2, _ptr(u), _ptr(y), precision, _stream(stream)))

    def apply_diag_noalloc(self, l1: int, l2: int, u, y, precision: int = SGDG_FP64, stream=None):
        """sgdg_apply_diag without any device allocation (static scratch of
        SGDG_NOALLOC_SCRATCH_BYTES; for callers that may not allocate device
        memory, e.g. because another component owns it all)."""
        self._check(self.lib.sgdg_apply_diag_noalloc(self.h, l1, l2, _ptr(u), _ptr(y), precision,
                                                     _stream(stream)))

    def ct_precondition(self, r, z, stream=None):
        self._check(self.lib.sgdg_ct_precondition(self.h, _ptr(r), _ptr(z), _stream(stream)))

    def set_initial(self):
        self._check(self.lib.sgdg_set_initial(self.h))

    def advance_strip(self, stream=None, check: bool = True) -> StripStats:
        st = StripStats()
        code = self.lib.sgdg_advance_strip(self.h, _stream(stream), C.byref(st))
        if self._cb_error:
            raise RuntimeError("source callback failed: " + self._cb_error[0])
        if check:
            self._check(code)
        return st

    def checkpoint(self, path: str):
        self._check(self.lib.sgdg_checkpoint(self.h, os.fsencode(path)))

    def restore(self, path: str):
        self._check(self.lib.sgdg_restore(self.h, os.fsencode(path)))

    def get_solution(self, dst, on_device: bool = True):
        self._check(self.lib.sgdg_get_solution(self.h, _ptr(dst), int(on_device)))

    def get_end_value(self, dst, on_device: bool = True):
        self._check(self.lib.sgdg_get_end_value(self.h, _ptr(dst), int(on_device)))

    def eval_nodal(self, u, out, stream=None):
        self._check(self.lib.sgdg_eval_nodal(self.h, _ptr(u), _ptr(out), _stream(stream)))

    def profile(self, enable: bool):
        self._check(self.lib.sgdg_profile(self.h, int(enable)))

    def kernel_stats(self):
        arr = (KernelStat * len(KERNEL_KINDS))()
        self._check(self.lib.sgdg_kernel_stats(self.h, arr, len(KERNEL_KINDS)))
        return {KERNEL_KINDS[k]: {"launches": arr[k].launches, "ms": arr[k].ms, "bytes": arr[k].bytes,
                                  "flops": arr[k].flops}
                for k in range(len(KERNEL_KINDS))}

    def field_update(self, source: int = 0) -> float:
        """Vlasov-Poisson field from the end value (source 0) or from the last
        strip solution at the strip midpoint (source 1); returns 1/2 int |E|^2."""
        e = C.c_double()
        self._check(self.lib.sgdg_field_update(self.h, source, C.byref(e)))
        return e.value

    def resolve_strip(self, stream=None, check: bool = True) -> StripStats:
        st = StripStats()
        code = self.lib.sgdg_resolve_strip(self.h, _stream(stream), C.byref(st))
        if check:
            self._check(code)
        return st

    def advance_strip_vp(self, tol: float = 1e-8, max_fp: int = 10, stream=None, check: bool = True):
        """One Vlasov-Poisson strip with the field iterated to consistency
        (sgdg_advance_strip_vp): returns (stats of the last solve, re-solves,
        last relative change of the potential)."""
        st = StripStats()
        steps = C.c_int()
        change = C.c_double()
        code = self.lib.sgdg_advance_strip_vp(self.h, _stream(stream), tol, max_fp, C.byref(st), C.byref(steps),
                                              C.byref(change))
        if check:
            self._check(code)
        return st, steps.value, change.value

    def coarse_values(self, u, R: int, lx: int, lv: int, out, stream=None):
        self._check(self.lib.sgdg_coarse_values(self.h, _ptr(u), R, lx, lv, _ptr(out), _stream(stream)))

    def coarse_diff(self, a, b, R: int, lx: int, lv: int, out, stream=None):
        self._check(self.lib.sgdg_coarse_diff(self.h, _ptr(a), _ptr(b), R, lx, lv, _ptr(out), _stream(stream)))

    def add_coarse(self, c, lx: int, lv: int, u, stream=None):
        self._check(self.lib.sgdg_add_coarse(self.h, _ptr(c), lx, lv, _ptr(u), _stream(stream)))

    def set_vp_stop(self, criterion: int):
        """Fixed-point stop of advance_strip_vp: 0 relative change of phi, 1 the norms of Sect. 5.3."""
        self._check(self.lib.sgdg_set_vp_stop(self.h, criterion))

    def h1_norm(self, u, stream=None) -> float:
        out = C.c_double()
        self._check(self.lib.sgdg_h1_norm(self.h, _ptr(u), C.byref(out), _stream(stream)))
        return out.value

    def set_warm_start(self, mode: int):
        self._check(self.lib.sgdg_set_warm_start(self.h, mode))

    def extrapolated_guess(self, dst):
        self._check(self.lib.sgdg_extrapolated_guess(self.h, _ptr(dst)))

    def set_guess(self, u):
        self._check(self.lib.sgdg_set_guess(self.h, _ptr(u)))

    def get_field(self) -> np.ndarray:
        """E per finest x cell, shape (d, n_cells)."""
        nv, nc = C.c_int(), C.c_int()
        self._check(self.lib.sgdg_finest_x(self.h, C.byref(nv), C.byref(nc)))
        E = np.empty((self.info.d, nc.value))
        self._check(self.lib.sgdg_get_field(self.h, _ptr(E), nc.value))
        return E

    def set_field(self, E: np.ndarray):
        """A caller-supplied field, shape (d, n_cells) per finest x cell."""
        E = np.ascontiguousarray(E, dtype=np.float64)
        self._check(self.lib.sgdg_set_field(self.h, _ptr(E), E.shape[-1]))

    def density_potential(self):
        nv, nc = C.c_int(), C.c_int()
        self._check(self.lib.sgdg_finest_x(self.h, C.byref(nv), C.byref(nc)))
        rho, phi = np.empty(nv.value), np.empty(nv.value)
        self._check(self.lib.sgdg_get_density_potential(self.h, _ptr(rho), _ptr(phi)))
        return rho, phi

    def autotune(self, u, y, precision: int = SGDG_MIXED_FP32, stream=None):
        self._check(self.lib.sgdg_autotune(self.h, _ptr(u), _ptr(y), precision, _stream(stream)))

    def set_sweep_variant(self, variant: int):
        """0: fused branch A where a tile plan fits; 1: unfused kernels (default)."""
        self._check(self.lib.sgdg_set_sweep_variant(self.h, variant))

    def fused_plan_info(self, grid: int, pair_bytes: int = 8):
        """(tiles, chains per group, ELL width, shared bytes, S entries per chain, restricted outputs per chain)."""
        io = (C.c_int * 4)()
        do = (C.c_double * 2)()
        self._check(self.lib.sgdg_fused_plan_info(self.h, grid, pair_bytes, io, do))
        return tuple(io) + tuple(do)

    def copy_tuning(self, other: "Solver"):
        """Take over another handle's autotuned launch shapes (same problem sizes)."""
        self._check(self.lib.sgdg_copy_tuning(self.h, other.h))

    def set_launch_shape(self, code: int):
        """Pin every sweep launch site to one shape (0: tuned or default)."""
        self._check(self.lib.sgdg_set_launch_shape(self.h, code))

    def launch_count(self) -> int:
        return int(self.lib.sgdg_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            self.lib.sgdg_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def alu_peak(precision: int, device: int = 0, iters: int = 1 << 16):
    """Measured multiply-add peak of the device in GFLOP/s (sgdg_alu_peak):
    precision SGDG_MIXED_FP32 (FFMA) or SGDG_FP64 (DFMA).  Returns (GFLOP/s, ms)."""
    lib = load_library()
    g, ms = C.c_double(), C.c_double()
    st = lib.sgdg_alu_peak(device, precision, iters, C.byref(g), C.byref(ms))
    if st != 0:
        raise SgdgError(st, "sgdg_alu_peak")
    return g.value, ms.value


def _mesh_struct(m, keep: list) -> Mesh:
    """sgdg_mesh over contiguous copies of a coarse mesh's arrays (kept alive in keep)."""
    coords = np.ascontiguousarray(m.coords, dtype=np.float64)
    cells = np.ascontiguousarray(m.cells, dtype=np.int32)
    lo = np.ascontiguousarray(m.lo, dtype=np.float64)
    hi = np.ascontiguousarray(m.hi, dtype=np.float64)
    per = np.ascontiguousarray([int(p) for p in m.periodic], dtype=np.int32)
    keep += [coords, cells, lo, hi, per]
    dp = C.POINTER(C.c_double)
    ip = C.POINTER(C.c_int)
    return Mesh(m.dim, coords.shape[0], coords.ctypes.data_as(dp), cells.shape[0], cells.ctypes.data_as(ip),
                lo.ctypes.data_as(dp), hi.ctypes.data_as(dp), per.ctypes.data_as(ip))


def validate_mesh(m) -> None:
    """sgdg_validate_mesh (host only): raises SgdgError (EINVAL) naming the
    failed check of a coarse mesh."""
    lib = load_library()
    keep: list = []
    ms = _mesh_struct(m, keep)
    st = lib.sgdg_validate_mesh(C.byref(ms))
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())


class _Marshal:
    """Callback and struct marshalling outside a Solver (host-only calls)."""

    def __init__(self):
        self._keep: list = []
        self._cb_error: List[str] = []

    _fn = lambda self, f, d: Solver._fn(self, f, d)
    _tfn = lambda self, f: Solver._tfn(self, f)
    _product = lambda self, pr, d: Solver._product(self, pr, d)

    def coeffs(self, problem, time_quad: int = 0) -> "Coeffs":
        """beta and sigma with their time factors (u0, f, g left empty)."""
        d = problem.d
        co = Coeffs()
        for p in range(6):
            co.beta[p] = self._product(problem.beta[p], d) if p < 2 * d else Product(0.0, FN(), None, FN(), None)
        co.sigma = self._product(problem.sigma, d)
        for p in range(2 * d):
            co.beta_t[p] = self._tfn(getattr(problem.beta[p], "ft", None))
        co.sigma_t = self._tfn(getattr(problem.sigma, "ft", None))
        co.time_quad = int(time_quad)
        self._keep.append(co)
        return co


def _csr_out(call):
    """Run a two-pass CSR query: sizes first, then the arrays."""
    lib = load_library()
    nrows, nnz = C.c_int(), C.c_int()
    st = call(C.byref(nrows), C.byref(nnz), None, None, None)
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())
    rowptr = np.empty(nrows.value + 1, dtype=np.int32)
    col = np.empty(nnz.value, dtype=np.int32)
    val = np.empty(nnz.value, dtype=np.float64)
    st = call(C.byref(nrows), C.byref(nnz), rowptr.ctypes.data, col.ctypes.data, val.ctypes.data)
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())
    return rowptr, col, val


def inspect_level(mesh, L: int, level: int) -> np.ndarray:
    """sgdg_inspect_level: the vertex coordinates [n][dim] of one level, in the
    library's canonical order (host only)."""
    lib = load_library()
    keep: list = []
    ms = _mesh_struct(mesh, keep)
    n = C.c_int()
    st = lib.sgdg_inspect_level(C.byref(ms), L, level, C.byref(n), None)
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())
    coords = np.empty((n.value, mesh.dim), dtype=np.float64)
    st = lib.sgdg_inspect_level(C.byref(ms), L, level, C.byref(n), coords.ctypes.data)
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())
    return coords


def inspect_embedding(mesh, L: int, level: int):
    """sgdg_inspect_embedding: E_{level+1 <- level} as CSR arrays (rowptr, col, val)."""
    lib = load_library()
    keep: list = []
    ms = _mesh_struct(mesh, keep)
    return _csr_out(lambda nr, nz, rp, cl, vl: lib.sgdg_inspect_embedding(C.byref(ms), L, level, nr, nz, rp, cl, vl))


def inspect_factor(problem, side: int, L: int, level: int, kind: int = 0, test: int = 0, trial: int = 0,
                   weight=(), restrict=(), face=(-1, 0), product: int = -1):
    """sgdg_inspect_factor: one factor of side 0 (x) or 1 (v) of the problem's
    coefficients, assembled on level L and projected to `level`, as CSR
    arrays (rowptr, col, val).  weight: function ids (0..5 beta components,
    6 sigma); restrict: (id, sign) pairs; face: (axis, side) for kind 1."""
    lib = load_library()
    m = _Marshal()
    co = m.coeffs(problem)
    spec = FactorSpec()
    spec.kind, spec.test, spec.trial = kind, test, trial
    spec.n_weight = len(weight)
    for i, w in enumerate(weight):
        spec.weight[i] = w
    spec.n_restrict = len(restrict)
    for i, (fid, sg) in enumerate(restrict):
        spec.restrict_fn[i], spec.restrict_sign[i] = fid, sg
    spec.face_axis, spec.face_side = face
    mesh = problem.mesh_x if side == 0 else problem.mesh_v
    ms = _mesh_struct(mesh, m._keep)
    if product < 0:
        out = _csr_out(lambda nr, nz, rp, cl, vl: lib.sgdg_inspect_factor(C.byref(ms), C.byref(co), side, L, level,
                                                                          C.byref(spec), nr, nz, rp, cl, vl))
    else:   # sgdg_inspect_product: 0 = R_level X_{level+1}, 1 = X_level E_{level-1}
        out = _csr_out(lambda nr, nz, rp, cl, vl: lib.sgdg_inspect_product(
            C.byref(ms), C.byref(co), side, L, level, C.byref(spec), product, nr, nz, rp, cl, vl))
    if m._cb_error:
        raise RuntimeError("coefficient callback failed: " + m._cb_error[0])
    return out


def inspect_load(mesh, L: int, level: int, fns=(), deriv: int = 0) -> np.ndarray:
    """sgdg_inspect_load: int (prod fns) D phi_i on level L restricted to
    `level` (D: value, or d/dy_deriv for deriv >= 1)."""
    lib = load_library()
    m = _Marshal()
    ms = _mesh_struct(mesh, m._keep)
    arr = (FN * max(1, len(fns)))(*[m._fn(f, mesh.dim) for f in fns])
    n = inspect_level(mesh, L, level).shape[0]
    out = np.empty(n)
    st = lib.sgdg_inspect_load(C.byref(ms), L, level, len(fns), C.cast(arr, C.c_void_p), None, deriv,
                               out.ctypes.data)
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())
    if m._cb_error:
        raise RuntimeError("coefficient callback failed: " + m._cb_error[0])
    return out


def _spec_dict(f: FactorSpec) -> dict:
    return {"kind": f.kind, "test": f.test, "trial": f.trial, "weight": tuple(f.weight[:f.n_weight]),
            "restrict": tuple((f.restrict_fn[i], f.restrict_sign[i]) for i in range(f.n_restrict)),
            "face": (f.face_axis, f.face_side)}


def inspect_terms(problem, t0: float = 0.0, time_quad: int = 0):
    """sgdg_inspect_terms: the Kronecker terms of the problem's operator with
    the time couplings of the strip (t0, t0 + dt): a list of (tau (2 x 2),
    x factor spec, v factor spec), specs as dicts of sgdg_factor_spec's
    fields (keywords of ``inspect_factor``); time_quad: Gauss points per
    strip with time factors (0: 3)."""
    lib = load_library()
    m = _Marshal()
    co = m.coeffs(problem, time_quad)
    mx, mv = _mesh_struct(problem.mesh_x, m._keep), _mesh_struct(problem.mesh_v, m._keep)
    n = C.c_int()
    args = (C.byref(mx), C.byref(mv), C.byref(co), float(problem.dt), float(problem.delta), float(t0))
    st = lib.sgdg_inspect_terms(*args, 0, C.byref(n), None, None, None)
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())
    tau = np.zeros((n.value, 2, 2))
    xs, vs = (FactorSpec * max(1, n.value))(), (FactorSpec * max(1, n.value))()
    st = lib.sgdg_inspect_terms(*args, n.value, C.byref(n), tau.ctypes.data, C.cast(xs, C.c_void_p),
                                C.cast(vs, C.c_void_p))
    if st != 0:
        raise SgdgError(st, lib.sgdg_last_error(None).decode())
    if m._cb_error:
        raise RuntimeError("coefficient callback failed: " + m._cb_error[0])
    return [(tau[k], _spec_dict(xs[k]), _spec_dict(vs[k])) for k in range(n.value)]


def checkpoint_verify(path: str) -> CheckpointInfo:
    """sgdg_checkpoint_verify: the restore checks on a checkpoint file alone
    (host only).  Returns its CheckpointInfo; raises SgdgError (EIO) for a
    truncated or corrupted file."""
    lib = load_library()
    info = CheckpointInfo()
    st = lib.sgdg_checkpoint_verify(os.fsencode(path), C.byref(info))
    if st != 0:
        raise SgdgError(st, f"sgdg_checkpoint_verify({path})")
    return info


class Batch:
    """Independent problems advanced together (sgdg_batch_*): one CUDA graph per
    batch apply, concurrent strip solves."""

    def __init__(self, solvers):
        self.lib = load_library()
        self.solvers = list(solvers)
        arr = (C.c_void_p * len(self.solvers))(*[s.h for s in self.solvers])
        b = C.c_void_p()
        st = self.lib.sgdg_batch_create(len(self.solvers), arr, C.byref(b))
        if st != 0:
            raise SgdgError(st, self.lib.sgdg_last_error(None).decode())
        self.b = b

    def apply(self, us, ys, precision: int = SGDG_MIXED_FP32, stream=None):
        n = len(self.solvers)
        ua = (C.c_void_p * n)(*[_ptr(u) for u in us])
        ya = (C.c_void_p * n)(*[_ptr(y) for y in ys])
        st = self.lib.sgdg_batch_apply(self.b, ua, ya, precision, _stream(stream))
        if st != 0:
            raise SgdgError(st, self.lib.sgdg_last_error(None).decode())

    def advance(self):
        n = len(self.solvers)
        stats = (StripStats * n)()
        st = self.lib.sgdg_batch_advance(self.b, stats)
        if st != 0:
            raise SgdgError(st, self.lib.sgdg_last_error(None).decode())
        return list(stats)

    def close(self):
        if getattr(self, "b", None):
            self.lib.sgdg_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Mlp:
    """The library's BF16 MLP (sgdg_mlp_*): 3 layers, FP64 batches on the device."""

    def __init__(self, n_in: int, width: int, n_out: int, max_batch: int, seed: int = 0):
        self.lib = load_library()
        m = C.c_void_p()
        st = self.lib.sgdg_mlp_create(n_in, width, n_out, max_batch, seed, C.byref(m))
        if st != 0:
            raise SgdgError(st, "mlp create")
        self.m = m
        self.n_in, self.width, self.n_out = n_in, width, n_out

    def _chk(self, st, what):
        if st != 0:
            raise SgdgError(st, what)

    def set_scaling(self, in_scale: float, out_scale: float):
        self._chk(self.lib.sgdg_mlp_set_scaling(self.m, in_scale, out_scale), "mlp scaling")

    def forward(self, x, batch: int, y, stream=None):
        self._chk(self.lib.sgdg_mlp_forward(self.m, _ptr(x), batch, _ptr(y), _stream(stream)), "mlp forward")

    def train_step(self, x, t, batch: int, lr: float, stream=None) -> float:
        loss = C.c_double()
        self._chk(self.lib.sgdg_mlp_train_step(self.m, _ptr(x), _ptr(t), batch, lr, C.byref(loss),
                                               _stream(stream)), "mlp train step")
        return loss.value

    def num_params(self) -> int:
        return int(self.lib.sgdg_mlp_num_params(self.m))

    def gradients(self, x, t, batch: int):
        g = np.empty(self.num_params(), dtype=np.float32)
        loss = C.c_double()
        self._chk(self.lib.sgdg_mlp_gradients(self.m, _ptr(x), _ptr(t), batch, _ptr(g), C.byref(loss)),
                  "mlp gradients")
        return g, loss.value

    def get_params(self) -> np.ndarray:
        p = np.empty(self.num_params(), dtype=np.float32)
        self._chk(self.lib.sgdg_mlp_get_params(self.m, _ptr(p)), "mlp params")
        return p

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._chk(self.lib.sgdg_mlp_set_params(self.m, _ptr(p)), "mlp params")

    def close(self):
        if getattr(self, "m", None):
            self.lib.sgdg_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
