"""Benchmark: sparse-grid SD-Galerkin operator apply (GDoF/s) and strip solves.

Workload (default): the 4D transport problem, d = 2, Omega_x = [0,1]^2,
Omega_v = [-1,1]^2, 8-triangle coarse meshes, sparse level L = 9 (grids
(l, 9-l)), time-DG degree 1, beta = (v, E(x)), sigma = 0.1: 61,590,186 spatial
coefficients, 123,180,372 DoF per strip vector (FP32: 493 MB, FP64: 985 MB,
both larger than L2).  A step is one application of the strip operator
A^(delta) to a seeded U[-1,1] vector, resident in HBM.

Reported: value = GDoF/s of the mixed-precision (FP32) apply; the FP64 and
BF16-storage applies; the end-to-end apply through the C ABI with host
buffers; the roofline of the whole apply and of its dominant kernel (FP32
ALU: executed flops over the measured FFMA peak, the bound at the apply's
arithmetic intensity; the HBM view, algorithmic bytes over the measured copy
bandwidth, beside it); strip solves at 1e-8 on the same workload (mixed vs
FP64); the d = 3 (6-D) apply at L = 7 with its HBM footprint; the batched
apply of 48 instances of uneven L (one CUDA graph); batched strips against
the plain FP64 solver; the oracle timed on one host core and on all of them.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import sgdg_workloads as W  # noqa: E402

METRIC = "operator-apply GDoF/s; s/time-strip at 1e-8 rel. residual, mixed vs FP64"


# ALU peaks from the unit counts and the maximum SM clock (2,070 MHz), used
# only when the measured ones (sgdg_alu_peak, timed at the start of the run)
# are unavailable: FP32 - 152 SMs x 128 FP32 lanes x 2 flops per multiply-add;
# FP64 - the nominal GB300 non-tensor FP64 rate (1.25 TFLOP/s).
FP32_PEAK_GFLOPS = 152 * 128 * 2 * 2.070
FP64_PEAK_GFLOPS = 1250.0


def _traffic(kind: str, L: int, key: str = "dram_bytes_per_launch"):
    """DRAM bytes per launch of a sweep kernel kind from the committed ncu
    launch-list summary, when it was taken on this workload and on the kernel
    sources as they are now (None otherwise)."""
    import hashlib
    p = os.path.join(ROOT, "profiles", "sweep_traffic_transport2d_L9.json")
    if L != 9 or not os.path.exists(p):
        return None
    with open(p) as f:
        d = json.load(f)
    h = hashlib.sha256()
    for rel in d["kernel_sources"]:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    if h.hexdigest() != d["kernel_sources_sha256"]:
        return None
    return d.get(key, {}).get(kind)


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


class Ranks:
    """The replicas of a multi-GPU run: one process per GPU under torchrun,
    each with its own problem instance and no data-path collective.  Barrier
    and max-over-ranks reductions of timings on `device` (NCCL on the GPUs;
    gloo on the host cores in the tests).  dist None: a single process."""

    def __init__(self, dist=None, device="cpu"):
        self.dist = dist
        self.device = device

    def barrier(self):
        if self.dist:
            self.dist.barrier()
        if str(self.device).startswith("cuda"):
            import torch
            torch.cuda.synchronize()

    def max(self, x: float) -> float:
        if not self.dist:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())


_T0 = time.perf_counter()


def log(msg: str):
    """Progress of the run on stderr (the JSON line alone goes to stdout)."""
    print(f"[bench {time.perf_counter() - _T0:7.1f} s] {msg}", file=sys.stderr, flush=True)


def whole_job(world: int, units_per_rank: float, seconds: float) -> float:
    """Weak scaling: every rank processes units_per_rank; `seconds` is the
    slowest rank's time, so the job's rate is world x units / seconds."""
    return world * units_per_rank / seconds


def cpu_info():
    """Host CPU model and logical core count (for the baseline's record)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.split(":")[0].strip() in ("Model name", "Model"):
                model = ln.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    model = ln.split(":", 1)[1].strip()
                    break
    return {"nproc": os.cpu_count(), "model": model}


_POOL_OP = None


def _pool_init(L):
    global _POOL_OP
    os.environ["OMP_NUM_THREADS"] = "1"
    from oracle.operator import SparseGridOperator
    _POOL_OP = SparseGridOperator(W.transport_2d(L=L, sigma=0.1))
    u = W.uniform_vector(_POOL_OP.size, seed=7)
    _POOL_OP.apply(u)                               # builds the projected factors


def _pool_blocks(args):
    """Blocks (i, j) of the oracle's blockwise apply: A_ij u_j for target grid i."""
    pairs, u = args
    op = _POOL_OP
    return [(i, op.apply_block(op.terms, op.grids[i], op.grids[j], op.block(u, j))) for i, j in pairs]


def _pool_apply(pool, nw, op, u):
    """y = A u with the (target, source) blocks spread over the pool's workers."""
    pairs = [(i, j) for i in range(len(op.grids)) for j in range(len(op.grids))]
    chunks = [pairs[k::nw] for k in range(nw)]
    y = [np.zeros(op.shape[i] + (op.R,)) for i in range(len(op.grids))]
    for part in pool.map(_pool_blocks, [(c, u) for c in chunks]):
        for i, blk in part:
            y[i] += blk
    return np.concatenate([b.ravel() for b in y])


def cpu_baseline(steps: int = 4, L: int = 5, all_cores: bool = True):
    """The oracle's blockwise apply (Sect. 4.2) on the host cores, as it stands,
    on a bounded sample of the same workload family (d = 2, level L): on one
    core, and on all cores with the target grids spread over a process pool
    (spawned, so that no worker inherits the CUDA context)."""
    from oracle.operator import SparseGridOperator
    info = cpu_info()
    prob = W.transport_2d(L=L, sigma=0.1)
    op = SparseGridOperator(prob)
    u = W.uniform_vector(op.size, seed=7)
    op.apply(u)                                     # warm-up: builds the projected factors
    t = time.perf_counter()
    for _ in range(steps):
        op.apply(u)
    dt = (time.perf_counter() - t) / steps
    res = {"value": op.size / dt / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
           "sample": f"blockwise FP64 apply, d=2 L={L} ({op.size} DoF), {steps} applies after 1 warm-up; "
                     f"numpy/scipy, one process", "nproc": info["nproc"], "cpu_model": info["model"]}
    if all_cores and (info["nproc"] or 1) > 1:
        import multiprocessing as mp
        nw = min(info["nproc"], len(op.grids) ** 2)
        with mp.get_context("spawn").Pool(nw, initializer=_pool_init, initargs=(L,)) as pool:
            y = _pool_apply(pool, nw, op, u)                          # warm-up
            t = time.perf_counter()
            for _ in range(steps):
                _pool_apply(pool, nw, op, u)
            dtp = (time.perf_counter() - t) / steps
        ref = op.apply(u)
        res["all_cores"] = {"value": op.size / dtp / 1e9, "unit": "GDoF/s", "cores": nw,
                            "sample": f"same apply, its {len(op.grids) ** 2} (target, source) grid blocks "
                                      f"spread over {nw} spawned worker processes (one core each)",
                            "max_abs_diff_vs_one_core": float(np.abs(y - ref).max())}
    return res, dt, op.size


def run_reference(args, rank, world):
    if rank != 0:
        return
    W_, K = args.warmup, args.steps
    from oracle.operator import SparseGridOperator
    L = args.ref_L
    prob = W.transport_2d(L=L, sigma=0.1)
    op = SparseGridOperator(prob)
    u = W.uniform_vector(op.size, seed=7)
    for _ in range(max(1, W_)):
        op.apply(u)
    t = time.perf_counter()
    for _ in range(K):
        op.apply(u)
    dt = (time.perf_counter() - t) / K
    val = op.size / dt / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GDoF/s", "n_gpus": world,
            "steps": K, "warmup": W_, "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"transport_2d d=2 L={L} sigma=0.1 operator apply (oracle sample)",
                       "dof_per_step": op.size},
            "cpu_baseline": {"value": val, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
                             "sample": f"blockwise FP64 apply, d=2 L={L} ({op.size} DoF) per step"},
            "e2e": {"value": val, "unit": "GDoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--L", type=int, default=9)
    ap.add_argument("--ref-L", type=int, default=5)
    ap.add_argument("--strip-L", type=int, default=9, help="level of the strip-solve timing (-1: skip)")
    ap.add_argument("--strips-mixed", type=int, default=3, help="mixed-precision strips solved")
    ap.add_argument("--strips-fp64", type=int, default=2, help="plain FP64 strips solved")
    ap.add_argument("--inner-its", type=int, default=48, help="GMRES steps per component solve (strips)")
    ap.add_argument("--inner-rtol", type=float, default=1e-3, help="early stop of a component solve (strips)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", type=int, default=8, help="instances in the batched strip measurement (0: skip)")
    ap.add_argument("--batch-levels", type=int, nargs="+", default=[5, 6, 7])
    ap.add_argument("--warmstart", action="store_true",
                    help="learned warm start: train on Landau runs, evaluate on held-out seeds (opt-in)")
    ap.add_argument("--ws-L", type=int, default=5)
    ap.add_argument("--ws-train-seeds", type=int, default=20)
    ap.add_argument("--ws-strips", type=int, default=24, help="strips per training run and per evaluation run")
    ap.add_argument("--d3-L", type=int, default=7,
                    help="level of the d = 3 (6-D) apply measurement (transport_3d; -1: skip)")
    ap.add_argument("--batch-apply", type=int, default=48,
                    help="instances in the full-size batched apply (L from {6,7,8,9}, seed 0; 0: skip)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    import paper_2204_05988_gb300 as P
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    ranks = Ranks(dist, "cuda")
    barrier = ranks.barrier
    # measured ALU peaks (register-only multiply-add kernels), the roofline
    # denominators of the FP32 sweep and of the FP64 apply
    try:
        fp32_peak, fp32_peak_src = P.alu_peak(P.SGDG_MIXED_FP32, local, 1 << 18)[0], "measured (sgdg_alu_peak FFMA)"
        fp64_peak, fp64_peak_src = P.alu_peak(P.SGDG_FP64, local, 1 << 13)[0], "measured (sgdg_alu_peak DFMA)"
    except P.SgdgError:
        fp32_peak, fp32_peak_src = FP32_PEAK_GFLOPS, "derived: 152 SMs x 128 lanes x 2 x 2.07 GHz"
        fp64_peak, fp64_peak_src = FP64_PEAK_GFLOPS, "nominal GB300 FP64 rate"

    log(f"peaks: FP32 {fp32_peak:.0f} GFLOP/s, FP64 {fp64_peak:.0f} GFLOP/s")
    prob = W.transport_2d(L=args.L, sigma=0.1)
    t0 = time.perf_counter()
    s = P.Solver(prob, device=local)
    setup_s = time.perf_counter() - t0
    n = s.n_coeffs
    # (r+1) dim V_L, the unique count of the paper's convention: the grids
    # (l, L-l) overlap in the grids (l, L-1-l) of the nested spaces
    sh = s.shapes
    unique = 2 * (sum(a * b for a, b in sh) - sum(sh[l][0] * sh[l + 1][1] for l in range(len(sh) - 1)))
    u64 = torch.tensor(W.uniform_vector(n, seed=1 + rank), dtype=torch.float64, device="cuda")
    u32 = u64.float()
    u16 = u64.to(torch.bfloat16)
    y32 = torch.empty_like(u32)
    y64 = torch.empty_like(u64)
    y16 = torch.empty_like(u16)
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    s.autotune(u32, y32, P.SGDG_MIXED_FP32, stream)
    s.autotune(u64, y64, P.SGDG_FP64, stream)
    s.autotune(u16, y16, P.SGDG_BF16_STORE, stream)
    torch.cuda.synchronize()
    tune_s = time.perf_counter() - t0

    def timed(fn, K, Wm):
        for _ in range(Wm):
            fn()
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(K):
            fn()
        e1.record(stream)
        barrier()
        return ranks.max(e0.elapsed_time(e1) / K)

    log(f"set-up {setup_s:.1f} s, autotune {tune_s:.1f} s")
    # ---- FP32 apply (headline), clocks sampled during the timed region
    for _ in range(args.warmup):
        s.apply_operator(u32, y32, P.SGDG_MIXED_FP32, stream)
    barrier()
    # clocks are sampled over the timed regions (FP32, FP64, BF16 storage), ~2 s of load
    with Clocks(local) as clk:
        l0 = s.launch_count()
        ms32 = timed(lambda: s.apply_operator(u32, y32, P.SGDG_MIXED_FP32, stream), args.steps, 0)
        launches = s.launch_count() - l0
        # ---- FP64 apply
        ms64 = timed(lambda: s.apply_operator(u64, y64, P.SGDG_FP64, stream), max(2, args.steps // 2), 1)
        # ---- BF16-storage apply
        ms16 = timed(lambda: s.apply_operator(u16, y16, P.SGDG_BF16_STORE, stream), args.steps, 1)
    clocks = clk.summary()
    value = whole_job(world, n, ms32 * 1e-3) / 1e9

    # errors of the reduced precisions against the FP64 apply of the same input
    # (the FP64 path matches the oracle to 1e-12)
    def rel(a, b):
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    s.apply_operator(u64, y64, P.SGDG_FP64, stream)
    s.apply_operator(u32, y32, P.SGDG_MIXED_FP32, stream)
    err32 = rel(y32.double(), y64)
    s.apply_operator(u16.double(), y64, P.SGDG_FP64, stream)
    s.apply_operator(u16, y16, P.SGDG_BF16_STORE, stream)
    err16 = rel(y16.double(), y64)

    log(f"applies: FP32 {ms32:.2f} ms, FP64 {ms64:.2f} ms, BF16 storage {ms16:.2f} ms")
    # ---- per-kernel roofline (one profiled apply per precision)
    peak, peak_kind = _peaks()
    roof = {}
    for name, (u_, y_, pr) in {"f32": (u32, y32, P.SGDG_MIXED_FP32), "f64": (u64, y64, P.SGDG_FP64),
                               "bf16": (u16, y16, P.SGDG_BF16_STORE)}.items():
        s.profile(True)
        s.apply_operator(u_, y_, pr, stream)
        st = s.kernel_stats()
        s.profile(False)
        roof[name] = st
    st = roof["f32"]
    dom = max(st, key=lambda k: st[k]["ms"])
    ach = st[dom]["bytes"] / (st[dom]["ms"] * 1e-3) / 1e9
    tot_ms = sum(v["ms"] for v in st.values())
    st64 = roof["f64"]
    dom64 = max(st64, key=lambda k: st64[k]["ms"])
    tot64 = sum(v["ms"] for v in st64.values())
    fl64 = sum(v["flops"] for v in st64.values())
    fp64_roof = {"bound": "alu", "kernel": dom64,
                 "achieved": st64[dom64]["flops"] / (st64[dom64]["ms"] * 1e-3) / 1e9, "peak": fp64_peak,
                 "unit": "GFLOP/s", "peak_source": fp64_peak_src,
                 "frac": st64[dom64]["flops"] / (st64[dom64]["ms"] * 1e-3) / 1e9 / fp64_peak,
                 "apply_GFLOPs": fl64 / (tot64 * 1e-3) / 1e9, "apply_frac": fl64 / (tot64 * 1e-3) / 1e9 / fp64_peak,
                 "share_of_apply": st64[dom64]["ms"] / tot64}
    # whole-apply effective bandwidth: the bytes the method must move per apply
    # (read u, write y, every pattern once, every factor value array once),
    # independent of the sweep's intermediates
    inf = s.info
    b_alg = (n * (4 + 4) + 4 * (inf.rows_x + inf.rows_v + 2 * (inf.L + 1))
             + 4 * inf.nnz_x * (1 + inf.n_x_factors) + 4 * inf.nnz_v * (1 + inf.n_v_factors))
    fl32 = sum(v["flops"] for v in st.values())
    per_kind = lambda stats: {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                  "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None,
                                  "GFLOPs": (v["flops"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                              for k, v in stats.items() if v["launches"]}
    # roofline.  The whole apply executes fl32 flops (2 per multiply-add of
    # every sweep launch) against B_alg algorithmic bytes (u read, y written,
    # every pattern and factor value array once): about 70 flop/B, far above
    # the ridge of the measured FP32 ALU and HBM peaks (about 11 flop/B), so
    # the apply's bound is the FP32 ALU - the headline.  Its HBM view (B_alg
    # over the apply time) and the dominant kernel are reported beside it; the
    # dominant kernel's own algorithmic bytes include the sweep's chain states
    # it reads (about 4 flop/B: HBM-side of the ridge), so it is given in both
    # terms, with the DRAM bytes per launch ncu measured (traffic).
    fl_apply_rate = fl32 / (ms32 * 1e-3) / 1e9
    nl = max(1, st[dom]["launches"])
    dom_flops = st[dom]["flops"] / (st[dom]["ms"] * 1e-3) / 1e9
    roofline = {"bound": "alu", "kernel": "operator apply (all sweep launches)",
                "achieved": fl_apply_rate, "peak": fp32_peak, "unit": "GFLOP/s",
                "frac": fl_apply_rate / fp32_peak, "peak_source": fp32_peak_src,
                "traffic": _traffic("apply", args.L, "dram_bytes_per_apply"),
                "alg_flops_per_launch": fl32,
                "flops_definition": "2 per multiply-add of every sweep launch (matrix rows at their register "
                                    "length), per apply",
                "arithmetic_intensity_flop_per_B": fl32 / b_alg,
                "ridge_flop_per_B": fp32_peak / peak,
                "hbm_view": {"achieved": b_alg / (ms32 * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                             "frac": b_alg / (ms32 * 1e-3) / 1e9 / peak, "peak_source": f"{peak_kind} hbm_gbs",
                             "alg_bytes_per_launch": b_alg,
                             "b_alg_definition": "8 B x DoF (u in, y out, FP32) + int32 patterns + FP32 value "
                                                 "arrays of every factor, once"},
                "dominant_kernel": {"kernel": dom, "bound": "hbm",
                                    "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                                    "traffic": _traffic(dom, args.L),
                                    "alg_bytes_per_launch": st[dom]["bytes"] / nl,
                                    "alg_flops_per_launch": st[dom]["flops"] / nl,
                                    "mean_launch_ms": st[dom]["ms"] / nl,
                                    "arithmetic_intensity_flop_per_B": st[dom]["flops"] / max(1.0, st[dom]["bytes"]),
                                    "alu": {"achieved": dom_flops, "peak": fp32_peak, "unit": "GFLOP/s",
                                            "frac": dom_flops / fp32_peak},
                                    "share_of_apply": st[dom]["ms"] / tot_ms},
                "sweep_bytes": sum(v["bytes"] for v in st.values()),
                "sweep_GBps": sum(v["bytes"] for v in st.values()) / (tot_ms * 1e-3) / 1e9,
                "per_kind": per_kind(st), "f64_per_kind": per_kind(roof["f64"])}
    st16 = roof["bf16"]
    dom16 = max(st16, key=lambda k: st16[k]["ms"])
    bf16_apply = {"value": whole_job(world, n, ms16 * 1e-3) / 1e9, "unit": "GDoF/s", "ms_per_step": ms16,
                  "storage": "bfloat16 grid arrays, FP32 arithmetic and matrix values",
                  "rel_err_vs_fp64": err16,
                  "roofline": {"bound": "hbm", "kernel": dom16,
                               "achieved": st16[dom16]["bytes"] / (st16[dom16]["ms"] * 1e-3) / 1e9,
                               "peak": peak, "unit": "GB/s",
                               "frac": st16[dom16]["bytes"] / (st16[dom16]["ms"] * 1e-3) / 1e9 / peak,
                               "traffic": _traffic(dom16, args.L, "dram_bytes_per_launch_bf16"),
                               "alg_bytes_per_launch": st16[dom16]["bytes"] / max(1, st16[dom16]["launches"]),
                               "share_of_apply": st16[dom16]["ms"] / sum(v["ms"] for v in st16.values())},
                  "per_kind": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                   "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                               for k, v in st16.items() if v["launches"]}}

    log("profiled applies done")
    # ---- end to end through the C ABI with pinned host buffers (FP64 in/out, FP32 apply)
    hu = torch.empty(n, dtype=torch.float64, pin_memory=True)
    hu.copy_(u64.cpu())
    hy = torch.empty(n, dtype=torch.float64, pin_memory=True)
    for _ in range(2):
        s.apply_operator_host(hu, hy, P.SGDG_MIXED_FP32)
    barrier()
    # each call is synchronous (copies back included); host wall time per call
    ke = max(3, args.steps // 2)
    per = []
    for _ in range(ke):
        te = time.perf_counter()
        s.apply_operator_host(hu, hy, P.SGDG_MIXED_FP32)
        per.append(time.perf_counter() - te)
    barrier()
    e2e_s = ranks.max(float(np.median(per)))
    e2e = {"value": whole_job(world, n, e2e_s) / 1e9, "unit": "GDoF/s", "h2d_bytes_per_step": 8 * n,
           "d2h_bytes_per_step": 8 * n, "ms_per_step": e2e_s * 1e3, "statistic": f"median of {ke} calls",
           "ms_per_call": [round(x * 1e3, 2) for x in per]}
    s.close()
    del u64, u32, y32, y64, u16, y16
    torch.cuda.empty_cache()

    # ---- d = 3 (6-D phase space): the transport_3d workload (Kuhn cube meshes,
    # beta = (v, E(x)), sigma = 0) at level d3_L; FP32 and FP64 applies, the
    # handle's HBM footprint and the whole-apply algorithmic bandwidth
    d3 = None
    if args.d3_L >= 0:
        t0 = time.perf_counter()
        s3 = P.Solver(W.transport_3d(L=args.d3_L), device=local)
        setup3 = time.perf_counter() - t0
        n3 = s3.n_coeffs
        v64 = torch.tensor(W.uniform_vector(n3, seed=3 + rank), dtype=torch.float64, device="cuda")
        v32 = v64.float()
        w32, w64 = torch.empty_like(v32), torch.empty_like(v64)
        t0 = time.perf_counter()
        s3.autotune(v32, w32, P.SGDG_MIXED_FP32, stream)
        tune3 = time.perf_counter() - t0
        l0 = s3.launch_count()
        ms3 = timed(lambda: s3.apply_operator(v32, w32, P.SGDG_MIXED_FP32, stream), max(2, args.steps // 2), 2)
        launches3 = (s3.launch_count() - l0) // (max(2, args.steps // 2) + 2)
        ms3_64 = timed(lambda: s3.apply_operator(v64, w64, P.SGDG_FP64, stream), 2, 1)
        s3.apply_operator(v64, w64, P.SGDG_FP64, stream)
        s3.apply_operator(v32, w32, P.SGDG_MIXED_FP32, stream)
        err3 = float(torch.linalg.vector_norm(w32.double() - w64) / torch.linalg.vector_norm(w64))
        i3 = s3.info
        b3 = (n3 * (4 + 4) + 4 * (i3.rows_x + i3.rows_v + 2 * (i3.L + 1))
              + 4 * i3.nnz_x * (1 + i3.n_x_factors) + 4 * i3.nnz_v * (1 + i3.n_v_factors))
        s3.profile(True)
        s3.apply_operator(v32, w32, P.SGDG_MIXED_FP32, stream)
        st3 = s3.kernel_stats()
        s3.profile(False)
        tot3 = sum(v["ms"] for v in st3.values())
        d3 = {"workload": f"transport_3d d=3 L={args.d3_L} (6-D), Kuhn cube meshes, beta = (v, E(x)), sigma = 0, "
                          f"operator apply A^(delta) u",
              "dof_per_step": n3, "terms": i3.n_terms, "x_factors": i3.n_x_factors, "v_factors": i3.n_v_factors,
              "f32": {"value": whole_job(world, n3, ms3 * 1e-3) / 1e9, "unit": "GDoF/s", "ms_per_step": ms3},
              "f64": {"value": whole_job(world, n3, ms3_64 * 1e-3) / 1e9, "unit": "GDoF/s", "ms_per_step": ms3_64},
              "rel_err_f32_vs_fp64": err3,
              "hbm_footprint_bytes": i3.device_bytes,
              "roofline": {"bound": "hbm", "achieved": b3 / (ms3 * 1e-3) / 1e9, "peak": peak, "unit": "GB/s",
                           "frac": b3 / (ms3 * 1e-3) / 1e9 / peak, "alg_bytes_per_launch": b3,
                           "sweep_GBps": sum(v["bytes"] for v in st3.values()) / (tot3 * 1e-3) / 1e9},
              "launches_per_apply": launches3,
              "per_kind": per_kind(st3), "setup_s": round(setup3, 2), "autotune_s": round(tune3, 2)}
        log(f"d=3 L={args.d3_L}: FP32 {ms3:.2f} ms, FP64 {ms3_64:.2f} ms, {i3.device_bytes / 1e9:.1f} GB")
        s3.close()
        del v64, v32, w32, w64
        torch.cuda.empty_cache()

    # ---- strip solves at 1e-8 (mixed vs FP64), the d = 2 transport workload at
    # level strip_L, dt = 1/64: both arms start each strip from the linear
    # extrapolation of the last two solutions (warm start 3; the previous
    # solution on strip 2), so the ratio compares precisions only
    strip = None
    if args.strip_L >= 0:
        strip = {"workload": f"transport_2d d=2 L={args.strip_L} sigma=0.1 dt=1/64, rtol 1e-8, component solves "
                             f"GMRES({args.inner_its}) to {args.inner_rtol:g}, outer FGMRES(30); warm start: the previous solution "
                             f"(strip 2), then the extrapolation of the last two (both arms)"}
        for nm, pr, ns in (("mixed", P.SGDG_MIXED_FP32, args.strips_mixed), ("fp64", P.SGDG_FP64, args.strips_fp64)):
            if ns <= 0:
                continue
            ps = W.transport_2d(L=args.strip_L, sigma=0.1)
            t0 = time.perf_counter()
            sv = P.Solver(ps, precision=pr, rtol=1e-8, restart=30, inner_its=args.inner_its, inner_rtol=args.inner_rtol,
                          device=local)
            setup = time.perf_counter() - t0
            if pr == P.SGDG_MIXED_FP32:      # launch shapes of the FP32 applies the solve makes
                tu = torch.rand(sv.n_coeffs, dtype=torch.float32, device="cuda")
                sv.autotune(tu, torch.empty_like(tu), P.SGDG_MIXED_FP32, stream)
                del tu
            sv.set_warm_start(3)
            sv.set_initial()
            sts = []
            log(f"strip solver {nm}: set-up {setup:.1f} s")
            for _ in range(ns):
                r = sv.advance_strip(check=False)
                log(f"  strip {len(sts) + 1} {nm}: {r.seconds:.2f} s, outer {r.outer_its}, rel {r.rel_residual:.2e}")
                sts.append({"s": round(r.seconds, 4), "outer": r.outer_its, "inner": r.inner_its_total,
                            "applies": r.applies, "rel_res": r.rel_residual, "status": r.status})
            # strip 2 of both arms starts from the previous strip's solution (the
            # extrapolation needs two), strip 3 on from the extrapolation
            strip[nm] = {"s_per_strip": sts[1]["s"] if len(sts) > 1 else sts[0]["s"],
                         "statistic": "strip 2 (both arms: previous-solution start)",
                         "s_per_strip_extrapolated": (float(np.median([x["s"] for x in sts[2:]]))
                                                      if len(sts) > 2 else None),
                         "strips_timed": ns, "total_s": round(sum(x["s"] for x in sts), 3),
                         "max_rel_residual": max(x["rel_res"] for x in sts), "strips": sts,
                         "dof": sv.n_coeffs, "setup_s": round(setup, 2)}
            sv.close()
            torch.cuda.empty_cache()
        if "mixed" in strip and "fp64" in strip:
            strip["speedup_mixed_vs_fp64"] = strip["fp64"]["s_per_strip"] / strip["mixed"]["s_per_strip"]

    # ---- the batched apply at full size: 48 independent instances, L drawn
    # from {6, 7, 8, 9} (seed 0), every member's sweep captured into one CUDA
    # graph and replayed; FP32 and BF16 storage
    batch_apply = None
    if args.batch_apply > 0:
        probs = W.batched_4d(n=args.batch_apply, seed=0, levels=(6, 7, 8, 9))
        tb = time.perf_counter()
        solvers = [P.Solver(pr, precision=P.SGDG_MIXED_FP32, device=local) for pr in probs]
        bsetup = time.perf_counter() - tb
        dof = sum(sv.n_coeffs for sv in solvers)
        log(f"batched apply: {len(solvers)} handles set up in {bsetup:.1f} s")
        batch_apply = {"workload": f"{len(probs)} x transport_4d free streaming (beta = (v, 0)), "
                                   f"L drawn from {{6,7,8,9}} (seed 0)",
                       "levels": [p.L for p in probs], "dof_total": dof, "setup_s": round(bsetup, 2)}
        for nm, dt_, pr in (("f32", torch.float32, P.SGDG_MIXED_FP32), ("bf16", torch.bfloat16, P.SGDG_BF16_STORE)):
            bus = [torch.tensor(W.uniform_vector(sv.n_coeffs, seed=100 + k), device="cuda").to(dt_)
                   for k, sv in enumerate(solvers)]
            bys = [torch.empty_like(x) for x in bus]
            ta = time.perf_counter()
            tuned = {}                      # one autotuned handle per level; the others copy its shapes
            for sv, x, y, pb in zip(solvers, bus, bys, probs):
                if pb.L in tuned:
                    sv.copy_tuning(tuned[pb.L])
                else:
                    sv.autotune(x, y, pr, stream)
                    tuned[pb.L] = sv
            tune = time.perf_counter() - ta
            B = P.Batch(solvers)
            B.apply(bus, bys, pr, stream)          # capture
            l0 = sum(sv.launch_count() for sv in solvers)
            bms = timed(lambda: B.apply(bus, bys, pr, stream), args.steps, 2)
            batch_apply[nm] = {"apply_graph_ms": bms, "GDoFps": dof / (bms * 1e-3) / 1e9, "autotune_s": round(tune, 2)}
            log(f"batched apply {nm}: {bms:.2f} ms")
            B.close()
            del bus, bys
            torch.cuda.empty_cache()
        for sv in solvers:
            sv.close()
        torch.cuda.empty_cache()

    # ---- batched strips against the plain FP64 solver, on a reduced batch
    # (the Krylov bases of config 3's 48 instances at L 6-9 do not fit in HBM):
    # `batch` instances of uneven L, members concurrently; both arms start from
    # the extrapolated guess (warm start 3); strip 3 is timed (the first with
    # two earlier solutions to extrapolate from)
    batch = None
    if args.batch > 0:
        probs = W.batched_4d(n=args.batch, seed=0, levels=tuple(args.batch_levels))
        tb = time.perf_counter()
        solvers = [P.Solver(pr, precision=P.SGDG_MIXED_FP32, rtol=1e-8, restart=30, inner_its=12,
                            inner_rtol=1e-2, device=local) for pr in probs]
        bsetup = time.perf_counter() - tb
        bdof = sum(sv.n_coeffs for sv in solvers)
        bus = [torch.tensor(W.uniform_vector(sv.n_coeffs, seed=100 + k), dtype=torch.float32, device="cuda")
               for k, sv in enumerate(solvers)]
        bys = [torch.empty_like(x) for x in bus]
        for sv, x, y in zip(solvers, bus, bys):
            sv.autotune(x, y, P.SGDG_MIXED_FP32, stream)
        B = P.Batch(solvers)
        for sv in solvers:
            sv.set_warm_start(3)
            sv.set_initial()
        tstr = []
        for _ in range(3):
            t1 = time.perf_counter()
            st = B.advance()
            tstr.append(time.perf_counter() - t1)
            log(f"batched strip {len(tstr)}: {tstr[-1]:.2f} s")
        B.close()
        for sv in solvers:
            sv.close()
        t64, its64, res64 = 0.0, [], []
        for pr in probs:
            sv = P.Solver(pr, precision=P.SGDG_FP64, rtol=1e-8, restart=30, inner_its=12, inner_rtol=1e-2,
                          device=local)
            sv.set_warm_start(3)
            sv.set_initial()
            for k in range(3):
                r = sv.advance_strip(check=False)
            t64 += r.seconds
            its64.append(r.outer_its)
            res64.append(r.rel_residual)
            sv.close()
        batch = {"workload": f"{args.batch} x transport_4d free streaming, L from {sorted(set(p.L for p in probs))} "
                             f"(reduced from config 3's 48 at L 6-9: Krylov bases)",
                 "warm_start": "extrapolation of the last two strip solutions, both arms",
                 "levels": [p.L for p in probs], "dof_total": bdof,
                 "setup_s": round(bsetup, 2),
                 "s_per_batched_strip": round(tstr[-1], 4),
                 "max_rel_residual": max(x.rel_residual for x in st),
                 "outer_its": [x.outer_its for x in st],
                 "strips_per_s_batched_mixed": len(probs) / tstr[-1],
                 "plain_fp64": {"s_for_all_members": round(t64, 4), "strips_per_s": len(probs) / t64,
                                "outer_its": its64, "max_rel_residual": max(res64)},
                 "strips_per_s_ratio": (len(probs) / tstr[-1]) / (len(probs) / t64)}

    # ---- learned warm start (config-5 physics, Landau damping with the field
    # recomputed per strip): pairs from runs of the plain solver with seeded
    # amplitude and phase, the library's BF16 MLP trained on them, then
    # held-out seeds 100-103 solved from the extrapolated guess (the method
    # without the network) and from the learned one, at 1e-8
    warm = None
    if args.warmstart:
        from paper_2204_05988_gb300 import warmstart as WS

        def landau(seed):
            rng = np.random.default_rng(seed)
            return W.landau_4d(L=args.ws_L, alpha=float(rng.uniform(0.005, 0.02)),
                               phase=float(rng.uniform(0.0, 2.0 * np.pi)), n_strips=args.ws_strips)
        tw = time.perf_counter()
        pairs = WS.collect([landau(sd) for sd in range(args.ws_train_seeds)], n_strips=args.ws_strips, lx=2, lv=2)
        tcol = time.perf_counter() - tw
        tw = time.perf_counter()
        net, losses = WS.train(pairs, width=256, steps=2000, batch=32, lr=1e-3)
        ttrain = time.perf_counter() - tw
        log(f"warm start: {len(pairs.x)} pairs in {tcol:.1f} s, trained in {ttrain:.1f} s")
        ev = {"extrapolated": [], "learned": [], "previous": []}
        for sd in (100, 101, 102, 103):
            r = WS.evaluate(lambda sd=sd: landau(sd), net, n_strips=args.ws_strips, lx=2, lv=2)
            for k in ev:
                ev[k] += r[k][2:]
        warm = {"workload": f"landau_4d L={args.ws_L}, {args.ws_train_seeds} training seeds x {args.ws_strips} strips "
                            f"({len(pairs.x)} pairs), held-out seeds 100-103, strips 3-{args.ws_strips}, rtol 1e-8, "
                            f"mixed precision",
                "pairs": len(pairs.x), "collect_s": round(tcol, 2), "train_s": round(ttrain, 2),
                "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-20:]))}
        for k, v in ev.items():
            warm[k] = {"outer_its": int(sum(x[0] for x in v)), "seconds": round(sum(x[2] for x in v), 3),
                       "median_initial_rel_residual": float(np.median([x[1] for x in v])),
                       "max_rel_residual": float(max(x[3] for x in v))}
        warm["outer_its_learned_vs_extrapolated"] = warm["learned"]["outer_its"] / max(1, warm["extrapolated"]["outer_its"])
        warm["seconds_learned_vs_extrapolated"] = warm["learned"]["seconds"] / max(1e-9, warm["extrapolated"]["seconds"])
        net.close()

    if rank == 0:
        cpu = None
        if not args.no_cpu:
            log("cpu baseline")
            cpu, _, _ = cpu_baseline()
            log("cpu baseline done")
        line = {"metric": METRIC, "value": value, "unit": "GDoF/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms32, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": f"transport_2d d=2 L={args.L} sigma=0.1 operator apply A^(delta) u",
                           "dof_per_step": n, "unique_dof_per_step": unique,
                           "unique_GDoFps": unique / (ms32 * 1e-3) / 1e9 * world,
                           "terms": s.info.n_terms, "x_factors": s.info.n_x_factors,
                           "v_factors": s.info.n_v_factors, "l2": "inputs larger than L2 (493 MB f32)",
                           "parallelism": f"replicas x{world}", "setup_s": round(setup_s, 2),
                           "autotune_s": round(tune_s, 2)},
                "fp64_apply": {"value": whole_job(world, n, ms64 * 1e-3) / 1e9, "unit": "GDoF/s", "ms_per_step": ms64,
                               "roofline": fp64_roof},
                "bf16_apply": bf16_apply,
                "rel_err_vs_fp64_apply": {"f32": err32, "bf16_storage": err16},
                "gpu_launches": launches, "clocks": clocks, "roofline": roofline, "e2e": e2e,
                "strip": strip, "d3_apply": d3, "batch_apply": batch_apply, "batch": batch, "warm_start": warm,
                "cpu_baseline": cpu,
                "peaks": {"fp32_alu_gflops": fp32_peak, "fp32_source": fp32_peak_src,
                          "fp64_alu_gflops": fp64_peak, "fp64_source": fp64_peak_src,
                          "hbm_gbs": peak, "hbm_source": peak_kind}}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
