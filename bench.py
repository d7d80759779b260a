"""Benchmark: sparse-grid SD-Galerkin operator apply (GDoF/s) and strip solves.

Workload (default): the 4D transport problem, d = 2, Omega_x = [0,1]^2,
Omega_v = [-1,1]^2, 8-triangle coarse meshes, sparse level L = 9 (grids
(l, 9-l)), time-DG degree 1, beta = (v, E(x)), sigma = 0.1: 61,590,186 spatial
coefficients, 123,180,372 DoF per strip vector (FP32: 493 MB, FP64: 985 MB,
both larger than L2).  A step is one application of the strip operator
A^(delta) to a seeded U[-1,1] vector, resident in HBM.

Reported: value = GDoF/s of the mixed-precision (FP32) apply; the FP64 apply,
the end-to-end apply through the C ABI with host buffers, per-kernel roofline,
strip solves at 1e-8 (mixed vs FP64), the oracle timed on the host cores.

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


# ALU peaks derived from the unit counts and the maximum SM clock (2,070 MHz):
# FP32 - 152 SMs x 128 FP32 lanes x 2 flops per multiply-add; FP64 - the
# nominal GB300 non-tensor FP64 rate (1.25 TFLOP/s), far below FP32.
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


def whole_job(world: int, units_per_rank: float, seconds: float) -> float:
    """Weak scaling: every rank processes units_per_rank; `seconds` is the
    slowest rank's time, so the job's rate is world x units / seconds."""
    return world * units_per_rank / seconds


def cpu_baseline(steps: int = 4, L: int = 5):
    """The oracle's blockwise apply (Sect. 4.2) on the host cores, as it stands,
    on a bounded sample of the same workload family (d = 2, level L)."""
    from oracle.operator import SparseGridOperator
    prob = W.transport_2d(L=L, sigma=0.1)
    op = SparseGridOperator(prob)
    u = W.uniform_vector(op.size, seed=7)
    op.apply(u)                                     # warm-up: builds the projected factors
    t = time.perf_counter()
    for _ in range(steps):
        op.apply(u)
    dt = (time.perf_counter() - t) / steps
    return {"value": op.size / dt / 1e9, "unit": "GDoF/s", "cores": 1, "kind": "oracle",
            "sample": f"blockwise FP64 apply, d=2 L={L} ({op.size} DoF), {steps} applies after 1 warm-up; "
                      f"numpy/scipy single thread"}, dt, op.size


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
    ap.add_argument("--strip-L", type=int, default=7, help="level of the strip-solve timing (-1: skip)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--batch", type=int, default=8, help="instances in the batch measurement (0: skip)")
    ap.add_argument("--batch-levels", type=int, nargs="+", default=[5, 6, 7])
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
                 "achieved": st64[dom64]["flops"] / (st64[dom64]["ms"] * 1e-3) / 1e9, "peak": FP64_PEAK_GFLOPS,
                 "unit": "GFLOP/s", "peak_source": "nominal GB300 FP64 rate",
                 "frac": st64[dom64]["flops"] / (st64[dom64]["ms"] * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                 "apply_GFLOPs": fl64 / (tot64 * 1e-3) / 1e9, "apply_frac": fl64 / (tot64 * 1e-3) / 1e9 / FP64_PEAK_GFLOPS,
                 "share_of_apply": st64[dom64]["ms"] / tot64}
    # whole-apply effective bandwidth: the bytes the method must move per apply
    # (read u, write y, every pattern once, every factor value array once),
    # independent of the sweep's intermediates
    inf = s.info
    b_alg = (n * (4 + 4) + 4 * (inf.rows_x + inf.rows_v + 2 * (inf.L + 1))
             + 4 * inf.nnz_x * (1 + inf.n_x_factors) + 4 * inf.nnz_v * (1 + inf.n_v_factors))
    roofline = {"bound": "hbm", "kernel": dom, "achieved": ach, "peak": peak, "unit": "GB/s",
                "frac": ach / peak, "peak_source": f"{peak_kind} hbm_gbs", "traffic": _traffic(dom, args.L),
                "alg_bytes_per_launch": st[dom]["bytes"] / max(1, st[dom]["launches"]),
                "share_of_apply": st[dom]["ms"] / tot_ms,
                "apply_effective": {"b_alg_bytes": b_alg, "GBps": b_alg / (ms32 * 1e-3) / 1e9,
                                    "frac": b_alg / (ms32 * 1e-3) / 1e9 / peak,
                                    "sweep_bytes": sum(v["bytes"] for v in st.values()),
                                    "sweep_GBps": sum(v["bytes"] for v in st.values()) / (tot_ms * 1e-3) / 1e9},
                "fp32_alu": {"achieved": st[dom]["flops"] / (st[dom]["ms"] * 1e-3) / 1e9, "peak": FP32_PEAK_GFLOPS,
                             "unit": "GFLOP/s",
                             "frac": st[dom]["flops"] / (st[dom]["ms"] * 1e-3) / 1e9 / FP32_PEAK_GFLOPS},
                "per_kind": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                 "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None,
                                 "GFLOPs": (v["flops"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                             for k, v in st.items() if v["launches"]},
                "f64_per_kind": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                                     "GBps": (v["bytes"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None,
                                     "GFLOPs": (v["flops"] / (v["ms"] * 1e-3) / 1e9) if v["ms"] > 0 else None}
                                 for k, v in roof["f64"].items() if v["launches"]}}
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

    # ---- strip solves at 1e-8 (mixed vs FP64)
    strip = None
    if args.strip_L >= 0:
        strip = {"workload": f"transport_2d d=2 L={args.strip_L} sigma=0.1 dt=1/64, strips 1-2, rtol 1e-8"}
        for nm, pr in (("mixed", P.SGDG_MIXED_FP32), ("fp64", P.SGDG_FP64)):
            ps = W.transport_2d(L=args.strip_L, sigma=0.1)
            sv = P.Solver(ps, precision=pr, rtol=1e-8, restart=30, inner_its=12, inner_rtol=1e-2, device=local)
            sv.set_initial()
            sts = []
            for _ in range(2):
                r = sv.advance_strip(check=False)
                sts.append({"s": round(r.seconds, 4), "outer": r.outer_its, "inner": r.inner_its_total,
                            "applies": r.applies, "rel_res": r.rel_residual, "status": r.status})
            strip[nm] = {"s_per_strip": sts[-1]["s"], "strips": sts, "dof": sv.n_coeffs}
            sv.close()
        strip["speedup_mixed_vs_fp64"] = strip["fp64"]["s_per_strip"] / strip["mixed"]["s_per_strip"]

    # ---- batch of independent instances of uneven L: one CUDA graph per apply,
    # concurrent strip solves
    batch = None
    if args.batch > 0:
        probs = W.batched_4d(n=args.batch, seed=0, levels=tuple(args.batch_levels))
        tb = time.perf_counter()
        solvers = [P.Solver(pr, precision=P.SGDG_MIXED_FP32, rtol=1e-8, restart=30, inner_its=12,
                            inner_rtol=1e-2, device=local) for pr in probs]
        bsetup = time.perf_counter() - tb
        bus = [torch.tensor(W.uniform_vector(sv.n_coeffs, seed=100 + k), dtype=torch.float32, device="cuda")
               for k, sv in enumerate(solvers)]
        bys = [torch.empty_like(x) for x in bus]
        for sv, x, y in zip(solvers, bus, bys):
            sv.autotune(x, y, P.SGDG_MIXED_FP32, stream)
        B = P.Batch(solvers)
        B.apply(bus, bys, P.SGDG_MIXED_FP32, stream)          # capture
        bms = timed(lambda: B.apply(bus, bys, P.SGDG_MIXED_FP32, stream), args.steps, 1)
        dof = sum(sv.n_coeffs for sv in solvers)
        # batched mixed precision with the extrapolated guess (warm start 3):
        # all members concurrently; strip 3 is timed (the first with two
        # earlier solutions to extrapolate from)
        for sv in solvers:
            sv.set_warm_start(3)
            sv.set_initial()
        tstr = []
        for _ in range(3):
            t1 = time.perf_counter()
            st = B.advance()
            tstr.append(time.perf_counter() - t1)
        B.close()
        for sv in solvers:
            sv.close()
        # the plain FP64 solver on the same instances, one after another,
        # previous-strip guess; strip 3 of each is timed
        t64, its64, res64 = 0.0, [], []
        for pr in probs:
            sv = P.Solver(pr, precision=P.SGDG_FP64, rtol=1e-8, restart=30, inner_its=12, inner_rtol=1e-2,
                          device=local)
            sv.set_warm_start(1)
            sv.set_initial()
            for k in range(3):
                r = sv.advance_strip(check=False)
            t64 += r.seconds
            its64.append(r.outer_its)
            res64.append(r.rel_residual)
            sv.close()
        batch = {"workload": f"{args.batch} x transport_4d free streaming, L from {sorted(set(p.L for p in probs))}",
                 "levels": [p.L for p in probs], "dof_total": dof, "setup_s": round(bsetup, 2),
                 "apply_graph_ms": bms, "apply_GDoFps": dof / (bms * 1e-3) / 1e9,
                 "s_per_batched_strip": round(tstr[-1], 4),
                 "max_rel_residual": max(x.rel_residual for x in st),
                 "outer_its": [x.outer_its for x in st],
                 "strips_per_s_batched_mixed": len(probs) / tstr[-1],
                 "plain_fp64": {"s_for_all_members": round(t64, 4), "strips_per_s": len(probs) / t64,
                                "outer_its": its64, "max_rel_residual": max(res64)},
                 "strips_per_s_ratio": (len(probs) / tstr[-1]) / (len(probs) / t64)}

    if rank == 0:
        cpu = None
        if not args.no_cpu:
            cpu, _, _ = cpu_baseline()
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
                "strip": strip, "batch": batch, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
