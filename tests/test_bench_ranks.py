"""The multi-GPU path of bench.py on the host cores (no GPU): the replicas'
barrier and max-over-ranks timing over a world-size-2 gloo group, the
whole-job aggregate, and the reference arm under torchrun, where rank 0
alone runs and prints."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402

pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


_RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="env://")
rk = bench.Ranks(dist, "cpu")
rank = dist.get_rank()
rk.barrier()
t = rk.max([1.5, 3.25][rank])
print(json.dumps({{"rank": rank, "max": t, "value": bench.whole_job(dist.get_world_size(), 10.0, t)}}))
dist.destroy_process_group()
"""


def test_max_over_two_gloo_ranks():
    port = _free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
        procs.append(subprocess.Popen([sys.executable, "-c", _RANK_SCRIPT.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=120)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    assert sorted(o["rank"] for o in outs) == [0, 1]
    for o in outs:
        assert o["max"] == 3.25                      # the slowest rank's time, on every rank
        assert o["value"] == pytest.approx(2 * 10.0 / 3.25)


def test_single_process_ranks_and_aggregate():
    rk = bench.Ranks()
    rk.barrier()
    assert rk.max(2.5) == 2.5
    assert bench.whole_job(1, 123.0, 2.0) == 61.5
    assert bench.whole_job(4, 123.0, 2.0) == 4 * bench.whole_job(1, 123.0, 2.0)


def test_reference_arm_under_torchrun():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--ref-L", "2"]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1                            # rank 0 alone prints
    ln = lines[0]
    assert ln["impl"] == "reference" and ln["n_gpus"] == 2 and ln["value"] > 0
    assert ln["cpu_baseline"]["kind"] == "oracle" and ln["e2e"]["h2d_bytes_per_step"] == 0
