"""In-tree build of libsgdg.so for sm_103a (nvcc + g++, no cmake).

Compiles every translation unit in ``csrc/`` in parallel and links the shared
library into ``_lib/libsgdg.so`` next to this file.  ``python -m
paper_2204_05988_gb300.build`` or ``build()`` from Python.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT_DIR, "libsgdg.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc() -> str:
    for c in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libsgdg")


def _sources():
    cu = sorted(f for f in os.listdir(CSRC) if f.endswith(".cu"))
    cpp = sorted(f for f in os.listdir(CSRC) if f.endswith(".cpp"))
    return cu, cpp


def _run(cmd):
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("build failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
    return r.stdout + r.stderr


def build(verbose: bool = False, ptxas_v: bool = False) -> str:
    nvcc = _nvcc()
    obj_dir = os.path.join(OUT_DIR, "obj")
    os.makedirs(obj_dir, exist_ok=True)
    cu, cpp = _sources()
    inc = ["-I", os.path.join(os.path.dirname(HERE), "include")]
    cmds = []
    objs = []
    for f in cu:
        o = os.path.join(obj_dir, f + ".o")
        objs.append(o)
        cmd = [nvcc, *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-fopenmp",
               "--expt-relaxed-constexpr", *inc, "-c", os.path.join(CSRC, f), "-o", o]
        if ptxas_v:
            cmd.insert(1, "-Xptxas=-v")
        cmds.append(cmd)
    for f in cpp:
        o = os.path.join(obj_dir, f + ".o")
        objs.append(o)
        cmds.append(["g++", "-O3", "-std=c++17", "-fPIC", "-fopenmp", *inc,
                     "-I", "/usr/local/cuda/include", "-c", os.path.join(CSRC, f), "-o", o])
    with cf.ThreadPoolExecutor(max_workers=max(2, os.cpu_count() or 2)) as ex:
        outs = list(ex.map(_run, cmds))
    if verbose:
        for o in outs:
            if o.strip():
                print(o)
    tmp = LIB + ".tmp"
    _run([nvcc, *ARCH, "-shared", "-Xcompiler", "-fopenmp", "-o", tmp, *objs, "-lcudart", "-lgomp"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(verbose=True, ptxas_v="-v" in sys.argv))
