"""The header as a plain C99 caller sees it (CPU only, no device calls):
`tests/c/abi_check.c` compiles with gcc against include/sgdg.h alone, links
the built libsgdg.so, and its struct sizes equal the library's
(sgdg_struct_sizes) - header/ABI drift that the Python binding's own layout
checks would not see fails here.  It also calls the host-only entry points
from C (mesh check, levels, embedding, a factor with a C callback) and
checks their results."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_c99_caller_matches_library_layouts(tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("gcc not available")
    from paper_2204_05988_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build.build()
    exe = tmp_path / "abi_check"
    libdir = os.path.dirname(LIB_PATH)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_check.c"), "-o", str(exe), "-L", libdir,
                    "-Wl,-rpath," + libdir, "-l:" + os.path.basename(LIB_PATH), "-lm"], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    rows = [l.split() for l in out.stdout.splitlines() if not l.startswith(("offset", "host calls"))]
    assert len(rows) == 10 and all(r[1] == r[2] for r in rows), out.stdout
    assert "host calls ok" in out.stdout, out.stdout
