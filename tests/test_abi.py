"""The C-ABI library loads and exports every entry point include/sgdg.h declares
(CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "sgdg.h")) as f:
        src = f.read()
    return sorted(set(re.findall(r"^\s*(?:sgdg_status|void|const char\*|long long|int)\s+(sgdg_\w+)\s*\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_05988_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build.build()
    return ctypes.CDLL(LIB_PATH)


def test_header_declares_entry_points():
    names = _declared()
    assert "sgdg_create" in names and "sgdg_apply_operator" in names and len(names) >= 15


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_declares_exactly_the_header(lib):
    from paper_2204_05988_gb300 import EXPORTS
    assert sorted(EXPORTS) == _declared()


def test_binding_fails_loudly_without_library(tmp_path):
    import paper_2204_05988_gb300 as P
    saved = P._lib
    P._lib = None
    try:
        with pytest.raises(RuntimeError):
            P.load_library(str(tmp_path / "missing.so"))
    finally:
        P._lib = saved


def test_binding_structs_match_the_library_layouts(lib):
    """ctypes structures of the binding have the sizes the library compiled
    (a field missing on either side changes them)."""
    import ctypes as C
    import paper_2204_05988_gb300 as P
    out = (C.c_int * 10)()
    assert lib.sgdg_struct_sizes(out, 10) == 10
    mine = [C.sizeof(t) for t in (P.Mesh, P.Product, P.Source, P.Coeffs, P.Config, P.Info, P.StripStats,
                                  P.KernelStat, P.CheckpointInfo, P.FactorSpec)]
    assert list(out) == mine


def test_binding_rejects_p2_problems():
    """The library's spaces are continuous P1 on simplices; a problem asking
    for P2 or for tensor-product Q elements (the oracle's r = 2 and Q_r paths)
    is refused before anything reaches the device."""
    import paper_2204_05988_gb300 as P
    import sgdg_workloads as W
    with pytest.raises(ValueError):
        P.Solver(W.periodic_advection_1d(L=1, r=2))
    with pytest.raises(ValueError):
        P.Solver(W.periodic_advection_2d(L=1, element="Q"))
