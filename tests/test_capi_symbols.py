"""The C ABI library builds for sm_103a and exports every function declared in include/phicomb.h
(no compute call: runs without a GPU)."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"^[A-Za-z_][\w \*]*?\b(phic_\w+)\s*\(", src, flags=re.M))
    return names


def test_library_exports_every_declared_function():
    from paper_2509_26475_gb300 import build, capi

    build.build()
    lib = capi.load()
    declared = _declared()
    assert len(declared) >= 10
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    bound = {n for n, _, _ in capi.SIGNATURES}
    assert declared == bound, (declared ^ bound)
    assert lib.phic_version() >= 100
    assert lib.phic_status_string(4) == b"grid barrier wait timed out"


def test_host_queries_without_gpu():
    import ctypes

    from paper_2509_26475_gb300 import capi

    lib = capi.load(build_if_missing=True)
    out = ctypes.c_size_t(0)
    assert lib.phic_solve_workspace_size(262144, 1810432, 3, 2, 0, ctypes.byref(out)) == 0
    # A_1 copy (nnz doubles) + V x2, D x2, S (8 doubles/row) + F x2, E (4 doubles/row) + control
    assert out.value >= 1810432 * 8 + 262144 * 8 * (5 * 8 + 3 * 4)
    assert lib.phic_solve_workspace_size(10, 50, 16, 1, 0, ctypes.byref(out)) == capi.PHIC_INVALID_ARG
    assert lib.phic_select_workspace_size(1000, 61, ctypes.byref(out)) == 0
    assert out.value >= 1000 * 62 * 8


def test_binding_struct_layouts_match_the_library():
    """Every public struct has the same size in the ctypes binding as in the compiled library."""
    import ctypes

    from paper_2509_26475_gb300 import capi

    lib = capi.load(build_if_missing=True)
    count = lib.phic_struct_sizes(None, 0)
    assert count == len(capi.STRUCTS)
    sizes = (ctypes.c_size_t * count)()
    assert lib.phic_struct_sizes(sizes, count) == count
    for cls, size in zip(capi.STRUCTS, sizes):
        assert ctypes.sizeof(cls) == size, (cls.__name__, ctypes.sizeof(cls), size)
