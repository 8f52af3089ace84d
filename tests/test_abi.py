"""CPU checks of the boundary: the library builds, loads without a GPU and
exports every entry point include/llg.h declares; argument errors are caught
on the host (no device call is made for them)."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "llg.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?[a-z_ ]+\*?\s*\b(llg_[a-z0-9_]+)\s*\(", txt, flags=re.M)))


def test_header_and_binding_agree():
    from paper_2607_15290_b300 import _abi
    assert declared_symbols() == sorted(_abi.EXPORTS)


def test_library_exports_every_declared_symbol():
    from paper_2607_15290_b300 import _abi, build
    build.build()
    lib = C.CDLL(_abi.LIB_PATH)
    for name in declared_symbols():
        assert hasattr(lib, name), name


def test_host_side_argument_errors():
    from paper_2607_15290_b300 import _abi
    L = _abi.lib()
    g = _abi.Grid()
    g.dim = 2
    g.n[0], g.n[1], g.n[2] = 12, 16, 1          # 12 is not a power of two
    g.L[0] = g.L[1] = g.L[2] = 1.0
    h = C.c_void_p()
    assert L.llg_create(C.byref(g), None, C.byref(h)) == 2      # LLG_ERR_UNSUPPORTED_SIZE
    g.n[0] = 2048
    assert L.llg_create(C.byref(g), None, C.byref(h)) == 2
    g.n[0], g.dim = 16, 4
    assert L.llg_create(C.byref(g), None, C.byref(h)) == 1      # LLG_ERR_INVALID_ARG
    g.dim = 2
    g.L[1] = -1.0
    assert L.llg_create(C.byref(g), None, C.byref(h)) == 1
    assert L.llg_create(None, None, C.byref(h)) == 1
    assert L.llg_saddle_apply(None, None, None, None, None, 0) == 1
    assert L.llg_last_error(None) == b"null context"


def test_axis_shape_names():
    """The autotuner's shape names parse to the (kind, E, TW, CB) the C ABI takes."""
    from paper_2607_15290_b300 import parse_axis_shape
    assert parse_axis_shape("register(E8,TW16)") == (0, 8, 16, 0)
    assert parse_axis_shape("staged(TW32,CB16)") == (1, 8, 32, 16)
    assert parse_axis_shape("paired(E8,TW16)") == (3, 8, 16, 0)
    assert parse_axis_shape("tma(TW8)") == (4, 8, 8, 0)
    assert parse_axis_shape(" tma(E16,TW16) ") == (4, 16, 16, 0)
    for bad in ("tma", "tma()", "cufft(TW8)", "register(E8)", "register(E8,TW16,X3)"):
        with pytest.raises(ValueError):
            parse_axis_shape(bad)
