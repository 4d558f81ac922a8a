"""The C-ABI library loads and exports every entry point that include/*.h
declares (no GPU needed: nothing here launches work)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        txt = open(h).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        for m in re.finditer(r"\b(qdt_[a-z0-9_]+)\s*\(", txt):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_2606_04316_gb300 import build
    build.build()
    return ctypes.CDLL(build.LIB)


def test_every_declared_symbol_is_exported(lib):
    names = declared_symbols()
    assert {"qdt_create", "qdt_transform", "qdt_set_basis", "qdt_set_coefficients"} <= names
    for n in sorted(names):
        assert hasattr(lib, n), n


def test_binding_names_match_header():
    from paper_2606_04316_gb300 import qdt
    assert set(qdt.EXPORTS) == declared_symbols()


def test_version_and_null_context(lib):
    lib.qdt_version.restype = ctypes.c_char_p
    assert lib.qdt_version().startswith(b"qdt")
    lib.qdt_last_error.restype = ctypes.c_char_p
    lib.qdt_last_error.argtypes = [ctypes.c_void_p]
    assert lib.qdt_last_error(None) == b"null context"
    lib.qdt_transform.argtypes = [ctypes.c_void_p, ctypes.c_uint, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_size_t,
                                  ctypes.c_void_p]
    assert lib.qdt_transform(None, 1, 0, 1, 0.0, 0, None, 0, None) == -1


def test_packed_size_formula(lib):
    lib.qdt_packed_size.restype = ctypes.c_size_t
    lib.qdt_packed_size.argtypes = [ctypes.c_void_p, ctypes.c_uint, ctypes.c_int, ctypes.c_int]
    n = 40
    nP = n * (n + 1) // 2
    assert lib.qdt_packed_size(None, 1, 0, n) == nP * (nP + 1) // 2 * 16 * 8
    assert lib.qdt_packed_size(None, 7, 0, n) == 3 * nP * (nP + 1) // 2 * 16 * 8
