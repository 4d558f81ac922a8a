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


def test_null_context_arguments_are_refused(lib):
    """Every entry point that takes a context refuses a null one with
    QDT_ERR_ARG (-1) instead of crashing (no GPU touched)."""
    vp, i, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    calls = [
        ("qdt_set_route", [vp, i, i], (None, 0, 0)),
        ("qdt_check_bounded_wait", [vp, d], (None, 0.05)),
        ("qdt_f32_error_ratio", [vp, ctypes.c_uint, i, i, d, vp], (None, 1, 0, 1, 0.0, None)),
        ("qdt_set_coefficients", [vp, i, vp, vp], (None, 1, None, None)),
        ("qdt_set_spinor_coefficients", [vp, i, vp, vp], (None, 1, None, None)),
        ("qdt_set_rkb_coefficients", [vp, i, vp, vp, d, i], (None, 1, None, None, 137.0, 0)),
    ]
    for name, argtypes, args in calls:
        f = getattr(lib, name)
        f.argtypes = argtypes
        f.restype = ctypes.c_int
        assert f(*args) == -1, name
    lib.qdt_num_functions.argtypes = [vp]
    assert lib.qdt_num_functions(None) == 0


def test_unrestricted_packed_size_of_null_context_is_restricted_formula(lib):
    """Without a context the size is that of quaternion input (16 reals per
    canonical pair of Kramers pairs)."""
    lib.qdt_packed_size.restype = ctypes.c_size_t
    lib.qdt_packed_size.argtypes = [ctypes.c_void_p, ctypes.c_uint, ctypes.c_int, ctypes.c_int]
    assert lib.qdt_packed_size(None, 1, 3, 3) == 0
    assert lib.qdt_packed_size(None, 1, 2, 5) == 6 * 7 // 2 * 16 * 8
