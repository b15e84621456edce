"""The C-ABI library builds, loads and exports every entry point declared in include/tnrsvd.h
(no compute calls: this runs without a GPU)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "tnrsvd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"\b(tnr_[a-z0-9_]+)\s*\(", src)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_1707_07803_gb300 import build, tnrsvd

    if not os.path.exists(tnrsvd.LIB_PATH):
        build.build()
    return tnrsvd.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 14
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_1707_07803_gb300 import tnrsvd

    assert sorted(tnrsvd.exported_names()) == _declared()


def test_host_side_argument_errors(lib):
    """Argument validation happens on the host before any device work (no GPU needed)."""
    import ctypes

    from paper_1707_07803_gb300 import tnrsvd as T

    b = ctypes.c_size_t(0)
    I = (ctypes.c_int64 * 2)(2, 3)
    J = (ctypes.c_int64 * 2)(2, 2)
    assert lib.tnr_sparse_workspace(4, 4, 10, 2, I, J, ctypes.byref(b)) == -1  # prod I = 6 != 4
    I2 = (ctypes.c_int64 * 2)(2, 2)
    assert lib.tnr_sparse_workspace(4, 4, 10, 2, I2, J, ctypes.byref(b)) == 0 and b.value > 0
    assert lib.tnr_strerror(-2) == b"duplicate (row, col) entry in the COO input"
    m = T.tnr_mpo()
    m.d = 0
    o = T._opts(0.0, 0, 0)
    assert lib.tnr_solve_query(ctypes.byref(m), 4, 4, ctypes.byref(o), None, None, ctypes.byref(b)) == -1
    # batched solve: bad batch arguments are rejected before any device work
    P = (T.tnr_problem * 1)()
    assert lib.tnr_solve_batched(-1, P, 0, None, 256, None) == -1
    assert lib.tnr_solve_batched(1, P, 0, None, 256, None) == -1  # no workspace
    assert lib.tnr_solve_batched(1, P, 64, ctypes.c_void_p(256), 256, None) == -1  # more workers than status slots
    assert lib.tnr_solve_batched(1, P, 1, ctypes.c_void_p(256), 100, None) == -1  # stride not a multiple of 256
    assert lib.tnr_solve_batched(0, None, 0, None, 0, None) == 0  # empty batch
