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


def _host_problem(T, d, x, r, k, p):
    """A tnr_problem whose pointers are placeholders: only host-side planning may look at it."""
    A = T.tnr_mpo()
    A.d = d
    for i in range(d):
        A.I[i] = A.J[i] = x
        A.core[i] = 4096 * (i + 1)
    for i in range(d + 1):
        A.R[i] = 1 if i in (0, d) else r
    K, m, prod = k + p, 0, 1
    while prod < K:  # leading sites merged until prod I >= K (Section 6.3)
        prod *= x
        m += 1
    dm = d - max(m, 1) + 1
    U, V = T.tnr_mpo(), T.tnr_mpo()
    for M in (U, V):
        M.d = dm
        for i in range(dm):
            M.core[i] = 1 << 20
            M.cap[i] = 1 << 20
    return A, U, V


def test_persistent_batch_planning_on_the_host(lib):
    """tnr_batch_workspace plans every problem on the host (no device memory is touched), and
    tnr_batch_create refuses bad batch arguments before any device work."""
    import ctypes

    from paper_1707_07803_gb300 import tnrsvd as T

    keep = []
    probs = (T.tnr_problem * 2)()
    for i, (d, x, r, k) in enumerate([(4, 2, 2, 2), (5, 4, 3, 4)]):
        A, U, V = _host_problem(T, d, x, r, k, k)
        keep += [A, U, V]
        P = probs[i]
        P.A, P.U, P.V = ctypes.pointer(A), ctypes.pointer(U), ctypes.pointer(V)
        P.k, P.p, P.q, P.seed = k, k, 1, i
        P.S = 1 << 20
        P.opts = T._opts(1e-12, 2 * k, T.TNR_MIXED)
    b1, b2 = ctypes.c_size_t(0), ctypes.c_size_t(0)
    assert lib.tnr_batch_workspace(1, probs, ctypes.byref(b1)) == 0 and b1.value > 0
    assert lib.tnr_batch_workspace(2, probs, ctypes.byref(b2)) == 0 and b2.value > b1.value
    probs[1].k = 1 << 20  # K = k + p beyond prod I: refused by the plan
    assert lib.tnr_batch_workspace(2, probs, ctypes.byref(b2)) == -1
    h = ctypes.c_void_p(0)
    ws = ctypes.c_void_p(1 << 30)
    assert lib.tnr_batch_create(0, probs, 0, ws, 1 << 20, None, ctypes.byref(h)) == -1  # empty batch
    assert lib.tnr_batch_create(1, probs, 1 << 3, ws, 1 << 20, None, ctypes.byref(h)) == -1  # unknown flag bit
    assert lib.tnr_batch_create(1, probs, 0, None, 1 << 20, None, ctypes.byref(h)) == -1  # no workspace
    assert not h.value
    assert lib.tnr_batch_launch(None, None) == -1 and lib.tnr_batch_collect(None, None) == -1
    assert lib.tnr_batch_destroy(None) == 0


def test_noalloc_binding_checks_buffers_before_the_call():
    """The allocation-free conversion's binding rejects outputs that are too small, of the wrong
    dtype or not contiguous, and host tensors, before the library is called (no GPU needed)."""
    import torch

    from paper_1707_07803_gb300 import tnrsvd as T

    chk = T._need_buffer
    ok = torch.zeros(32, dtype=torch.float64)
    chk(ok, torch.float64, 32, "X", need_cuda=False)
    with pytest.raises(ValueError, match="room for 33"):
        chk(ok, torch.float64, 33, "X", need_cuda=False)
    with pytest.raises(ValueError, match="dtype"):
        chk(ok.float(), torch.float64, 8, "X", need_cuda=False)
    with pytest.raises(ValueError, match="contiguous"):
        chk(torch.zeros(8, 8, dtype=torch.float64).t(), torch.float64, 8, "X", need_cuda=False)
    with pytest.raises(ValueError, match="CUDA"):
        chk(None, torch.uint8, 0, "digits", need_cuda=False)
    rows = torch.arange(8, dtype=torch.int64)
    vals = torch.ones(8, dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):  # host tensors never reach the library
        T.tnr_sparse_to_mpo_noalloc(8, 8, rows, rows, vals, [2, 4], [2, 4], torch.zeros(32, dtype=torch.float64),
                                    torch.zeros(16, dtype=torch.uint8), max_blocks=8)
    with pytest.raises(ValueError, match="max_blocks"):
        T.tnr_sparse_to_mpo_noalloc(8, 8, rows, rows, vals, [2, 4], [2, 4], None, None, max_blocks=-1)


def test_zipup_planning_reaches_the_stated_batched_shapes(lib):
    """With the zip-up rounding the persistent batch plans problems of the stated batched sizes
    (ranks to 32, K to 64, d to 20), whose full products (2048-wide bonds) the two-sweep plan
    refuses; the single solve refuses the zip-up option (host-side checks only)."""
    import ctypes

    from paper_1707_07803_gb300 import tnrsvd as T

    keep = []
    shapes = [(20, 4, 32, 32), (20, 2, 32, 32), (8, 4, 4, 8), (14, 2, 17, 16)]
    probs = (T.tnr_problem * len(shapes))()
    for i, (d, x, r, k) in enumerate(shapes):
        A, U, V = _host_problem(T, d, x, r, k, k)
        keep += [A, U, V]
        P = probs[i]
        P.A, P.U, P.V = ctypes.pointer(A), ctypes.pointer(U), ctypes.pointer(V)
        P.k, P.p, P.q, P.seed = k, k, 1, i
        P.S = 1 << 20
        P.opts = T._opts(1e-12, 2 * k, T.TNR_MIXED, T.TNR_ROUND_ZIPUP)
    b = ctypes.c_size_t(0)
    assert lib.tnr_batch_workspace(len(shapes), probs, ctypes.byref(b)) == 0
    assert 0 < b.value < (1 << 30)  # well under a GB for these four problems
    two = T._opts(1e-12, 64, T.TNR_MIXED)
    probs[0].opts = two
    assert lib.tnr_batch_workspace(1, probs, ctypes.byref(b)) == -5  # two-sweep: products too wide
    probs[0].opts = T._opts(1e-12, 64, T.TNR_MIXED, 7)
    assert lib.tnr_batch_workspace(1, probs, ctypes.byref(b)) == -1  # unknown rounding
    zo = T._opts(1e-12, 64, T.TNR_FP64, T.TNR_ROUND_ZIPUP)
    S = ctypes.c_void_p(1 << 20)
    assert lib.tnr_solve(probs[2].A, 8, 8, 1, 0, ctypes.byref(zo), probs[2].U, S, probs[2].V, ctypes.c_void_p(1 << 20),
                         1 << 20, None) == -1


def test_flat_operator_layout_on_the_host():
    """Mpo.from_numpy(..., flat=True): the cores are views into one buffer, back to back in site
    order and in the memory order of the unflattened cores (checked on the CPU device), so one copy
    of its host image moves the whole operator."""
    import numpy as np

    from paper_1707_07803_gb300 import tnrsvd as T

    rng = np.random.default_rng(3)
    cores = [rng.standard_normal((1, 4, 3, 2)), rng.standard_normal((2, 5, 1, 3)), rng.standard_normal((3, 2, 2, 1))]
    A = T.Mpo.from_numpy(cores, device="cpu", flat=True)
    B = T.Mpo.from_numpy(cores, device="cpu")
    assert A.flat is not None and B.flat is None
    assert A.flat.numel() == sum(c.size for c in cores)
    off = 0
    for a, b, c in zip(A.cores, B.cores, cores):
        assert a.data_ptr() == A.flat.data_ptr() + 8 * off
        assert np.array_equal(a.numpy(), b.numpy())
        off += c.size
    assert A.R == B.R == [1, 2, 3, 1] and A.I == [4, 5, 2] and A.J == [3, 1, 2]
    assert [np.array_equal(x, y) for x, y in zip(A.to_numpy(), cores)] == [True] * 3
