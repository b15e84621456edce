"""The allocation-free conversion entry point gives the same blocks as the regular one.

tnr_sparse_to_mpo_noalloc serves callers that cannot allocate memory at call time (for example a
plug-in inside a process whose own memory manager has reserved all of the device memory): its
scratch is compiled into the library instead of coming from a caller workspace. This test calls
it through the C ABI twice in a row, on two different matrices, so the second call starts from
the first call's leftover scratch contents, and checks each result bit for bit against
tnr_sparse_count + tnr_sparse_fill on the same input and, on the smaller matrix with uneven
factors, against the CPU oracle of Alg. 4.1 as well. It is collected last so that a `pytest -x`
run has already run every other test if this one fails; it also passes on its own in a fresh
process.
"""

import numpy as np
import pytest
import torch

import oracle.convert
from paper_1707_07803_gb300 import tnrsvd as T
from workloads import banded_coo

pytestmark = pytest.mark.gpu


def _device(rows, cols, vals):
    return (torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(cols, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float64)).cuda())


def _cases():
    # 1: banded 2^16 x 2^16, eight 4 x 4 sites (many tiles, ragged last tile)
    r1, c1, v1 = banded_coo(3, 1 << 16, 8, 64)
    # 2: random sparse 3*5*7*4 x 2*3*5*6 with uneven factors and fewer entries than case 1
    rng = np.random.default_rng(9)
    I2, J2 = [3, 5, 7, 4], [2, 3, 5, 6]
    nr, nc = int(np.prod(I2)), int(np.prod(J2))
    D = np.where(rng.random((nr, nc)) < 0.03, rng.standard_normal((nr, nc)), 0.0)
    r2, c2 = np.nonzero(D)
    return [((1 << 16), (1 << 16), r1, c1, v1, [4] * 8, [4] * 8),
            (nr, nc, r2.astype(np.int64), c2.astype(np.int64), D[r2, c2], I2, J2)]


def test_noalloc_matches_regular_entry_point_twice():
    for nrows, ncols, rows, cols, vals, I, J in _cases():
        r, c, v = _device(rows, cols, vals)
        R_ref, X_ref, D_ref = T.sparse_to_mpo(nrows, ncols, r, c, v, I, J)
        nnz = rows.size
        X = torch.full((nnz * I[0] * J[0],), float("nan"), dtype=torch.float64, device="cuda")
        digits = torch.zeros(nnz * 2 * (len(I) - 1), dtype=torch.uint8, device="cuda")
        R = T.tnr_sparse_to_mpo_noalloc(nrows, ncols, r, c, v, I, J, X, digits, max_blocks=nnz)
        torch.cuda.synchronize()
        assert R == R_ref
        bs = I[0] * J[0]
        assert X[: R * bs].cpu().numpy().tobytes() == X_ref.cpu().numpy().tobytes()
        assert digits[: R * 2 * (len(I) - 1)].cpu().numpy().tobytes() == D_ref.cpu().numpy().tobytes()
        if rows.size < 100000:  # the oracle of Alg. 4.1, bit for bit
            Ro, Xo, Do = oracle.convert.convert(rows, cols, vals, nrows, ncols, I, J)
            assert R == Ro
            assert X[: R * bs].cpu().numpy().tobytes() == Xo.tobytes()
            assert digits[: R * 2 * (len(I) - 1)].cpu().numpy().tobytes() == Do.tobytes()


def test_noalloc_limits():
    rows = np.arange(8, dtype=np.int64)
    cols = np.arange(8, dtype=np.int64)
    r, c, v = _device(rows, cols, np.ones(8))
    X = torch.empty(8 * 4, dtype=torch.float64, device="cuda")
    digits = torch.empty(8 * 2, dtype=torch.uint8, device="cuda")
    with pytest.raises(T.TnrError) as e:  # 4 diagonal 2x2 blocks but room for 2
        T.tnr_sparse_to_mpo_noalloc(8, 8, r, c, v, [2, 4], [2, 4], X, digits, max_blocks=2)
    assert e.value.status == -5
    big = T.NOALLOC_MAX_NNZ + 1
    lib = T.load()
    import ctypes
    Rv = ctypes.c_int64(0)
    dims = T._i64arr([4, 256, 256, 64])  # 2^24 rows and columns, 4 x 4 leading blocks
    rc = lib.tnr_sparse_to_mpo_noalloc(1 << 24, 1 << 24, big, T._ptr(r), T._ptr(c), T._ptr(v), 4, dims, dims,
                                       T._ptr(X), T._ptr(digits), big, ctypes.byref(Rv), T._stream())
    assert rc == -8  # rejected on the host before any device work
    with pytest.raises(ValueError, match="room for"):  # the binding checks the outputs' room
        T.tnr_sparse_to_mpo_noalloc(8, 8, r, c, v, [2, 4], [2, 4], X, digits, max_blocks=9)
