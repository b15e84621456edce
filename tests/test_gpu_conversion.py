"""GPU parity for Alg. 4.1 (sparse -> MPO): bit-exact against the oracle, through the C ABI."""

import numpy as np
import pytest
import torch

from oracle import convert as oc
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import coo_to_device
from workloads import banded_coo

pytestmark = pytest.mark.gpu


def _gpu_convert(rows, cols, vals, nrows, ncols, I, J):
    r, c, v = coo_to_device(rows, cols, vals)
    R, X, digits = T.sparse_to_mpo(nrows, ncols, r, c, v, I, J)
    torch.cuda.synchronize()
    return R, X.cpu().numpy(), digits.cpu().numpy()


def _assert_same(got, want):
    Rg, Xg, Dg = got
    Rw, Xw, Dw = want
    assert Rg == Rw
    assert Xg.tobytes() == Xw.tobytes()  # bit-exact, including +0.0 fill
    assert Dg.reshape(Rw, -1).tobytes() == Dw.tobytes()


def _coo(D):
    r, c = np.nonzero(D)
    return r.astype(np.int64), c.astype(np.int64), D[r, c]


def test_paper_examples():
    A = np.zeros((2, 6))
    A[0, 0], A[1, 3] = 2.0, -5.0
    _assert_same(_gpu_convert(*_coo(A), 2, 6, [1, 1, 2], [1, 3, 2]), oc.convert(*_coo(A), 2, 6, [1, 1, 2], [1, 3, 2]))
    rng = np.random.default_rng(0)
    D = np.zeros((12, 12))
    for p, q in [(0, 3), (1, 1), (2, 2)]:
        D[3 * p:3 * p + 3, 3 * q:3 * q + 3] = rng.standard_normal((3, 3))
    _assert_same(_gpu_convert(*_coo(D), 12, 12, [3, 4], [3, 4]), oc.convert(*_coo(D), 12, 12, [3, 4], [3, 4]))


@pytest.mark.parametrize("I,J,density,seed", [
    ([4, 2, 3, 2], [2, 4, 2, 3], 0.05, 0),
    ([3, 5, 7], [2, 3, 5], 0.02, 1),       # ragged, non-power-of-two factors
    ([16, 4, 4], [16, 4, 4], 0.01, 2),     # 1024 x 1024: several tiles of 1024 entries
    ([64, 4, 4], [8, 4, 4], 0.03, 3),      # I1 = 64 rows per block-row
    ([5], [7], 0.3, 4),                    # d = 1: a single block
    ([1, 1, 2], [1, 3, 2], 0.5, 5),        # 1 x 1 blocks: rank = nnz
    ([8, 8], [8, 8], 1.0, 6),              # dense
])
def test_random_sparse_bit_exact(I, J, density, seed):
    rng = np.random.default_rng(seed)
    nr, nc = int(np.prod(I)), int(np.prod(J))
    D = np.where(rng.random((nr, nc)) < density, rng.standard_normal((nr, nc)), 0.0)
    rows, cols, vals = _coo(D)
    want = oc.convert(rows, cols, vals, nr, nc, I, J)
    got = _gpu_convert(rows, cols, vals, nr, nc, I, J)
    _assert_same(got, want)


def test_explicit_zero_values_make_blocks():
    rows = np.array([0, 5], dtype=np.int64)
    cols = np.array([1, 6], dtype=np.int64)
    vals = np.array([0.0, 3.0])
    want = oc.convert(rows, cols, vals, 8, 8, [2, 4], [2, 4])
    assert want[0] == 2
    _assert_same(_gpu_convert(rows, cols, vals, 8, 8, [2, 4], [2, 4]), want)


def test_empty():
    r, c, v = coo_to_device(np.zeros(0, np.int64), np.zeros(0, np.int64), np.zeros(0))
    R, X, digits = T.sparse_to_mpo(16, 16, r, c, v, [4, 4], [4, 4])
    assert R == 0 and X.numel() == 0


@pytest.mark.parametrize("kind", ["unsorted", "duplicate", "range"])
def test_rejects_bad_coo(kind):
    rows = np.array([0, 1, 2, 3], dtype=np.int64)
    cols = np.array([0, 1, 2, 3], dtype=np.int64)
    vals = np.ones(4)
    expect = {"unsorted": -3, "duplicate": -2, "range": -8}[kind]
    if kind == "unsorted":
        rows = rows[::-1].copy()
        cols = cols[::-1].copy()
    elif kind == "duplicate":
        rows[2], cols[2] = rows[1], cols[1]
    else:
        cols[3] = 99
    r, c, v = coo_to_device(rows, cols, vals)
    with pytest.raises(T.TnrError) as e:
        T.sparse_to_mpo(16, 16, r, c, v, [4, 4], [4, 4])
    assert e.value.status == expect


def test_banded_2pow20_bit_exact():
    """Full-size banded workload: 2^20 x 2^20, 8 nonzeros per row within half-band 64, ten 4x4 sites."""
    n = 1 << 20
    rows, cols, vals = banded_coo(0, n, 8, 64)
    I = J = [4] * 10
    want = oc.convert(rows, cols, vals, n, n, I, J)
    got = _gpu_convert(rows, cols, vals, n, n, I, J)
    assert want[0] > 5_000_000
    _assert_same(got, want)


def test_short_and_long_block_rows_in_one_matrix():
    """Block-rows assembled whole in shared memory (short segments) next to block-rows with more
    than 64 entries or more block values than the warp's buffer (left to the scatter fill), in one
    conversion; bit-exact against the oracle."""
    rng = np.random.default_rng(12)
    I, J = [4, 8, 8], [4, 8, 8]
    n = 256
    D = np.where(rng.random((n, n)) < 0.01, rng.standard_normal((n, n)), 0.0)
    for r in (5, 6, 77, 200):  # dense rows: their block-rows have > 64 entries
        D[r] = rng.standard_normal(n)
    D[130:134, :] = np.where(rng.random((4, n)) < 0.3, 1.5, 0.0)  # many blocks (nb * 16 > 512)
    rows, cols, vals = _coo(D)
    _assert_same(_gpu_convert(rows, cols, vals, n, n, I, J), oc.convert(rows, cols, vals, n, n, I, J))


def test_wide_matrix_with_64_bit_block_columns():
    """64 x 2^33 (sites 4 x 4, 4 x 256, 4 x 256, 1 x 256, 1 x 128): block columns beyond 2^30 take
    the 64-bit rank and digit paths of the block-row fill; bit-exact against the oracle."""
    rng = np.random.default_rng(21)
    I, J = [4, 4, 4, 1, 1], [4, 256, 256, 256, 128]
    nr, nc = 64, 1 << 33
    rows, cols = [], []
    for r in range(nr):
        cs = np.unique(rng.integers(0, nc, size=7))  # 28 entries per block-row: the whole-block path
        rows += [r] * cs.size
        cols += list(cs)
    rows = np.array(rows, dtype=np.int64)
    cols = np.array(cols, dtype=np.int64)
    vals = rng.standard_normal(rows.size)
    vals[vals == 0.0] = 1.0
    _assert_same(_gpu_convert(rows, cols, vals, nr, nc, I, J), oc.convert(rows, cols, vals, nr, nc, I, J))
