"""Pins for the Alg. 4.1 oracle (Section 4): paper examples, Lemmas 4.2/4.3, exact reconstruction."""

import numpy as np
import pytest

from oracle import convert, mpo, rounding
from tests.conftest import golden_path
from workloads import banded_coo


def _coo(D):
    r, c = np.nonzero(D)
    return r.astype(np.int64), c.astype(np.int64), D[r, c]


def _golden_2x6():
    g = {"digits": []}
    lines = [l.strip() for l in open(golden_path("conversion_2x6.txt")) if l.strip() and not l.startswith("#")]
    i = 0
    while i < len(lines):
        tok = lines[i].split()
        if tok[0] == "matrix":
            nr, nc = int(tok[1]), int(tok[2])
            g["A"] = np.array([[float(x) for x in lines[i + 1 + r].split()] for r in range(nr)])
            i += nr
        elif tok[0] in ("I", "J", "bounds"):
            g[tok[0]] = [int(x) for x in tok[1:]]
        elif tok[0] == "rank":
            g["rank"] = int(tok[1])
        elif tok[0] == "X":
            g["X"] = [float(x) for x in tok[1:]]
        elif tok[0] == "digits":
            g["digits"].append([int(x) for x in tok[1:]])
        i += 1
    return g


def test_example_2x6_exact_cores():
    """Lemma 4.1 example: cores 1x1x1x2, 2x1x3x2, 2x2x2x1 and the two Kronecker terms."""
    g = _golden_2x6()
    rows, cols, vals = _coo(g["A"])
    R, X, digits = convert.convert(rows, cols, vals, 2, 6, g["I"], g["J"])
    assert R == g["rank"]
    np.testing.assert_array_equal(X, g["X"])
    np.testing.assert_array_equal(digits, g["digits"])
    cores = convert.block_cores(R, X, digits, g["I"], g["J"])
    assert [c.shape for c in cores] == [(1, 1, 1, 2), (2, 1, 3, 2), (2, 2, 2, 1)]
    np.testing.assert_array_equal(mpo.dense(cores), g["A"])
    # The Kronecker form written out in the example.
    E11 = np.array([[1.0, 0], [0, 0]])
    E22 = np.array([[0.0, 0], [0, 1]])
    row = np.array([[1.0, 0, 0]])
    np.testing.assert_array_equal(np.kron(np.kron(E11, row), [[2.0]]) + np.kron(np.kron(E22, row), [[-5.0]]), g["A"])
    assert mpo.rank_bounds(g["I"], g["J"]) == g["bounds"]  # R2 <= 1, R3 <= 3 although Alg. 4.1 gives 2, 2


def test_block_example_sumofkron():
    """Section 4.1: the 4x4-block pattern with A14, A22, A33 gives 3 rank-1 terms E_ij (x) A_ij."""
    rng = np.random.default_rng(0)
    I1 = J1 = 3
    blocks = {(0, 3): rng.standard_normal((I1, J1)), (1, 1): rng.standard_normal((I1, J1)),
              (2, 2): rng.standard_normal((I1, J1))}
    D = np.zeros((4 * I1, 4 * J1))
    ref = np.zeros_like(D)
    for (p, q), B in blocks.items():
        D[p * I1:(p + 1) * I1, q * J1:(q + 1) * J1] = B
        E = np.zeros((4, 4))
        E[p, q] = 1
        ref += np.kron(E, B)
    np.testing.assert_array_equal(D, ref)
    R, X, digits = convert.convert(*_coo(D), D.shape[0], D.shape[1], [I1, 4], [J1, 4])
    assert R == 3  # Lemma 4.2: rank = number of nonzero blocks
    np.testing.assert_array_equal(digits, [[0, 3], [1, 1], [2, 2]])
    for t, (p, q) in enumerate([(0, 3), (1, 1), (2, 2)]):
        np.testing.assert_array_equal(X[t * 9:(t + 1) * 9].reshape(3, 3, order="F"), blocks[(p, q)])
    np.testing.assert_array_equal(mpo.dense(convert.block_cores(R, X, digits, [I1, 4], [J1, 4])), D)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_random_sparse_exact_and_lemmas(seed):
    """Bit-exact reconstruction; Lemma 4.2 (rank = #blocks) and Lemma 4.3 (R >= nnz / (I1 J1))."""
    rng = np.random.default_rng(seed)
    I, J = [4, 2, 3, 2], [2, 4, 2, 3]
    nr, nc = int(np.prod(I)), int(np.prod(J))
    D = np.where(rng.random((nr, nc)) < 0.05, rng.standard_normal((nr, nc)), 0.0)
    rows, cols, vals = _coo(D)
    R, X, digits = convert.convert(rows, cols, vals, nr, nc, I, J)
    blk = {(r // I[0], c // J[0]) for r, c in zip(rows, cols)}
    assert R == len(blk)
    assert R >= int(np.ceil(len(vals) / (I[0] * J[0])))
    np.testing.assert_array_equal(mpo.dense(convert.block_cores(R, X, digits, I, J)), D)
    np.testing.assert_array_equal(convert.dense_from_blocks(R, X, digits, I, J), D)
    # Rank of the converted MPO is uniform (Lemma 4.2)
    cores = convert.block_cores(R, X, digits, I, J)
    assert [c.shape[3] for c in cores[:-1]] == [R] * (len(I) - 1)


def test_banded_generator_and_conversion_small():
    rows, cols, vals = banded_coo(0, 256, 8, 16)
    assert np.all(np.abs(rows - cols) <= 16)
    assert np.all(np.diff(rows * 256 + cols) > 0)  # sorted, distinct
    D = np.zeros((256, 256))
    D[rows, cols] = vals
    I = J = [4, 4, 4, 4]
    R, X, digits = convert.convert(rows, cols, vals, 256, 256, I, J)
    np.testing.assert_array_equal(convert.dense_from_blocks(R, X, digits, I, J), D)


def test_kron_of_three_2x2_rounds_to_rank_1():
    """Section 4.2 example: A(3) (x) A(2) (x) A(1) converts to uniform rank 16; rounding gives 1."""
    rng = np.random.default_rng(11)
    mats = [rng.standard_normal((2, 2)) for _ in range(3)]
    D = mpo.kron_chain(mats)
    R, X, digits = convert.convert(*_coo(D), 8, 8, [2, 2, 2], [2, 2, 2])
    assert R == 16
    cores = convert.block_cores(R, X, digits, [2, 2, 2], [2, 2, 2])
    rounded = rounding.round_mpo(cores, tol=1e-12)
    assert rounding.ranks(rounded) == [1, 1, 1, 1]
    np.testing.assert_allclose(mpo.dense(rounded), D, rtol=0, atol=1e-12 * np.abs(D).max())


def test_rejections():
    with pytest.raises(convert.ConversionError):
        convert.convert([0, 0], [1, 1], [1.0, 2.0], 4, 4, [2, 2], [2, 2])  # duplicate
    with pytest.raises(convert.ConversionError):
        convert.convert([0], [1], [1.0], 4, 4, [2, 3], [2, 2])  # prod(I) != nrows
    with pytest.raises(convert.ConversionError):
        convert.convert([5], [1], [1.0], 4, 4, [2, 2], [2, 2])  # out of range


def test_empty_matrix():
    R, X, digits = convert.convert([], [], [], 4, 4, [2, 2], [2, 2])
    assert R == 0 and X.size == 0 and digits.shape == (0, 2)
