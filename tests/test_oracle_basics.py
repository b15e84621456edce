"""Pins for the oracle's index conventions and MPO basics (Sections 2, 3, 5.2)."""

import itertools

import numpy as np
import pytest

from oracle import mpo
from tests.conftest import golden_path
from workloads import gaussian_mpo


def _read_rows(name):
    rows = []
    for line in open(golden_path(name)):
        line = line.strip()
        if line and not line.startswith("#"):
            rows.append([int(x) for x in line.split()])
    return np.array(rows)


def test_reshape_example_2_1():
    """Example 2.1/2.2: column-major reshape of the 4x3x2 tensor holding 1..24."""
    T = np.arange(1, 25, dtype=np.float64).reshape((4, 3, 2), order="F")
    M = T.reshape((4, 6), order="F")
    np.testing.assert_array_equal(M, _read_rows("reshape_example.txt"))
    np.testing.assert_array_equal(T.reshape(-1, order="F"), np.arange(1, 25))
    # Eq. (2.1): [i1 i2 i3] = i1 + I1 (i2 - 1) + I1 I2 (i3 - 1) (1-based)
    for i1, i2, i3 in itertools.product(range(4), range(3), range(2)):
        assert T[i1, i2, i3] == 1 + i1 + 4 * i2 + 12 * i3


def test_dense_bruteforce_entries():
    """A([i..],[j..]) = A1(:,i1,j1,:) A2(:,i2,j2,:) ... as a product of small matrices (Section 3)."""
    I, J, R = [2, 3, 2], [3, 2, 2], [1, 2, 3, 1]
    A = gaussian_mpo(5, I, J, R)
    D = mpo.dense(A)
    assert D.shape == (12, 12)
    for idx in itertools.product(*[range(n) for n in I]):
        for jdx in itertools.product(*[range(n) for n in J]):
            row = idx[0] + I[0] * (idx[1] + I[1] * idx[2])
            col = jdx[0] + J[0] * (jdx[1] + J[1] * jdx[2])
            val = np.eye(1)
            for k in range(3):
                val = val @ A[k][:, idx[k], jdx[k], :]
            assert abs(D[row, col] - val[0, 0]) <= 1e-14 * (1 + abs(val[0, 0]))


def test_theorem_3_1_kron_order():
    """Thm 3.1: a rank-1 MPO equals A^(d) (x) ... (x) A^(1), the first core being the LAST factor."""
    rng = np.random.default_rng(3)
    I, J = [2, 3, 4], [3, 2, 2]
    mats = [rng.standard_normal((i, j)) for i, j in zip(I, J)]
    cores = [m[None, :, :, None] for m in mats]
    np.testing.assert_allclose(mpo.dense(cores), mpo.kron_chain(mats), rtol=0, atol=1e-14)
    # Reversing the order gives a different matrix (the statement is not symmetric).
    assert not np.allclose(mpo.dense(cores), mpo.kron_chain(mats[::-1]))


def test_theorem_3_2_bounds_worked_example():
    """Thm 3.2 bounds for the factor-ordering example of Section 4.3."""
    for row in _read_rows("rank_bounds.txt"):
        I1, J1, I2, J2, I3, J3, b2, b3 = row
        assert mpo.rank_bounds([I1, I2, I3], [J1, J2, J3]) == [b2, b3]


def test_merge_count_section_6_3():
    """Section 6.3: K = 32 with 2x2 sites merges 5 cores; K = 100 merges 7 (128 >= 100)."""
    assert mpo.merge_count([2] * 20, [2] * 20, 32) == 5
    assert mpo.merge_count([2] * 20, [2] * 20, 100) == 7
    assert mpo.merge_count([4] * 6, [4] * 6, 20) == 3
    assert mpo.merge_count([4] * 2, [4] * 2, 17) is None


def test_merge_preserves_matrix():
    I, J, R = [2, 2, 3, 2], [2, 3, 2, 2], [1, 3, 4, 2, 1]
    A = gaussian_mpo(1, I, J, R)
    for m in (1, 2, 3, 4):
        Am = mpo.merge_leading(A, m)
        assert len(Am) == 4 - m + 1
        assert Am[0].shape[1] == int(np.prod(I[:m])) and Am[0].shape[2] == int(np.prod(J[:m]))
        np.testing.assert_allclose(mpo.dense(Am), mpo.dense(A), rtol=0, atol=1e-13)


@pytest.mark.parametrize("trans", [False, True])
def test_contract_equals_dense_product(trans):
    """Section 5.2: the per-site contraction represents the matrix product."""
    I, J, R = [3, 2, 2], [2, 4, 2], [1, 2, 3, 1]
    A = gaussian_mpo(2, I, J, R)
    rows = J if not trans else I
    K = 3
    X = gaussian_mpo(4, rows, [K, 1, 1], [1, 2, 2, 1])
    Y = mpo.contract(A, X, trans=trans)
    DA, DX = mpo.dense(A), mpo.dense(X)
    ref = (DA.T if trans else DA) @ DX
    np.testing.assert_allclose(mpo.dense(Y), ref, rtol=0, atol=1e-13)
    assert [c.shape[0] for c in Y] == [1, 4, 6]  # ranks multiply


def test_inner_sandwich_norm():
    I, J = [3, 2, 2], [2, 2, 3]
    A = gaussian_mpo(6, I, J, [1, 2, 2, 1])
    U = gaussian_mpo(7, I, [2, 1, 1], [1, 3, 2, 1])
    U2 = gaussian_mpo(8, I, [3, 1, 1], [1, 2, 2, 1])
    V = gaussian_mpo(9, J, [2, 1, 1], [1, 2, 3, 1])
    np.testing.assert_allclose(mpo.inner(U, U2), mpo.dense(U).T @ mpo.dense(U2), atol=1e-13)
    np.testing.assert_allclose(mpo.sandwich(U, A, V), mpo.dense(U).T @ mpo.dense(A) @ mpo.dense(V), atol=1e-13)
    assert abs(mpo.norm(A) - np.linalg.norm(mpo.dense(A))) < 1e-13
    np.testing.assert_allclose(mpo.dense(mpo.transpose(A)), mpo.dense(A).T, atol=0)
