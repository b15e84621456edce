"""The input builders of the paper's Section 6.3 workloads (CPU): the Hilbert entries, the TT-SVD
MPO builder (exact ranks and reconstruction within its tolerance), and the prescribed-sigma matrix
(its singular values are exactly 0.5^k, checked against a dense LAPACK SVD at N = 10)."""

import numpy as np

import workloads as W
from oracle import mpo


def test_hilbert_entries():
    H = W.hilbert_submatrix(4)
    assert H.shape == (16, 8)
    assert H[0, 0] == 1.0 and H[2, 3] == 1.0 / 6.0 and H[15, 7] == 1.0 / 23.0


def test_tt_svd_recovers_an_exact_mpo():
    I, J = [2, 3, 2, 2], [3, 2, 2, 1]
    A = W.gaussian_mpo(4, I, J, [1, 2, 3, 2, 1])
    D = mpo.dense(A)
    B = W.tt_svd_operator(D, I, J, 1e-14)
    assert [c.shape[3] for c in B][:-1] == [2, 3, 2]
    np.testing.assert_allclose(mpo.dense(B), D, atol=1e-12 * np.abs(D).max())


def test_tt_svd_error_within_tolerance_on_hilbert():
    D = W.hilbert_submatrix(8)
    I, J = [2] * 8, [2] * 7 + [1]
    for tol in (1e-4, 1e-8):
        B = W.tt_svd_operator(D, I, J, tol)
        assert np.linalg.norm(mpo.dense(B) - D) <= tol * np.linalg.norm(D) * (1 + 1e-9)


def test_prescribed_sigma_matrix_has_the_prescribed_values():
    c = W.paper_prescribed(10)
    D = mpo.dense(c["A"])
    assert D.shape == (1024, 1024)
    s = np.linalg.svd(D, compute_uv=False)
    np.testing.assert_allclose(s[:50], c["sigma"], rtol=1e-10, atol=1e-14)
    assert np.all(s[50:] < 1e-13)
    assert max(x.shape[3] for x in c["A"]) == 25  # the paper's maximal MPO rank
