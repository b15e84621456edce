"""Pins for the TNrSVD oracle (Algs. 5.1, 5.4): exact-recovery cases, dense cross-check, invariants."""

import numpy as np
import pytest

from oracle import mpo, rng, tnrsvd
from workloads import gaussian_mpo, prescribed_mpo


def test_exact_recovery_known_rank():
    """rank(A) = K: range(Q) = range(A) exactly, so the K singular values are recovered (Halko's
    exact case); here with q = 1 and a 2-site-or-more MPO after the merge."""
    K = 8
    sigma = 0.7 ** np.arange(K)
    A, U, V = prescribed_mpo(0, 1, 16, [2, 2, 2], K, 3, sigma)
    np.testing.assert_allclose(np.linalg.svd(mpo.dense(A), compute_uv=False)[:K], sigma, rtol=1e-12)
    Uo, S, Vo = tnrsvd.tnrsvd(A, 4, 4, 1, seed=2, tol=1e-13)
    np.testing.assert_allclose(S, sigma[:4], rtol=1e-12)
    assert tnrsvd.sv_error(S, sigma[:4]) < 1e-12


def test_single_site_after_merge_is_dense_rsvd():
    """K = number of rows: the merge leaves one site, Q spans everything and S is the full SVD."""
    A = gaussian_mpo(1, [4, 4], [4, 4], [1, 3, 1])
    U, S, V = tnrsvd.tnrsvd(A, 8, 8, 0, seed=0)
    np.testing.assert_allclose(S, np.linalg.svd(mpo.dense(A), compute_uv=False)[:8], rtol=1e-12)


@pytest.mark.parametrize("q", [0, 1, 2])
def test_dense_rsvd_cross_check(q):
    """Without truncation the MPO subspace iteration spans exactly the dense iteration's range, so
    its singular values agree with a dense rSVD run on the same Omega (Alg. 5.1 + 5.4)."""
    d = 4
    A = gaussian_mpo(0, [4] * d, [4] * d, [1, 3, 3, 3, 1], scale=1 / np.sqrt(12))
    k, p = 5, 5
    U, S, V, info = tnrsvd.tnrsvd(A, k, p, q, seed=3, tol=0.0, return_info=True)
    Am = mpo.merge_leading(A, info["merge"])
    O = mpo.dense(rng.omega(3, mpo.dims(Am)[1], k + p))
    Ud, Sd, Vd = tnrsvd.dense_rsvd(mpo.dense(A), O, q)
    np.testing.assert_allclose(S, Sd[:k], rtol=1e-11)
    # singular vectors agree up to sign
    DU, DV = mpo.dense(U), mpo.dense(V)
    for i in range(k):
        assert abs(abs(DU[:, i] @ Ud[:, i]) - 1) < 1e-9
        assert abs(abs(DV[:, i] @ Vd[:, i]) - 1) < 1e-9


def test_invariants_orthogonality_interlacing_sandwich():
    d = 5
    A = gaussian_mpo(4, [4] * d, [4] * d, [1, 3, 3, 3, 3, 1], scale=1 / np.sqrt(12))
    k, p = 6, 6
    U, S, V = tnrsvd.tnrsvd(A, k, p, 1, seed=0, tol=1e-14)
    np.testing.assert_allclose(mpo.inner(U, U), np.eye(k), atol=1e-12)
    np.testing.assert_allclose(mpo.inner(V, V), np.eye(k), atol=1e-12)
    Am = mpo.merge_leading(A, mpo.merge_count([4] * d, [4] * d, k + p))  # U, V use the merged sites
    np.testing.assert_allclose(mpo.sandwich(U, Am, V), np.diag(S), atol=1e-11 * S[0])
    true = np.linalg.svd(mpo.dense(A), compute_uv=False)
    assert np.all(S <= true[:k] * (1 + 1e-12))  # sigma_i(Q^T A) <= sigma_i(A)
    assert np.all(np.diff(S) <= 0)
