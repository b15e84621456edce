"""Pins of the block-form sparse TNrSVD oracle: the block operator equals the dense matrix of the
COO input, and the rSVD on it equals the MPO TNrSVD of the converted cores (untruncated) and the
dense rSVD with the same Omega."""

import numpy as np

import workloads as W
from oracle import convert as oc
from oracle import mpo as om
from oracle import rng
from oracle import sparse as osp
from oracle import tnrsvd as ot


def _case(seed, n_sites, per_row, half_band):
    n = 4 ** n_sites
    r, c, v = W.banded_coo(seed, n, per_row, half_band)
    I = J = [4] * n_sites
    R, X, digits = oc.convert(r, c, v, n, n, I, J)
    D = np.zeros((n, n))
    D[r, c] = v
    return n, I, J, R, X, digits, D


def test_block_operator_equals_dense():
    n, I, J, R, X, digits, D = _case(1, 4, 5, 20)
    Qd = np.random.default_rng(0).standard_normal((n, 7))
    np.testing.assert_allclose(osp.apply(R, X, digits, I, J, Qd), D @ Qd, rtol=0, atol=1e-12)
    np.testing.assert_allclose(osp.apply(R, X, digits, I, J, Qd, trans=True), D.T @ Qd, rtol=0, atol=1e-12)


def test_omega_dense_is_the_kronecker_product():
    J = [8, 2, 3]
    O = osp.omega_dense(5, J, 6)
    cores = rng.omega(5, J, 6)
    want = np.kron(np.kron(cores[2][0, :, 0, 0][:, None], cores[1][0, :, 0, 0][:, None]), cores[0][0, :, :, 0])
    np.testing.assert_allclose(O, want, rtol=0, atol=1e-15)


def test_equals_untruncated_mpo_tnrsvd_and_dense_rsvd():
    n, I, J, R, X, digits, D = _case(2, 3, 3, 6)  # 64 x 64
    k, p, q, seed = 3, 3, 1, 9
    U, S, V = osp.sparse_tnrsvd(R, X, digits, I, J, k, p, q, seed)
    cores = oc.block_cores(R, X, digits, I, J)
    _, S_mpo, _ = ot.tnrsvd(cores, k, p, q, seed, tol=0.0, max_rank=0)
    np.testing.assert_allclose(S, S_mpo, rtol=1e-11)
    m = om.merge_count(I, J, k + p)
    O = osp.omega_dense(seed, [int(np.prod(J[:m]))] + J[m:], k + p)
    Ud, Sd, Vd = ot.dense_rsvd(D, O, q)
    np.testing.assert_allclose(S, Sd[:k], rtol=1e-11)
    # U^T A V = diag(S)
    np.testing.assert_allclose(U.T @ D @ V, np.diag(S), atol=1e-11 * S[0])


def test_coo_form_equals_block_form():
    n, I, J, R, X, digits, D = _case(3, 4, 4, 12)
    r, c = np.nonzero(D)
    U1, S1, V1 = osp.sparse_tnrsvd(R, X, digits, I, J, 4, 4, 1, 3)
    U2, S2, V2 = osp.coo_tnrsvd(r, c, D[r, c], n, n, I, J, 4, 4, 1, 3)
    np.testing.assert_allclose(S1, S2, rtol=1e-12)
