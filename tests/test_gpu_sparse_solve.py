"""TNrSVD of a sparse matrix through its Alg. 4.1 block form (tnr_sparse_solve): parity with the
oracle's block-form rSVD (small, FP64: values and vectors) and, at the 2^20 banded size, with the
oracle's rSVD on the COO input (singular values, FP64 and mixed)."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import sparse as osp
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import coo_to_device, sv_rel_err

pytestmark = pytest.mark.gpu


def _convert(r, c, v, n, I, J):
    rd, cd, vd = coo_to_device(r, c, v)
    R, X, digits = T.sparse_to_mpo(n, n, rd, cd, vd, I, J)
    return R, X, digits


def _colwise_sign_free(A, B, tol):
    for j in range(A.shape[1]):
        a, b = A[:, j], B[:, j]
        s = np.sign(a @ b) if a @ b != 0 else 1.0
        assert np.linalg.norm(a - s * b) <= tol * max(np.linalg.norm(b), 1.0), j


@pytest.mark.parametrize("n_sites,q", [(5, 1), (4, 0), (6, 2)])
def test_small_matches_block_oracle(n_sites, q):
    n = 4 ** n_sites
    r, c, v = W.banded_coo(n_sites, n, 5, 20)
    I = J = [4] * n_sites
    R, X, digits = _convert(r, c, v, n, I, J)
    k, p, seed = 4, 4, 17
    U, S, V = T.tnr_sparse_solve(n, n, R, X, digits, I, J, k, p, q, seed, precision=T.TNR_FP64)
    torch.cuda.synchronize()
    from oracle import convert as oc
    Ro, Xo, Do = oc.convert(r, c, v, n, n, I, J)
    Uo, So, Vo = osp.sparse_tnrsvd(Ro, Xo, Do, I, J, k, p, q, seed)
    assert sv_rel_err(S.cpu().numpy(), So) <= 1e-10
    _colwise_sign_free(U.cpu().numpy(), Uo, 1e-8)
    _colwise_sign_free(V.cpu().numpy(), Vo, 1e-8)


@pytest.mark.parametrize("precision", [T.TNR_FP64, T.TNR_MIXED])
def test_banded_2_20_matches_coo_oracle(precision):
    n = 1 << 20
    r, c, v = W.banded_coo(0, n, 8, 64)
    I = J = [4] * 10
    R, X, digits = _convert(r, c, v, n, I, J)
    k, p, q, seed = 20, 10, 1, 5
    U, S, V = T.tnr_sparse_solve(n, n, R, X, digits, I, J, k, p, q, seed, precision=precision)
    torch.cuda.synchronize()
    _, So, _ = osp.coo_tnrsvd(r, c, v, n, n, I, J, k, p, q, seed)
    err = sv_rel_err(S.cpu().numpy(), So)
    assert err <= (1e-10 if precision == T.TNR_FP64 else 1e-6), err
