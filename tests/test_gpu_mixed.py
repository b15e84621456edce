"""GPU parity of the mixed-precision path (BF16 x3 split products, tcgen05 tensor cores for the
dense site-1 products, FP64 sweeps and SVDs) against the FP64 oracle."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import mpo as om
from oracle import tnrsvd as ot
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import dev_mpo, host_cores, sv_rel_err

pytestmark = pytest.mark.gpu

MIXED_SV_TOL = 1e-6  # relative singular-value error gate of the mixed-precision path


@pytest.mark.parametrize("trans", [0, 1])
@pytest.mark.parametrize("shape", [(64, 64, 25, 32, 5), (48, 40, 7, 20, 3), (16, 16, 1, 16, 1), (100, 80, 3, 40, 2)])
def test_contract_site1_tensor_cores(trans, shape):
    """Dense site-1 product on tcgen05 against the FP64 oracle product: elementwise within the
    BF16 x3 split error bound (16 mantissa bits per operand, FP32 accumulation)."""
    I1, J1, R2, K, S2 = shape
    A = W.gaussian_mpo(3, [I1, 4], [J1, 4], [1, R2, 1])
    rows = J1 if trans == 0 else I1
    X = W.gaussian_mpo(4, [rows, 4], [K, 1], [1, S2, 1])
    want = om.contract(A, X, trans=bool(trans))
    T.stats_reset()
    Y = T.tnr_mpo_contract(dev_mpo(A), trans, dev_mpo(X), precision=T.TNR_MIXED)
    torch.cuda.synchronize()
    tc_launches, _ = T.stats(T.stats_classes().index("contract_tc"))
    assert tc_launches >= 1  # the dense site ran on the tensor-core kernel
    got = host_cores(Y)
    ny = rows
    bound = 4.0 * 2.0 ** -16 * ny * np.abs(A[0]).max() * np.abs(X[0]).max() + 1e-300
    np.testing.assert_allclose(got[0], want[0], rtol=0, atol=bound)
    assert np.abs(got[0] - want[0]).max() > 0  # reduced precision really was used
    np.testing.assert_allclose(got[1], want[1], rtol=0, atol=4.0 * 2.0 ** -16 * 4 * np.abs(A[1]).max() * np.abs(X[1]).max())


def _mixed_solve(A, k, p, q, seed, tol, max_rank):
    U, S, V = T.tnr_solve(dev_mpo(A), k, p, q, seed, tol=tol, max_rank=max_rank, precision=T.TNR_MIXED)
    torch.cuda.synchronize()
    return U, S.cpu().numpy(), V


def test_mixed_c2_prescribed():
    """2^20 x 2^20 prescribed-sigma MPO (k=16, p=16, q=2) in mixed precision: singular values
    within 1e-6 of the FP64 oracle and of the exact sigma_j = 0.7^j."""
    c = W.c2_prescribed(tol=1e-8)
    _, So, _ = ot.tnrsvd(c["A"], c["k"], c["p"], c["q"], c["seed"], tol=1e-12, max_rank=c["max_rank"])
    U, S, V = _mixed_solve(c["A"], c["k"], c["p"], c["q"], c["seed"], c["tol"], c["max_rank"])
    assert sv_rel_err(S, So) <= MIXED_SV_TOL
    assert sv_rel_err(S, c["sigma"][:16]) <= MIXED_SV_TOL
    Uh, Vh = host_cores(U), host_cores(V)
    np.testing.assert_allclose(om.inner(Uh, Uh), np.eye(16), atol=1e-10)
    np.testing.assert_allclose(om.inner(Vh, Vh), np.eye(16), atol=1e-10)


def test_mixed_c1_gaussian():
    c = W.c1_plain_fp64()
    _, So, _ = ot.tnrsvd(c["A"], c["k"], c["p"], c["q"], c["seed"], tol=c["tol"], max_rank=c["max_rank"])
    _, S, _ = _mixed_solve(c["A"], c["k"], c["p"], c["q"], c["seed"], 1e-10, c["max_rank"])
    assert sv_rel_err(S, So) <= MIXED_SV_TOL
