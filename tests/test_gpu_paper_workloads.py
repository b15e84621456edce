"""The paper's Section 6.3 workloads on the GPU (single solve, tnr_solve):

* 50 prescribed singular values 0.5^k with random orthogonal U, V (maximal MPO rank 25), N sites of
  2 x 2, rank-50 approximation (K = 100, q = 1), the first 7 sites merged, the paper's rounding
  tolerance for each N: the singular values match the oracle (FP64: 1e-10) and the prescribed ones
  to the paper's target ||S - S^||_F / ||S||_F <= 1e-6 (also in mixed precision);
* the Hilbert submatrix H(:, 1:2^(N-1)) as an MPO (TT-SVD input builder, relative error 1e-11),
  rank-16 approximation (K = 32, q = 2, tolerance 1e-9, 5 sites merged): the oracle's singular
  values (1e-10) and the dense matrix's leading 16 (1e-8).
"""

import numpy as np
import pytest

import workloads as W
from oracle import tnrsvd as ot
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import dev_mpo, sv_rel_err

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("N", [10, 20, 35])
def test_prescribed_sigma_sweep_points(N):
    c = W.paper_prescribed(N)
    A = dev_mpo(c["A"])
    _, S, _ = T.tnr_solve(A, c["k"], c["p"], c["q"], c["seed"], tol=c["tol"], max_rank=c["max_rank"],
                          precision=T.TNR_FP64)
    S = S.cpu().numpy()
    assert sv_rel_err(S, c["sigma"]) <= 1e-6
    if N <= 20:  # the oracle at 2^20 x 2^20 with K = 100 takes a few seconds
        _, So, _ = ot.tnrsvd(c["A"], c["k"], c["p"], c["q"], c["seed"], tol=c["tol"], max_rank=c["max_rank"])
        assert sv_rel_err(S, So) <= 1e-10
    _, Sm, _ = T.tnr_solve(A, c["k"], c["p"], c["q"], c["seed"], tol=c["tol"], max_rank=c["max_rank"],
                           precision=T.TNR_MIXED)
    assert sv_rel_err(Sm.cpu().numpy(), c["sigma"]) <= 1e-6


@pytest.mark.parametrize("N", [10, 12])
def test_hilbert_submatrix(N):
    c = W.paper_hilbert(N)
    _, S, _ = T.tnr_solve(dev_mpo(c["A"]), c["k"], c["p"], c["q"], c["seed"], tol=c["tol"], max_rank=c["max_rank"],
                          precision=T.TNR_FP64)
    S = S.cpu().numpy()
    _, So, _ = ot.tnrsvd(c["A"], c["k"], c["p"], c["q"], c["seed"], tol=c["tol"], max_rank=c["max_rank"])
    assert sv_rel_err(S, So) <= 1e-10
    s_true = np.linalg.svd(c["dense"], compute_uv=False)[: c["k"]]
    assert sv_rel_err(S, s_true) <= 1e-8
