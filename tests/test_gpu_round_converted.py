"""Rounding of the MPO that Alg. 4.1 produces, on the GPU: the block form expanded into dense cores
(tnr_sparse_cores, bit-exact against the oracle's expansion), then SVD-based rounding through
tnr_orthogonalize on the one-column view (binding: round_operator), against the oracle's
rounding (oracle.rounding.round_mpo) and the dense matrix. Section 4.2's example: a Kronecker
product of three 2 x 2 matrices converts to rank 16 and rounds to rank 1."""

import numpy as np
import pytest
import torch

from oracle import convert as oc
from oracle import mpo as om
from oracle import rounding as orr
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import coo_to_device, host_cores

pytestmark = pytest.mark.gpu


def _coo(D):
    r, c = np.nonzero(D)
    return r.astype(np.int64), c.astype(np.int64), D[r, c]


def _convert_and_expand(D, I, J):
    rows, cols, vals = _coo(D)
    r, c, v = coo_to_device(rows, cols, vals)
    R, X, digits = T.sparse_to_mpo(D.shape[0], D.shape[1], r, c, v, I, J)
    A = T.tnr_sparse_cores(R, X, digits, I, J)
    torch.cuda.synchronize()
    Ro, Xo, Do = oc.convert(rows, cols, vals, D.shape[0], D.shape[1], I, J)
    assert R == Ro
    ref = oc.block_cores(Ro, Xo, Do, I, J)
    got = host_cores(A)
    for g, o in zip(got, ref):  # copy and integer work: bit for bit
        assert g.shape == o.shape and g.tobytes() == np.ascontiguousarray(o).tobytes()
    return A, ref


def test_kronecker_example_converts_to_rank_16_and_rounds_to_rank_1():
    rng = np.random.default_rng(11)
    mats = [rng.standard_normal((2, 2)) for _ in range(3)]
    D = om.kron_chain(mats)
    A, ref = _convert_and_expand(D, [2, 2, 2], [2, 2, 2])
    assert A.R == [1, 16, 16, 1]
    B = T.round_operator(A, tol=1e-12)
    assert B.R == [1, 1, 1, 1]
    np.testing.assert_allclose(om.dense(host_cores(B)), D, rtol=0, atol=1e-12 * np.abs(D).max())


@pytest.mark.parametrize("tol,want_rank", [(1e-2, 1), (1e-6, None)])
def test_rounding_matches_oracle_on_a_perturbed_kronecker(tol, want_rank):
    """kron(A3, A2, A1) plus a 1e-3 perturbation of a few entries: tol 1e-2 cuts the perturbation
    (rank 1 everywhere), tol 1e-6 keeps it; ranks and the rounded matrix equal the oracle's."""
    rng = np.random.default_rng(5)
    mats = [rng.standard_normal((3, 2)), rng.standard_normal((2, 4)), rng.standard_normal((4, 2))]
    D = om.kron_chain(mats)
    for _ in range(5):
        D[rng.integers(D.shape[0]), rng.integers(D.shape[1])] += 1e-3
    I, J = [3, 2, 4], [2, 4, 2]
    A, ref = _convert_and_expand(D, I, J)
    B = T.round_operator(A, tol=tol)
    Bo = orr.round_mpo(ref, tol=tol)
    assert B.R == orr.ranks(Bo)
    if want_rank is not None:
        assert B.R[1:-1] == [want_rank] * (len(I) - 1)
    np.testing.assert_allclose(om.dense(host_cores(B)), om.dense(Bo), rtol=0, atol=1e-10 * np.abs(D).max())
    assert np.linalg.norm(om.dense(host_cores(B)) - D) <= tol * np.linalg.norm(D) * (1 + 1e-9)


def test_banded_matrix_rounds_to_its_exact_ranks():
    """A random banded 256 x 256 matrix (four 4 x 4 sites): the converted MPO's bonds carry one rank
    per block; exact rounding (tol 1e-13) leaves the ranks of the matrix's unfoldings."""
    n = 256
    from workloads import banded_coo

    rows, cols, vals = banded_coo(7, n, 3, 2)
    D = np.zeros((n, n))
    D[rows, cols] = vals
    I = J = [4, 4, 4, 4]
    A, ref = _convert_and_expand(D, I, J)
    B = T.round_operator(A, tol=1e-13)
    Bo = orr.round_mpo(ref, tol=1e-13)
    assert B.R == orr.ranks(Bo)
    np.testing.assert_allclose(om.dense(host_cores(B)), D, rtol=0, atol=1e-11 * np.abs(D).max())
