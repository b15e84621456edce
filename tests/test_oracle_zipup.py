"""Pins for the truncate-as-you-go (zip-up) rounding of a product in the oracle.

The product op(A) X (Section 5.2) is rounded while it is formed, right to left (oracle.rounding.
zipup_product), then orthogonalised with the rounding of Section 5.4 (Alg. 5.2). Pinned here:
  * without truncation it is the exact product (dense comparison), for A X and A^T X;
  * on a left-canonical X with prescribed Schmidt spectra and op(A) = identity, the local matrix at
    every bond holds the exact Schmidt values, so the kept ranks follow the rule in closed form and
    the result is the construction with each spectrum cut;
  * whole TNrSVD runs agree with the two-sweep oracle wherever no truncation bites.
"""

import numpy as np
import pytest

from oracle import mpo, rounding
from oracle import tnrsvd as ot
from workloads import gaussian_mpo, prescribed_bond_mpo


def _identity_op(n):
    return [np.eye(int(x))[None, :, :, None].copy() for x in n]


@pytest.mark.parametrize("trans", [False, True])
def test_zipup_without_truncation_is_the_product(trans):
    I, J, K = [4, 3, 2, 2], [3, 2, 2, 3], 3
    A = gaussian_mpo(21, I, J, [1, 3, 2, 3, 1], scale=0.5)
    rows = I if trans else J
    X = gaussian_mpo(22, rows, [K, 1, 1, 1], [1, 2, 3, 2, 1])
    Y = rounding.zipup_product(A, X, trans, tol=0.0, max_rank=0)
    DA = mpo.dense(A)
    want = (DA.T if trans else DA) @ mpo.dense(X)
    np.testing.assert_allclose(mpo.dense(Y), want, atol=1e-12 * np.abs(want).max())
    # cores 2..d right-orthonormal (the zip-up leaves Y right-canonical)
    for c in Y[1:]:
        t = c.shape[0]
        M = c.reshape(t, -1, order="F")
        np.testing.assert_allclose(M @ M.T, np.eye(t), atol=1e-13)


_SPECTRA = [0.6 ** np.arange(6), 0.55 ** np.arange(7), 0.6 ** np.arange(5) * np.array([1, 1, 1, 1, 0.3])]
_N = [6, 42, 35, 5]
_G = 3.7


def _zip_ranks(spectra, tol, max_rank=0):
    d = len(spectra) + 1
    out = []
    for s in spectra:
        r = len(s)
        for cand in range(1, len(s) + 1):
            if np.sum(s[cand:] ** 2) <= tol ** 2 / (d - 1):
                r = cand
                break
        out.append(min(r, max_rank) if max_rank else r)
    return out


def _cut(cores, spectra, ranks):
    """The left-canonical construction with s_k cut to its first r_k values (s_k sits on core k+1's
    left bond)."""
    out = [c.copy() for c in cores]
    for k, r in enumerate(ranks):
        w = np.zeros(len(spectra[k]))
        w[:r] = 1.0
        out[k + 1] = out[k + 1] * w[:, None, None, None]
    return out


@pytest.mark.parametrize("tol,max_rank", [(0.02, 0), (0.05, 0), (0.1, 0), (0.2, 0), (0.02, 4)])
def test_zipup_exact_ranks_on_left_canonical_input(tol, max_rank):
    X, s = prescribed_bond_mpo(5, _N, _SPECTRA, _G, site1_split=(2, 3), canonical="left")
    ident = _identity_op([2] + _N[1:])
    Y = rounding.zipup_product(ident, X, False, tol=tol, max_rank=max_rank)
    want = _zip_ranks(s, tol, max_rank)
    assert rounding.ranks(Y)[1:-1] == want
    np.testing.assert_allclose(mpo.dense(Y), mpo.dense(_cut(X, s, want)), atol=1e-13 * _G)
    # then MPO-QR of the rounded product: ranks can only shrink, Q R stays within the bound
    Q, R = rounding.orthogonalize_zipup(ident, X, False, tol=tol, max_rank=max_rank)
    assert all(a <= b for a, b in zip(rounding.ranks(Q), rounding.ranks(Y)))
    np.testing.assert_allclose(mpo.inner(Q, Q), np.eye(3), atol=1e-13)
    DX = mpo.dense(X)
    if not max_rank:  # sum over bonds of the discarded parts: at most tol ||X|| each sweep
        assert np.linalg.norm(DX - mpo.dense(Q) @ R) <= 2 * tol * np.linalg.norm(DX)


def test_left_canonical_generator():
    """Cores 1..d-1 of the left-canonical construction have orthonormal columns; same Schmidt values."""
    X, s = prescribed_bond_mpo(5, _N, _SPECTRA, _G, canonical="left")
    for c in X[:-1]:
        M = c.reshape(-1, c.shape[3], order="F")
        np.testing.assert_allclose(M.T @ M, np.eye(c.shape[3]), atol=1e-13)
    T = mpo.dense(X)[:, 0].reshape(_N, order="F")
    for k in range(1, len(_N)):
        sv = np.linalg.svd(T.reshape(int(np.prod(_N[:k])), -1, order="F"), compute_uv=False)
        np.testing.assert_allclose(sv[: len(s[k - 1])], _G * s[k - 1], rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_zipup_tnrsvd_equals_two_sweep_without_truncation(seed):
    """No truncation (tol = 0): both roundings compute the same subspaces, so S, and U, V up to
    signs, agree."""
    rng = np.random.default_rng(seed)
    d = 5
    x = int(rng.choice([2, 3]))
    A = gaussian_mpo(100 + seed, [x] * d, [x] * d, [1, 2, 3, 3, 2, 1], scale=0.6)
    k, p = 2, 2
    U1, S1, V1 = ot.tnrsvd(A, k, p, 1, seed, tol=0.0, max_rank=0)
    U2, S2, V2 = ot.tnrsvd(A, k, p, 1, seed, tol=0.0, max_rank=0, rounding_mode="zipup")
    np.testing.assert_allclose(S2, S1, rtol=1e-12)
    np.testing.assert_allclose(np.abs(np.diag(mpo.inner(U1, U2))), 1.0, atol=1e-10)
    np.testing.assert_allclose(np.abs(np.diag(mpo.inner(V1, V2))), 1.0, atol=1e-10)


def test_zipup_tnrsvd_exact_recovery_with_rank_cap():
    """A = U diag(sigma) V^T of exact rank K (orthogonal MPOs U, V): the sketch captures range(A)
    exactly, so with K = k + p and the rank cap at K the zip-up TNrSVD returns sigma (Halko's
    exact case), as the two-sweep oracle does."""
    from workloads import prescribed_mpo

    K = 8
    sigma = 0.8 ** np.arange(K)
    A, _, _ = prescribed_mpo(3, 4, 16, [2, 2, 2, 2], K, 3, sigma)
    for mode in ("zipup", "two_sweep"):
        _, S, _ = ot.tnrsvd(A, 4, 4, 1, 9, tol=1e-13, max_rank=K, rounding_mode=mode)
        np.testing.assert_allclose(S, sigma[:4], rtol=1e-11)
