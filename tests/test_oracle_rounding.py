"""Pins for MPO-QR (Alg. 5.2), MPO-SVD (Alg. 5.3) and rounding in the oracle."""

import numpy as np
import pytest

from oracle import mpo, rounding
from workloads import gaussian_mpo, orthogonal_mpo


def _mps_bounds(I, K):
    """Bond bounds of a (prod I) x K matrix with K on site 1 (Thm 3.2 with J = (K, 1, ...))."""
    return mpo.rank_bounds(I, [K] + [1] * (len(I) - 1))


def test_keep_rank_closed_form():
    s = np.array([1.0, 0.1, 0.01, 0.001])
    assert rounding.keep_rank(s, 0.0, 0) == 4
    assert rounding.keep_rank(s, 0.0011, 0) == 3  # tail {0.001}: 1e-6 <= 1.21e-6
    assert rounding.keep_rank(s, 0.0101, 0) == 2  # tail sqrt(1e-4 + 1e-6) = 0.01005
    assert rounding.keep_rank(s, 10.0, 0) == 1  # never below 1
    assert rounding.keep_rank(s, 0.0, 2) == 2  # max_rank cap


@pytest.mark.parametrize("seed", [0, 1])
def test_orthogonalize_no_truncation(seed):
    I, K = [6, 2, 3, 2], 5
    Y = gaussian_mpo(seed, I, [K, 1, 1, 1], [1, 4, 3, 2, 1])
    Q, R = rounding.orthogonalize(Y, tol=0.0)
    np.testing.assert_allclose(mpo.inner(Q, Q), np.eye(K), atol=1e-13)  # Alg. 5.2: Q^T Q = I_K
    DQ, DY = mpo.dense(Q), mpo.dense(Y)
    np.testing.assert_allclose(DQ.T @ DQ, np.eye(K), atol=1e-13)
    np.testing.assert_allclose(DQ @ R, DY, atol=1e-12 * np.abs(DY).max())
    assert np.allclose(R, np.triu(R))
    # Same range as a dense LAPACK thin QR: Q Q^T equals the projector of range(Y).
    Qd, _ = np.linalg.qr(DY)
    np.testing.assert_allclose(DQ @ DQ.T, Qd @ Qd.T, atol=1e-12)
    for r, b in zip(rounding.ranks(Q)[1:-1], _mps_bounds(I, K)):
        assert r <= b


def test_orthogonalize_truncates_redundant_bonds():
    """An MPO with padded (linearly dependent) bonds rounds back to its canonical ranks."""
    I, K = [8, 2, 2, 2], 4
    Y = gaussian_mpo(3, I, [K, 1, 1, 1], [1, 2, 2, 2, 1])
    # Pad each bond by duplicating its directions: Y_k -> [Y_k, Y_k] / sqrt-free sum splitting.
    Z = []
    for k, c in enumerate(Y):
        r, i, kk, r2 = c.shape
        left = 1 if k == 0 else 2 * r
        right = 1 if k == len(Y) - 1 else 2 * r2
        n = np.zeros((left, i, kk, right))
        if k == 0:
            n[:, :, :, :r2] = c * 0.5
            n[:, :, :, r2:] = c * 0.5
        elif k == len(Y) - 1:
            n[:r] = c
            n[r:] = c
        else:
            n[:r, :, :, :r2] = c
            n[r:, :, :, r2:] = c
        Z.append(n)
    np.testing.assert_allclose(mpo.dense(Z), mpo.dense(Y), atol=1e-13)
    Q, R = rounding.orthogonalize(Z, tol=1e-12)
    assert rounding.ranks(Q) == [1, 2, 2, 2, 1]
    np.testing.assert_allclose(mpo.dense(Q) @ R, mpo.dense(Y), atol=1e-12)


def test_mpo_svd_matches_lapack():
    I, K = [8, 2, 3], 6
    Z = gaussian_mpo(4, I, [K, 1, 1], [1, 3, 2, 1])
    W, S, V = rounding.mpo_svd(Z, tol=0.0)
    B = mpo.dense(Z).T  # K x J
    np.testing.assert_allclose(S, np.linalg.svd(B, compute_uv=False), rtol=1e-13)
    np.testing.assert_allclose(W.T @ W, np.eye(K), atol=1e-13)
    np.testing.assert_allclose(mpo.inner(V, V), np.eye(K), atol=1e-13)
    np.testing.assert_allclose(W @ np.diag(S) @ mpo.dense(V).T, B, atol=1e-12)
    assert np.all(np.diff(S) <= 0) and np.all(S >= 0)


def test_orthogonal_generator_is_orthogonal():
    U = orthogonal_mpo(0, 16, [2, 2, 2], 8, 3)
    np.testing.assert_allclose(mpo.inner(U, U), np.eye(8), atol=1e-13)


def test_round_mpo_preserves_and_bounds():
    I, J = [2, 3, 2, 2], [3, 2, 2, 2]
    A = gaussian_mpo(9, I, J, [1, 4, 9, 4, 1])
    B = rounding.round_mpo(A, tol=0.0)
    np.testing.assert_allclose(mpo.dense(B), mpo.dense(A), atol=1e-12)
    for r, b in zip(rounding.ranks(B)[1:-1], mpo.rank_bounds(I, J)):
        assert r <= b


# ---- the truncation threshold delta = tol ||Y||_F / sqrt(d - 1) of the rounding (Section 3/5.4) ----
#
# MPOs with prescribed Schmidt spectra at every bond (workloads.prescribed_bond_mpo): the Schmidt
# values at bond k are g s_k, and truncating bond k keeps the product structure, scaling the other
# bonds' values by c_k = ||s_k[:r_k]||. The right-to-left sweep therefore sees, at bond k,
# g s_k prod_{j>k} c_j, and keeps the smallest r >= 1 whose discarded values have squared sum
# <= delta^2. The rounded tensor is the construction with each s_k cut to its first r_k values.
from workloads import prescribed_bond_mpo  # noqa: E402

# Spectra graded finely enough (ratio 0.6) that a threshold off by sqrt(d-1), by a factor g or
# by squaring ||Y|| changes at least one kept rank.
_SPECTRA = [0.6 ** np.arange(6), 0.55 ** np.arange(7), 0.6 ** np.arange(5) * np.array([1, 1, 1, 1, 0.3])]
_N = [6, 42, 35, 5]
_G = 3.7


def _expected_ranks(spectra, g, tol):
    d = len(spectra) + 1
    delta = tol * g / np.sqrt(d - 1)
    ranks = [None] * (d - 1)
    scale = 1.0
    for k in range(d - 2, -1, -1):  # right to left
        sv = g * spectra[k] * scale
        r = len(sv)
        for cand in range(1, len(sv) + 1):
            if np.sum(sv[cand:] ** 2) <= delta ** 2:
                r = cand
                break
        ranks[k] = r
        scale *= np.linalg.norm(spectra[k][:r])
    return ranks


def _truncated_dense(seed, spectra, g, ranks, split=None):
    cut = [s[:r] for s, r in zip(spectra, ranks)]
    n = list(_N)
    cores, _ = prescribed_bond_mpo(seed, n, spectra, g, site1_split=split)
    # zero the discarded coefficients in the same cores: the construction with s_k cut to r_k
    out = [c.copy() for c in cores]
    for k, s in enumerate(spectra):
        w = np.zeros_like(s)
        w[: ranks[k]] = 1.0
        out[k] = out[k] * w[None, None, None, :]
    del cut
    return mpo.dense(out)


@pytest.mark.parametrize("tol", [0.02, 0.05, 0.1, 0.2])
def test_round_mpo_threshold_exact_ranks(tol):
    cores, s = prescribed_bond_mpo(11, _N, _SPECTRA, _G)
    np.testing.assert_allclose(mpo.norm(cores), _G, rtol=1e-13)
    B = rounding.round_mpo(cores, tol=tol)
    want = _expected_ranks(s, _G, tol)
    assert rounding.ranks(B)[1:-1] == want
    D, DB = mpo.dense(cores), mpo.dense(B)
    np.testing.assert_allclose(DB, _truncated_dense(11, s, _G, want), atol=1e-13 * _G)
    # TT-rounding guarantee of the cited SVD-based rounding: ||Y - round(Y)||_F <= tol ||Y||_F
    assert np.linalg.norm(D - DB) <= tol * np.linalg.norm(D) * (1 + 1e-12)


@pytest.mark.parametrize("tol", [0.02, 0.05, 0.1, 0.2])
def test_orthogonalize_threshold_exact_ranks(tol):
    """The same pin through MPO-QR: Y is a tall matrix with K = 3 columns on site 1 (6 = 2 x 3)."""
    Y, s = prescribed_bond_mpo(12, _N, _SPECTRA, _G, site1_split=(2, 3))
    Q, R = rounding.orthogonalize(Y, tol=tol)
    want = _expected_ranks(s, _G, tol)
    assert rounding.ranks(Q)[1:-1] == want
    DY = mpo.dense(Y)
    DT = _truncated_dense(12, s, _G, want, split=(2, 3))
    np.testing.assert_allclose(mpo.dense(Q) @ R, DT, atol=1e-13 * _G)
    assert np.linalg.norm(DY - mpo.dense(Q) @ R) <= tol * np.linalg.norm(DY) * (1 + 1e-12)


def test_prescribed_bond_spectra_are_the_svd_of_the_unfoldings():
    """The generator's claim, checked against LAPACK on the dense unfoldings (no oracle code)."""
    cores, s = prescribed_bond_mpo(11, _N, _SPECTRA, _G)
    D = mpo.dense(cores)  # rows = the multi-index over all sites (J = 1)
    T = D[:, 0].reshape(_N, order="F")
    for k in range(1, len(_N)):
        left = int(np.prod(_N[:k]))
        sv = np.linalg.svd(T.reshape(left, -1, order="F"), compute_uv=False)
        np.testing.assert_allclose(sv[: len(s[k - 1])], _G * s[k - 1], rtol=1e-12, atol=1e-14)
        assert np.all(sv[len(s[k - 1]):] < 1e-12)
