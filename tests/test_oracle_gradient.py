"""Pins of the reference gradient (central finite differences of the oracle TNrSVD).

In the exact case (K >= rank A, no truncation) the finite-difference gradient of the sum of the
leading singular values must equal the closed form U_n V_n^T pushed through the multilinear
core map; a planted error in the closed form's singular vectors is detected."""

import numpy as np

import workloads as W
from oracle import gradient as og


def _entries(A, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        c = int(rng.integers(0, len(A)))
        out.append((c, int(rng.integers(0, A[c].size))))
    return out


def test_fd_matches_closed_form_when_exact():
    # 16 x 16 matrix, K = 16 = full dimension: the randomized SVD is exact
    A = W.gaussian_mpo(4, [4, 4], [4, 4], [1, 3, 1])
    ent = _entries(A, 10, 1)
    fd = og.fd_gradient(A, 8, 8, 1, 5, 3, ent)
    cf = og.closed_form_exact(A, 3, ent)
    assert np.linalg.norm(fd - cf) <= 1e-7 * np.linalg.norm(cf)


def test_fd_matches_closed_form_exact_recovery_low_rank():
    # 128 x 128 matrix of rank 8 = K (prescribed sigma = 0.7^j): the sketch spans range(A), and
    # to first order it keeps doing so under a perturbation, so the closed form holds
    A, _, _ = W.prescribed_mpo(0, 1, 16, [2, 2, 2], 8, 3, 0.7 ** np.arange(8))
    ent = _entries(A, 10, 2)
    fd = og.fd_gradient(A, 4, 4, 1, 7, 3, ent)
    cf = og.closed_form_exact(A, 3, ent)
    assert np.linalg.norm(fd - cf) <= 1e-6 * np.linalg.norm(cf)


def test_closed_form_detects_a_wrong_vector_pair():
    A = W.gaussian_mpo(4, [4, 4], [4, 4], [1, 3, 1])
    ent = _entries(A, 10, 1)
    fd = og.fd_gradient(A, 8, 8, 1, 5, 3, ent)
    D = og.mpo.dense(A)
    U, s, Vt = np.linalg.svd(D)
    G_wrong = U[:, [0, 1, 3]] @ Vt[[0, 1, 3]]  # third pair replaced by the fourth
    wrong = []
    for c, e in ent:
        Au = [x.copy() for x in A]
        unit = np.zeros(A[c].size)
        unit[e] = 1.0
        Au[c] = unit.reshape(A[c].shape, order="F")
        wrong.append(float(np.sum(G_wrong * og.mpo.dense(Au))))
    assert np.linalg.norm(fd - np.array(wrong)) > 1e-3 * np.linalg.norm(fd)
