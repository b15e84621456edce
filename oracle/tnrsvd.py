"""TNrSVD driver (Alg. 5.4 feeding Alg. 5.1) and a dense rSVD cross-check (test infrastructure).

tnrsvd(A, k, p, q, seed):
  K = k + p (oversampling, Section 5.1: compute rank K, keep the first k = K/2 in the paper).
  Merge leading sites until I_1 >= K and J_1 >= K (Section 6.3).
  Omega from Lemma 5.1 with the seeded stream of ``rng``.
  Y = A Omega; Q = MPO-QR(Y); q times { Y = A^T Q; Q = MPO-QR(Y); Y = A Q; Q = MPO-QR(Y) }   (Alg. 5.4)
  B = Q^T A is formed as the MPO Z = A^T Q (= B^T); W, S, V = MPO-SVD(Z)                     (Alg. 5.3)
  U = Q x_3 W^T on site 1 (Section 5.4); return the first k columns of U and V and S[:k].
"""

import numpy as np

from . import mpo, rng, rounding


def tnrsvd(A, k, p, q, seed, tol=0.0, max_rank=0, return_info=False, rounding_mode="two_sweep"):
    """rounding_mode: "two_sweep" (the product is formed, then orthogonalised with the rounding of
    Section 5.4) or "zipup" (every product is rounded while it is formed, right to left, then
    orthogonalised the same way; see rounding.zipup_product)."""
    K = int(k) + int(p)
    zip_ = rounding_mode == "zipup"
    if rounding_mode not in ("two_sweep", "zipup"):
        raise ValueError("rounding_mode must be 'two_sweep' or 'zipup'")

    def qr_of_product(X, trans):
        if zip_:
            return rounding.orthogonalize_zipup(Am, X, trans, tol, max_rank)
        return rounding.orthogonalize(mpo.contract(Am, X, trans=trans), tol, max_rank)

    I, J, _ = mpo.dims(A)
    m = mpo.merge_count(I, J, K)
    if m is None:
        raise ValueError("K exceeds prod(I) or prod(J): no merge reaches I_1 >= K, J_1 >= K")
    Am = mpo.merge_leading(A, m) if m > 1 else [c.copy() for c in A]
    Im, Jm, _ = mpo.dims(Am)
    Om = rng.omega(seed, Jm, K)
    info = {"merge": m, "ranks": []}
    Q, _ = qr_of_product(Om, False)
    info["ranks"].append(rounding.ranks(Q))
    for _ in range(int(q)):
        Q, _ = qr_of_product(Q, True)
        info["ranks"].append(rounding.ranks(Q))
        Q, _ = qr_of_product(Q, False)
        info["ranks"].append(rounding.ranks(Q))
    if zip_:
        W, S, V = rounding.mpo_svd_zipup(Am, Q, tol, max_rank)
    else:
        W, S, V = rounding.mpo_svd(mpo.contract(Am, Q, trans=True), tol, max_rank)
    info["ranks"].append(rounding.ranks(V))
    U = [c.copy() for c in Q]
    U[0] = np.einsum("aicb,ce->aieb", Q[0], W)[:, :, :k, :].copy()
    V = [c.copy() for c in V]
    V[0] = V[0][:, :, :k, :].copy()
    if return_info:
        return U, S[:k].copy(), V, info
    return U, S[:k].copy(), V


def dense_rsvd(A, O, q):
    """Alg. 5.1 with the subspace iteration of Alg. 5.4 on dense matrices (LAPACK QR/SVD)."""
    Q, _ = np.linalg.qr(A @ O)
    for _ in range(int(q)):
        Q, _ = np.linalg.qr(A.T @ Q)
        Q, _ = np.linalg.qr(A @ Q)
    B = Q.T @ A
    W, S, Vt = np.linalg.svd(B, full_matrices=False)
    return Q @ W, S, Vt.T


def sv_error(S, S_ref):
    """Relative singular-value error ||S - S_ref||_F / ||S_ref||_F (Section 6.3 metric)."""
    S = np.asarray(S, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    return float(np.linalg.norm(S - S_ref) / np.linalg.norm(S_ref))
