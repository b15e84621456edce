"""MPO-QR (Alg. 5.2) with integrated rounding, MPO-SVD (Alg. 5.3) and MPO rounding.

Test infrastructure only. Reading of Section 5.4 used here: "apply a left-to-right rounding
sweep first, followed by the right-to-left sweep of Alg. 5.2" is taken as
  1. left-to-right orthogonalisation: for k = 1..d-1, thin Householder QR (LAPACK) of core k
     reshaped (R_k I_k J_k) x R_{k+1}; Q replaces the core, R is absorbed into core k+1;
  2. right-to-left sweep of Alg. 5.2 with truncation: for k = d..2, SVD of core k reshaped
     R_k x (I_k J_k R_{k+1}) = U S V^T; keep the leading r singular triplets, core k <- V^T
     (orthonormal rows, as Alg. 5.2 requires of Q_i), and core k-1 <- core k-1 x_4 (U S);
  3. site 1 as Alg. 5.2 (or Alg. 5.3) states it.
Step 1 is the orthogonalisation half of the SVD-based TT rounding the paper cites (Oseledets,
p. 2308); step 2 is its compression half, fused with Alg. 5.2's sweep so the right-to-left
sweep is done once.

Truncation rule (the paper varies its tolerance per experiment and fixes no rule): with
delta = tol * ||Y||_F / sqrt(d - 1), at each bond keep the smallest r >= 1 such that
sum_{l > r} s_l^2 <= delta^2, then r <- min(r, max_rank) when max_rank > 0.
"""

import numpy as np


def keep_rank(s, delta, max_rank):
    """Smallest r >= 1 with sum_{l >= r} s_l^2 <= delta^2 (0-based), capped by max_rank."""
    s = np.asarray(s, dtype=np.float64)
    tail = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])  # tail[r] = sum_{l>=r} s_l^2
    r = len(s)
    for cand in range(1, len(s) + 1):
        if tail[cand] <= delta * delta:
            r = cand
            break
    if max_rank and max_rank > 0:
        r = min(r, int(max_rank))
    return max(r, 1)


def _lr_orthogonalize(cores):
    """Left-to-right QR sweep (step 1). Returns the new cores (last core carries the norm)."""
    cores = [c.copy() for c in cores]
    d = len(cores)
    for k in range(d - 1):
        t, I, Kx, t2 = cores[k].shape
        M = cores[k].reshape(t * I * Kx, t2, order="F")
        Q, Rf = np.linalg.qr(M, mode="reduced")
        n = Q.shape[1]
        cores[k] = Q.reshape(t, I, Kx, n, order="F")
        cores[k + 1] = np.einsum("ab,bijc->aijc", Rf, cores[k + 1])
    return cores


def _rl_truncate(cores, tol, max_rank):
    """Right-to-left truncating SVD sweep (step 2) over sites d..2. Returns cores, ranks."""
    d = len(cores)
    nrm = np.linalg.norm(cores[-1])
    delta = tol * nrm / np.sqrt(d - 1) if d > 1 else 0.0
    for k in range(d - 1, 0, -1):
        t, I, Kx, t2 = cores[k].shape
        M = cores[k].reshape(t, I * Kx * t2, order="F")
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        r = keep_rank(s, delta, max_rank)
        cores[k] = Vt[:r].reshape(r, I, Kx, t2, order="F")
        US = U[:, :r] * s[:r]
        cores[k - 1] = np.einsum("aijb,bc->aijc", cores[k - 1], US)
    return cores


def _site1_matrix(core):
    """Alg. 5.2/5.3: permute site 1 (1, I1, K, R2) to K x 1 x I1 x R2 and reshape to K x (I1 R2)."""
    _, I1, K, R2 = core.shape
    return core[0].transpose(1, 0, 2).reshape(K, I1 * R2, order="F")


def _site1_core(M, I1, R2):
    """Inverse permutation of ``_site1_matrix`` for a K x (I1 R2) matrix."""
    K = M.shape[0]
    return M.reshape(K, I1, R2, order="F").transpose(1, 0, 2)[None].copy()


def orthogonalize(Y, tol=0.0, max_rank=0):
    """MPO-QR of Y (rows I, K columns on site 1) with integrated rounding (Alg. 5.2, Sec. 5.4).

    Returns (Q, R) with Q^T Q = I_K and Y ~= Q R, R upper triangular K x K: the site-1 matrix
    A_1 (K x I1 R2) is factored as A_1 = R^T Q_1 through the thin QR of A_1^T.
    """
    cores = _lr_orthogonalize(Y)
    cores = _rl_truncate(cores, tol, max_rank)
    _, I1, K, R2 = cores[0].shape
    A1 = _site1_matrix(cores[0])
    Qt, Rt = np.linalg.qr(A1.T, mode="reduced")  # A1^T = Qt Rt, so A1 = Rt^T Qt^T
    cores[0] = _site1_core(Qt.T, I1, R2)
    return cores, Rt


def mpo_svd(Z, tol=0.0, max_rank=0):
    """Economical SVD B = W S V^T of B = Z^T (K x J) given Z (rows J, K columns on site 1).

    Alg. 5.3 with the rounding of Section 5.4: the same two sweeps as ``orthogonalize``, then
    the SVD of the K x (J1 R2) site-1 matrix gives W, S and V^(1). Returns (W, S, V) where V is
    an MPO with rows J and K columns on site 1, V^T V = I_K.
    """
    cores = _lr_orthogonalize(Z)
    cores = _rl_truncate(cores, tol, max_rank)
    _, J1, K, R2 = cores[0].shape
    A1 = _site1_matrix(cores[0])
    W, S, V1t = np.linalg.svd(A1, full_matrices=False)
    cores[0] = _site1_core(V1t, J1, R2)
    return W, S, cores


def round_mpo(A, tol=0.0, max_rank=0):
    """SVD-based MPO rounding (Section 3): the two sweeps with I_k J_k grouped as one index."""
    cores = _lr_orthogonalize(A)
    return _rl_truncate(cores, tol, max_rank)


def ranks(cores):
    return [cores[0].shape[0]] + [c.shape[3] for c in cores]


# ---- truncate-as-you-go (zip-up) rounding of a product: the product is rounded while it is formed ----
#
# Reading (a variant of Section 5.4's "rounding sweep first, then the sweep of Alg. 5.2"): the
# first sweep of the rounding is fused with the MPO x MPO product of Section 5.2, so the product
# cores of rank R_k S_k are never formed in full. The sweep runs right to left (the merged site 1
# of Section 6.3 carries I_1 K rows, so it is the one site left unfactored):
#   C_d = [1];  for k = d..2:
#     T_k = (product core k) x_4 C_{k+1}, reshaped (R_k S_k) x (n_k K_k t_{k+1});
#     T_k = U diag(s) V^T (SVD); keep the smallest r >= 1 with
#       sum_{l > r} s_l^2 <= tol^2 ||T_k||_F^2 / (d - 1),  then r <= max_rank if max_rank > 0;
#     core k <- V^T[:r] (orthonormal rows);  C_k <- U[:, :r] diag(s[:r]);
#   core 1 <- (product core 1) x_4 C_2.
# The threshold is relative to the local matrix T_k: the norm of the whole product is not known
# before the sweep ends (it equals ||T_k||_F when the not-yet-swept left part is orthonormal,
# which is when this truncation is the optimal one). The result is then rounded and
# orthogonalised exactly as ``orthogonalize`` does (its two sweeps and the site-1 step), now on
# bonds of at most max_rank.

def zipup_product(A, X, trans=False, tol=0.0, max_rank=0):
    """op(A) X (Section 5.2) formed and truncated site by site, right to left (see above)."""
    from .mpo import contract

    d = len(A)
    cores = [None] * d
    C = np.ones((1, 1))
    for k in range(d - 1, -1, -1):
        Yk = contract([A[k]], [X[k]], trans)[0]  # (R S, n, Kx, R' S'): the product core of site k
        T = np.einsum("axcb,bt->axct", Yk, C)  # absorb the carried factor into the right bond
        if k == 0:
            cores[0] = T
            break
        rs, n, kx, t = T.shape
        M = T.reshape(rs, n * kx * t, order="F")
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        delta = tol * np.linalg.norm(s) / np.sqrt(d - 1) if d > 1 else 0.0
        r = keep_rank(s, delta, max_rank)
        cores[k] = Vt[:r].reshape(r, n, kx, t, order="F")
        C = U[:, :r] * s[:r]
    return cores


def orthogonalize_zipup(A, X, trans=False, tol=0.0, max_rank=0):
    """MPO-QR (Alg. 5.2 with the rounding of Section 5.4) of op(A) X rounded as it is formed."""
    return orthogonalize(zipup_product(A, X, trans, tol, max_rank), tol, max_rank)


def mpo_svd_zipup(A, X, tol=0.0, max_rank=0):
    """MPO-SVD (Alg. 5.3) of B = (A^T X)^T with A^T X rounded as it is formed."""
    return mpo_svd(zipup_product(A, X, True, tol, max_rank), tol, max_rank)
