"""TNrSVD of a sparse matrix held in the block form of Alg. 4.1 (test infrastructure only).

The MPO that Alg. 4.1 produces has rank R (the number of nonzero I_1 x J_1 blocks, Lemma 4.2) at
every bond, so MPO-times-MPO products with it (Section 5.2) multiply ranks by R. The block form
applies the same operator directly: A = sum_t E^(d)_t (x) ... (x) E^(2)_t (x) X_t (Eq. (4.1)),
and the Kronecker factor E^(d)_t (x) ... (x) E^(2)_t only selects the block row p_t and block
column q_t (p = i_2 + I_2 (i_3 + ...), Eq. (2.1)); so A Q adds X_t Q[q_t J_1 : (q_t + 1) J_1] to rows
p_t I_1 .. p_t I_1 + I_1 - 1, and A^T Q adds X_t^T Q[p_t I_1 : ...] to the rows of block column q_t.

sparse_tnrsvd runs Alg. 5.4 / 5.1 with this operator on dense tall matrices: Omega is the
random MPO of Lemma 5.1 over the merged column dims (merge rule of Section 6.3), expanded to
its dense (prod J) x K matrix; every QR and the final SVD are LAPACK's. Without truncation
(tol = 0, no rank cap) TNrSVD's MPO products and roundings are exact, so its result is the
same as this one in exact arithmetic (the test pins it against the MPO oracle on small cases).
"""

import numpy as np

from . import mpo, rng


def block_rows_cols(digits, I, J):
    """(p_t, q_t): the block-row and block-column numbers of every block (mixed radix, i_2 fastest)."""
    d = len(I)
    R = digits.shape[0]
    p = np.zeros(R, dtype=np.int64)
    q = np.zeros(R, dtype=np.int64)
    sp, sq = 1, 1
    for k in range(1, d):
        p += digits[:, 2 * (k - 1)].astype(np.int64) * sp
        q += digits[:, 2 * (k - 1) + 1].astype(np.int64) * sq
        sp *= int(I[k])
        sq *= int(J[k])
    return p, q


def apply(R, X, digits, I, J, Qd, trans=False):
    """A Qd (trans=False) or A^T Qd with A in block form; Qd is dense (ncols x K) or (nrows x K)."""
    I1, J1 = int(I[0]), int(J[0])
    p, q = block_rows_cols(digits, I, J)
    Xb = X.reshape(R, J1, I1).transpose(0, 2, 1)  # Xb[t] = X_t (I1 x J1)
    K = Qd.shape[1]
    if not trans:
        nrows = int(np.prod(np.asarray(I, dtype=object)))
        out = np.zeros((nrows, K))
        src = Qd.reshape(-1, J1, K)[q]              # (R, J1, K): the block column's rows of Qd
        contrib = np.einsum("tij,tjk->tik", Xb, src)  # (R, I1, K)
        np.add.at(out.reshape(-1, I1, K), p, contrib)
    else:
        ncols = int(np.prod(np.asarray(J, dtype=object)))
        out = np.zeros((ncols, K))
        src = Qd.reshape(-1, I1, K)[p]
        contrib = np.einsum("tij,tik->tjk", Xb, src)  # X_t^T Qd-block: (R, J1, K)
        np.add.at(out.reshape(-1, J1, K), q, contrib)
    return out


def omega_dense(seed, J, K):
    """Dense (prod J) x K matrix of the Lemma 5.1 MPO over the merged column dims."""
    return mpo.dense(rng.omega(seed, J, K))


def sparse_tnrsvd(R, X, digits, I, J, k, p, q, seed):
    """Returns (U (nrows x k), S (k), V (ncols x k)) of Alg. 5.4 / 5.1 with the block operator."""
    K = int(k) + int(p)
    m = mpo.merge_count(I, J, K)
    if m is None:
        raise ValueError("K exceeds prod(I) or prod(J)")
    Jm = [int(np.prod(J[:m]))] + [int(x) for x in J[m:]]
    O = omega_dense(seed, Jm, K)
    Q, _ = np.linalg.qr(apply(R, X, digits, I, J, O))
    for _ in range(int(q)):
        Q, _ = np.linalg.qr(apply(R, X, digits, I, J, Q, trans=True))
        Q, _ = np.linalg.qr(apply(R, X, digits, I, J, Q))
    Z = apply(R, X, digits, I, J, Q, trans=True)  # B^T = A^T Q
    Qz, Rz = np.linalg.qr(Z)                      # B = Rz^T Qz^T
    W, S, Zt = np.linalg.svd(Rz.T)
    return Q @ W[:, :k], S[:k], (Qz @ Zt.T)[:, :k]


def coo_tnrsvd(rows, cols, vals, nrows, ncols, I, J, k, p, q, seed):
    """The same computation with the operator taken straight from the COO input (scipy.sparse
    CSR products as the matmul step); used at sizes where the block loop above is too slow."""
    import scipy.sparse as sp

    K = int(k) + int(p)
    m = mpo.merge_count(I, J, K)
    if m is None:
        raise ValueError("K exceeds prod(I) or prod(J)")
    Jm = [int(np.prod(J[:m]))] + [int(x) for x in J[m:]]
    A = sp.csr_matrix((np.asarray(vals, dtype=np.float64), (np.asarray(rows), np.asarray(cols))),
                      shape=(int(nrows), int(ncols)))
    At = A.T.tocsr()
    O = omega_dense(seed, Jm, K)
    Q, _ = np.linalg.qr(A @ O)
    for _ in range(int(q)):
        Q, _ = np.linalg.qr(At @ Q)
        Q, _ = np.linalg.qr(A @ Q)
    Z = At @ Q
    Qz, Rz = np.linalg.qr(Z)
    W, S, Zt = np.linalg.svd(Rz.T)
    return Q @ W[:, :k], S[:k], (Qz @ Zt.T)[:, :k]
