"""Reference gradient of the TNrSVD singular values with respect to the MPO cores (test
infrastructure only).

The differentiable form of the method keeps the ranks fixed (tol = 0: only exactly-zero singular
values are dropped; max_rank = K), so the map cores -> S is smooth where the singular values
of every step are simple. The reference gradient of L(A) = sum_{i < n_sv} S_i is taken by
central finite differences of the oracle forward (``tnrsvd.tnrsvd``): for a core entry e,
  dL/de ~= (L(A + h E_e) - L(A - h E_e)) / (2 h),
whose truncation error is O(h^2) and rounding error O(eps / h).

closed_form_exact() is the independent pin: when the randomized SVD is exact (K >= rank A and
no truncation), S are the singular values of the dense matrix, so dL/dA_dense = U_n V_n^T, and
because the dense matrix is multilinear in the cores (Thm 3.1's Kronecker structure), dL/de is
<U_n V_n^T, dense(A with core c replaced by the unit tensor E_e)>.
"""

import numpy as np

from . import mpo, tnrsvd


def loss(A, k, p, q, seed, n_sv, max_rank=None):
    K = int(k) + int(p)
    _, S, _ = tnrsvd.tnrsvd(A, k, p, q, seed, tol=0.0, max_rank=K if max_rank is None else max_rank)
    return float(np.sum(S[:n_sv]))


def fd_gradient(A, k, p, q, seed, n_sv, entries, h=1e-6, max_rank=None):
    """entries: list of (core index, flat Fortran-order index). Returns an array of dL/de."""
    out = []
    for c, e in entries:
        Ap = [x.copy() for x in A]
        Am = [x.copy() for x in A]
        fp = Ap[c].reshape(-1, order="F")
        fm = Am[c].reshape(-1, order="F")
        v = A[c].reshape(-1, order="F")[e]
        fp[e] = v + h
        fm[e] = v - h
        Ap[c] = fp.reshape(A[c].shape, order="F")
        Am[c] = fm.reshape(A[c].shape, order="F")
        out.append((loss(Ap, k, p, q, seed, n_sv, max_rank) - loss(Am, k, p, q, seed, n_sv, max_rank)) / (2 * h))
    return np.array(out)


def closed_form_exact(A, n_sv, entries):
    """dL/de for L = sum of the n_sv largest singular values of the dense matrix of A."""
    D = mpo.dense(A)
    U, s, Vt = np.linalg.svd(D, full_matrices=False)
    G = U[:, :n_sv] @ Vt[:n_sv]
    out = []
    for c, e in entries:
        Au = [x.copy() for x in A]
        unit = np.zeros(A[c].size)
        unit[e] = 1.0
        Au[c] = unit.reshape(A[c].shape, order="F")
        out.append(float(np.sum(G * mpo.dense(Au))))
    return np.array(out)
