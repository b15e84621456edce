"""MPO basics for the oracle (test infrastructure only; see package docstring).

An MPO is a list of float64 cores; core k has shape (R_k, I_k, J_k, R_{k+1}) with
R_1 = R_{d+1} = 1 (Section 3). A matrix with K columns carried by site 1 (the Y, Q, U, V
matrices of Section 5) is an MPO whose site-1 core is (1, I_1, K, R_2) and whose other cores
have J_k = 1, exactly as the paper writes them in Lemma 5.1 and Algs. 5.2-5.3.
"""

import numpy as np


def dims(cores):
    """Return (I, J, R) lists of an MPO: row dims, column dims and the d+1 ranks."""
    I = [c.shape[1] for c in cores]
    J = [c.shape[2] for c in cores]
    R = [cores[0].shape[0]] + [c.shape[3] for c in cores]
    return I, J, R


def check(cores):
    """Validate bond consistency (Section 3: R_k of core k equals R_k of core k-1's last mode)."""
    assert cores[0].shape[0] == 1 and cores[-1].shape[3] == 1, "R_1 = R_{d+1} = 1 (Section 3)"
    for a, b in zip(cores[:-1], cores[1:]):
        assert a.shape[3] == b.shape[0], "bond mismatch"


def dense(cores):
    """Contract an MPO into its dense matrix A([i1..id],[j1..jd]) (Section 3, Eq. (2.1)).

    Rows and columns are multi-indices with the first site varying fastest:
    row = i1 + I1*(i2 + I2*(i3 + ...)). The contraction is the plain sum over bond indices.
    """
    check(cores)
    T = cores[0][0]  # (I1, J1, R2)
    for c in cores[1:]:
        nr, nc = T.shape[0], T.shape[1]
        # new row index (a, i) -> a + nr*i ; new column (b, j) -> b + nc*j
        T = np.einsum("abr,rijs->iajbs", T, c)
        T = T.reshape(c.shape[1] * nr, c.shape[2] * nc, c.shape[3])
    return T[:, :, 0].copy()


def kron_chain(mats):
    """A^(d) (x) ... (x) A^(1) for mats = [A^(1), ..., A^(d)] (Thm 3.1 order reversal)."""
    out = np.ones((1, 1))
    for m in mats:
        out = np.kron(m, out)
    return out


def rank_bounds(I, J):
    """Thm 3.2: R_k <= min(prod_{i<k} I_i J_i, prod_{i>=k} I_i J_i) for k = 2..d."""
    d = len(I)
    IJ = [int(a) * int(b) for a, b in zip(I, J)]
    out = []
    for k in range(1, d):
        left = int(np.prod(IJ[:k], dtype=object))
        right = int(np.prod(IJ[k:], dtype=object))
        out.append(min(left, right))
    return out


def merge_count(I, J, K):
    """Smallest m with prod_{k<=m} I_k >= K and prod_{k<=m} J_k >= K.

    Algs. 5.2/5.3 require I_1 >= K and J_1 >= K; Section 6.3 meets this by contracting the
    first few MPO tensors (5 cores for K = 32 with 2x2 sites, 7 cores for K = 100).
    Returns None when even all d sites together are too small.
    """
    pi, pj = 1, 1
    for m in range(1, len(I) + 1):
        pi *= int(I[m - 1])
        pj *= int(J[m - 1])
        if pi >= K and pj >= K:
            return m
    return None


def merge_leading(cores, m):
    """Contract cores 1..m into one core 1 x (I1..Im) x (J1..Jm) x R_{m+1} (Section 6.3).

    The merged row index is the multi-index [i1..im] of Eq. (2.1) (site 1 fastest), and the
    same for columns, so the merged MPO represents the same matrix.
    """
    T = cores[0][0]  # (I1, J1, R2)
    for c in cores[1:m]:
        nr, nc = T.shape[0], T.shape[1]
        T = np.einsum("abr,rijs->iajbs", T, c).reshape(c.shape[1] * nr, c.shape[2] * nc, c.shape[3])
    return [T[None]] + [c.copy() for c in cores[m:]]


def contract(A, X, trans=False):
    """MPO x MPO product over the shared physical index (Section 5.2).

    trans=False: Y = A X. Per site, Y_k((r,s), i, c, (r',s')) = sum_j A_k(r,i,j,r') X_k(s,j,c,s').
    trans=True:  Y = A^T X. Per site, Y_k((r,s), j, c, (r',s')) = sum_i A_k(r,i,j,r') X_k(s,i,c,s').
    Product bonds are numbered (r, s) -> r + R*s. Ranks multiply (Section 5.2).
    """
    assert len(A) == len(X)
    out = []
    for a, x in zip(A, X):
        R, Ia, Ja, R2 = a.shape
        S, Ix, Kx, S2 = x.shape
        if not trans:
            assert Ja == Ix
            y = np.einsum("rijt,sjku->srikut", a, x).reshape(S * R, Ia, Kx, S2 * R2)
        else:
            assert Ia == Ix
            y = np.einsum("rijt,siku->srjkut", a, x).reshape(S * R, Ja, Kx, S2 * R2)
        out.append(y)
    return out


def transpose(A):
    """MPO of A^T: swap I_k and J_k in every core (no arithmetic)."""
    return [c.transpose(0, 2, 1, 3).copy() for c in A]


def inner(X, Y):
    """X^T Y for two MPOs with equal row dims and J_k = 1 for k >= 2 (K columns on site 1).

    Transfer matrices from the right: E_{d+1} = 1, E_k(a,b) = sum_{i,a',b'} X_k(a,i,0,a')
    Y_k(b,i,0,b') E_{k+1}(a',b'); finally G(c,e) = sum X_1(0,i,c,a') Y_1(0,i,e,b') E_2(a',b').
    """
    E = np.ones((1, 1))
    for x, y in zip(reversed(X[1:]), reversed(Y[1:])):
        E = np.einsum("aiu,biv,uv->ab", x[:, :, 0, :], y[:, :, 0, :], E)
    return np.einsum("icu,iev,uv->ce", X[0][0], Y[0][0], E)


def sandwich(U, A, V):
    """U^T A V for MPO U (rows I, k cols on site 1), operator A (I x J), V (rows J, k cols)."""
    E = np.ones((1, 1, 1))
    for u, a, v in zip(reversed(U[1:]), reversed(A[1:]), reversed(V[1:])):
        E = np.einsum("aix,bijy,cjz,xyz->abc", u[:, :, 0, :], a, v[:, :, 0, :], E)
    return np.einsum("ipx,ijy,jqz,xyz->pq", U[0][0], A[0][0], V[0][0], E)


def norm(cores):
    """Frobenius norm of an MPO via <A, A> transfer matrices (grouping I_k J_k as one index)."""
    E = np.ones((1, 1))
    for c in reversed(cores):
        E = np.einsum("aijx,bijy,xy->ab", c, c, E)
    return float(np.sqrt(E[0, 0]))


def flat(core):
    """Core -> 1-D float64 array in memory order (r fastest, then i, j, r')."""
    return np.asarray(core, dtype=np.float64).reshape(-1, order="F")


def unflat(buf, shape):
    """Inverse of ``flat``."""
    return np.asarray(buf, dtype=np.float64)[: int(np.prod(shape))].reshape(shape, order="F")
