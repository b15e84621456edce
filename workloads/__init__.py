"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module only draws and assembles inputs; it holds none of the method's arithmetic
(no contraction, orthogonalisation, SVD sweep or conversion of the paper). All generators
use numpy.random.default_rng(seed) (PCG64) and return float64 MPO cores as numpy arrays of
logical shape (R_k, I_k, J_k, R_{k+1}), or COO triplets for sparse matrices.

Workloads (sizes and distributions follow the paper's experiments, Section 6):
  gaussian_mpo    i.i.d. N(0,1) cores scaled by a constant (plain FP64 case: d=6, 4x4 sites, ranks 3)
  prescribed_mpo  A = U diag(sigma) V^T with orthogonal MPOs U, V (the construction of Section 6.3's
                  second experiment, there with TT_RAND; here from QR'd Gaussian cores)
  banded_coo      random banded sparse matrix standing in for the UF collection matrices of
                  Sections 6.1-6.2, which are not available here.
"""

import numpy as np


def gaussian_mpo(seed, I, J, R, scale=None):
    """Cores k = 1..d drawn in turn, each in memory order (r fastest), as N(0,1) * scale.

    ``scale`` is a float or a callable(k, core_shape) -> float; default 1.
    """
    rng = np.random.default_rng(seed)
    d = len(I)
    assert len(J) == d and len(R) == d + 1 and R[0] == 1 and R[-1] == 1
    cores = []
    for k in range(d):
        shape = (int(R[k]), int(I[k]), int(J[k]), int(R[k + 1]))
        g = rng.standard_normal(int(np.prod(shape))).reshape(shape, order="F")
        s = 1.0 if scale is None else (scale(k, shape) if callable(scale) else float(scale))
        cores.append(g * s)
    return cores


def _right_orthogonal_core(rng, r, n, r2):
    """r x n x 1 x r2 core whose r x (n r2) unfolding has orthonormal rows (needs r <= n r2)."""
    G = rng.standard_normal((n * r2, r))
    Qt, _ = np.linalg.qr(G)  # (n r2) x r orthonormal columns
    return Qt.T.reshape(r, n, 1, r2, order="F")


def orthogonal_mpo(seed, I1, dims, K, rank):
    """A rows x K matrix with orthonormal columns as an MPO with K on site 1.

    Site 1 is 1 x I1 x K x rank whose K x (I1 rank) matrix has orthonormal rows; sites 2..d are
    right-orthogonal rank x I_k x 1 x rank' cores, with the last bonds shrunk so that every
    unfolding can be right-orthogonal (rank' <= product of the remaining dims).
    """
    rng = np.random.default_rng(seed)
    d = 1 + len(dims)
    ranks = [1]
    for k in range(1, d):
        tail = int(np.prod(dims[k - 1:]))
        ranks.append(min(rank, tail))
    ranks.append(1)
    G = rng.standard_normal((I1 * ranks[1], K))
    Qt, _ = np.linalg.qr(G)  # (I1 R2) x K
    site1 = Qt.T.reshape(K, I1, ranks[1], order="F").transpose(1, 0, 2)[None]  # (1, I1, K, R2)
    cores = [site1.copy()]
    for k in range(1, d):
        cores.append(_right_orthogonal_core(rng, ranks[k], int(dims[k - 1]), ranks[k + 1]))
    return cores


def prescribed_mpo(seed_u, seed_v, I1, dims, K, rank, sigma):
    """A = U diag(sigma) V^T with U, V from ``orthogonal_mpo`` (square: the same site dims).

    Site 1: A_1(0, i, j, (a, b)) = sum_c U_1(0, i, c, a) sigma_c V_1(0, j, c, b); sites k >= 2:
    A_k((a,b), i, j, (a',b')) = U_k(a, i, 0, a') V_k(b, j, 0, b'); bonds (a, b) -> a + R_U b.
    The exact singular values of A are ``sigma`` (length K).
    """
    U = orthogonal_mpo(seed_u, I1, dims, K, rank)
    V = orthogonal_mpo(seed_v, I1, dims, K, rank)
    sigma = np.asarray(sigma, dtype=np.float64)
    cores = []
    u, v = U[0][0], V[0][0]  # (I1, K, a), (J1, K, b)
    c1 = np.einsum("ica,c,jcb->ijba", u, sigma, v)  # (I1, J1, b, a)
    ra, rb = u.shape[2], v.shape[2]
    cores.append(c1.reshape(I1, I1, rb * ra)[None].copy())  # (b, a) -> b*ra + a = a + ra*b
    for uk, vk in zip(U[1:], V[1:]):
        a1, n, _, a2 = uk.shape
        b1, _, _, b2 = vk.shape
        ck = np.einsum("aiu,bjv->baijvu", uk[:, :, 0, :], vk[:, :, 0, :])
        cores.append(ck.reshape(b1 * a1, n, n, b2 * a2).copy())
    return cores, U, V


def banded_coo(seed, n, per_row, half_band):
    """Sparse n x n matrix: each row i holds ``per_row`` distinct columns drawn uniformly from
    [i - half_band, i + half_band] intersected with [0, n), values N(0,1); COO sorted by (row, col).
    """
    rng = np.random.default_rng(seed)
    rows = np.arange(n, dtype=np.int64)
    lo = np.maximum(rows - half_band, 0)
    hi = np.minimum(rows + half_band, n - 1)
    width = hi - lo + 1
    assert width.min() >= per_row
    cols = np.empty((n, per_row), dtype=np.int64)
    todo = np.arange(n)
    while todo.size:
        u = rng.random((todo.size, per_row))
        c = lo[todo, None] + np.floor(u * width[todo, None]).astype(np.int64)
        c.sort(axis=1)
        bad = (np.diff(c, axis=1) == 0).any(axis=1)
        cols[todo[~bad]] = c[~bad]
        todo = todo[bad]
    vals = rng.standard_normal(n * per_row)
    vals[vals == 0.0] = 1.0  # no signed zeros in the inputs
    return np.repeat(rows, per_row), cols.reshape(-1), vals


# Named configurations of the paper-shaped workloads.

def c1_plain_fp64(seed=0):
    """4096 x 4096 Gaussian MPO: d=6, I=J=4, ranks 3, N(0,1)/sqrt(4*3); k=10, p=10, q=1."""
    d = 6
    A = gaussian_mpo(seed, [4] * d, [4] * d, [1] + [3] * (d - 1) + [1], scale=1.0 / np.sqrt(12.0))
    return dict(A=A, k=10, p=10, q=1, seed=seed, tol=1e-14, max_rank=0)


def c2_prescribed(seed_u=0, seed_v=1, seed_omega=2, tol=1e-12, max_rank=32):
    """2^20 x 2^20 MPO with sigma_j = 0.7^j (j < 32), built in merged layout (64, 4 x 7): U, V
    orthogonal rank-5 MPOs; A ranks 25 (16 at the last bond); k=16, p=16, q=2."""
    K = 32
    sigma = 0.7 ** np.arange(K)
    A, U, V = prescribed_mpo(seed_u, seed_v, 64, [4] * 7, K, 5, sigma)
    return dict(A=A, k=16, p=16, q=2, seed=seed_omega, tol=tol, max_rank=max_rank, sigma=sigma)


def batched_gaussian(seed, n, d_range=(8, 20), phys=(2, 4), rank_range=(4, 32), ks=(8, 16, 32), q=1, tol=1e-12):
    """Independent Gaussian-core MPOs for the batched solver, drawn problem by problem.

    Per problem: d uniform in d_range (inclusive), I_k = J_k = one value drawn from ``phys`` (the
    same for all sites), interior ranks uniform in rank_range (inclusive), cores N(0,1) scaled by
    1/sqrt(I_k R_k), k drawn from ``ks``, p = k, the given q, Omega seed = seed * 100003 + index,
    tol as given and max_rank = K = k + p. Returns a list of dicts (A: list of cores, k, p, q,
    seed, tol, max_rank).
    """
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        d = int(rng.integers(d_range[0], d_range[1] + 1))
        x = int(rng.choice(phys))
        R = [1] + [int(r) for r in rng.integers(rank_range[0], rank_range[1] + 1, size=d - 1)] + [1]
        k = int(rng.choice(ks))
        cores = gaussian_mpo(int(rng.integers(0, 2**31 - 1)), [x] * d, [x] * d, R,
                             scale=lambda kk, shape: 1.0 / np.sqrt(shape[1] * shape[0]))
        out.append(dict(A=cores, k=k, p=k, q=q, seed=seed * 100003 + i, tol=tol, max_rank=2 * k))
    return out


def prescribed_bond_mpo(seed, n, spectra, g=1.0, site1_split=None, canonical="right"):
    """An MPO whose Schmidt spectrum at every bond is prescribed (cores grouped as one physical
    index per site; interior bonds r_k = len(spectra[k-1])).

    n[k] is the physical size of site k (n[0] >= r_1, n[k] >= r_{k-1} r_k, n[-1] >= r_{d-1}); each
    spectra[k] is normalised to unit norm. Cores: site 1 is g * U_1[x, l_1] s_1[l_1]; site k is
    W_k[x, (l_{k-1}, l_k)] s_k[l_k]; site d is W_d[x, l_{d-1}], with U_1 and every W_k having
    orthonormal columns drawn by QR of Gaussian matrices (seeded). Because the coefficient tensor is
    a product over bonds and the basis functions are orthonormal, the Schmidt values at bond k are
    exactly g * s_k (and ||A||_F = g).

    site1_split=(I1, K): return site 1 as (1, I1, K, r_1) (a tall matrix with K columns on site 1,
    J_k = 1 elsewhere); otherwise every core is (r, n_k, 1, r'). canonical="left" moves each s_k
    (and g) onto the left bond of core k+1 instead (cores 1..d-1 then have orthonormal columns;
    the Schmidt values are the same). Returns (cores, normalised spectra).
    """
    rng = np.random.default_rng(seed)
    s = [np.asarray(x, dtype=np.float64) / np.linalg.norm(x) for x in spectra]
    d = len(s) + 1
    r = [1] + [len(x) for x in s] + [1]

    def orth(rows, cols):
        Q, _ = np.linalg.qr(rng.standard_normal((rows, cols)))
        return Q

    cores = []
    for k in range(d):
        rl, rr = r[k], r[k + 1]
        W = orth(int(n[k]), rl * rr).reshape(int(n[k]), rl, rr, order="F")  # column (l, l') -> l + rl l'
        c = W.transpose(1, 0, 2)  # (rl, n, rr)
        if canonical == "left":
            if k > 0:
                c = c * s[k - 1][:, None, None]
            if k == d - 1:
                c = c * float(g)
        else:
            if k < d - 1:
                c = c * s[k][None, None, :]
            if k == 0:
                c = c * float(g)
        cores.append(c[:, :, None, :].copy())
    if site1_split is not None:
        I1, K = site1_split
        assert I1 * K == int(n[0])
        cores[0] = cores[0][0, :, 0, :].reshape(I1, K, r[1], order="F")[None].copy()
    return cores, s


# Section 6.3's second experiment: N sites of 2 x 2, 50 prescribed singular values 0.5^k, random
# orthogonal U and V, rank-50 approximation (K = 100, q = 1), the paper's rounding tolerance for
# each N, and the first 7 sites merged (I_1 = 128 >= K).
PAPER_SIGMA_TOLS = {10: 1e-5, 15: 1e-6, 20: 1e-8, 25: 1e-8, 30: 1e-9, 35: 1e-10, 40: 1e-11, 45: 1e-12, 50: 1e-13}


def paper_prescribed(N, seed_u=0, seed_v=1, seed_omega=2, rank=5):
    """2^N x 2^N MPO A = U diag(0.5^k) V^T (k < 50) in the merged layout (site 1: 128 = 2^7 rows,
    sites 2..N-6: 2 x 2), U and V orthogonal MPOs of rank `rank` (A's ranks rank^2 = 25, the paper's
    maximal rank); k = 50, p = 50, q = 1, tol from PAPER_SIGMA_TOLS. max_rank = 40 bounds the
    buffers and never binds: range(A) lies in range(U) (and range(A^T) in range(V)), so every Q of
    the iteration has bond ranks of at most `rank`."""
    if N not in PAPER_SIGMA_TOLS:
        raise ValueError("N must be one of 10, 15, ..., 50")
    sigma = 0.5 ** np.arange(50)
    A, U, V = prescribed_mpo(seed_u, seed_v, 128, [2] * (N - 7), 50, rank, sigma)
    return dict(A=A, k=50, p=50, q=1, seed=seed_omega, tol=PAPER_SIGMA_TOLS[N], max_rank=40, sigma=sigma)


def hilbert_submatrix(N):
    """Dense H(:, 1:2^(N-1)) of the 2^N x 2^N Hilbert matrix, H(i, j) = 1 / (i + j - 1) (1-based)."""
    i = np.arange(1, 2 ** N + 1, dtype=np.float64)[:, None]
    j = np.arange(1, 2 ** (N - 1) + 1, dtype=np.float64)[None, :]
    return 1.0 / (i + j - 1.0)


def tt_svd_operator(D, I, J, tol):
    """MPO of a dense matrix by successive truncated SVDs (the TT-SVD of the tensor-train
    literature; an input builder for tests and benchmarks, not a step of the method). Row and column
    multi-indices are column-major (first site fastest), as everywhere in this package; at each of
    the d - 1 splits the smallest rank whose discarded squared singular values are at most
    (tol ||D||_F)^2 / (d - 1) is kept. Returns the cores (R_k, I_k, J_k, R_{k+1})."""
    d = len(I)
    T = np.asarray(D, dtype=np.float64).reshape(list(I) + list(J), order="F")
    # interleave to (i1, j1, i2, j2, ...): site k's physical pair adjacent
    perm = [x for k in range(d) for x in (k, d + k)]
    T = T.transpose(perm)
    delta2 = (tol * np.linalg.norm(D)) ** 2 / max(d - 1, 1)
    cores, r = [], 1
    M = T.reshape(r * I[0] * J[0], -1, order="F")
    for k in range(d - 1):
        U, s, Vt = np.linalg.svd(M, full_matrices=False)
        tail = np.concatenate([np.cumsum((s ** 2)[::-1])[::-1], [0.0]])
        keep = next(c for c in range(1, len(s) + 1) if tail[c] <= delta2)
        cores.append(U[:, :keep].reshape(r, I[k], J[k], keep, order="F"))
        M = (s[:keep, None] * Vt[:keep]).reshape(keep * I[k + 1] * J[k + 1], -1, order="F")
        r = keep
    cores.append(M.reshape(r, I[d - 1], J[d - 1], 1, order="F"))
    return cores


def paper_hilbert(N, tol=1e-11, seed_omega=2):
    """Section 6.3's first experiment, H(:, 1:2^(N-1)) with N row sites and N - 1 column sites of 2
    (the last site has J = 1), as an MPO from tt_svd_operator (the paper used TT-cross with relative
    error 1e-11); rank-16 approximation, K = 32, q = 2, rounding tolerance 1e-9 (5 sites merged).
    For N <= 12 (a dense 4096 x 2048 matrix at most). max_rank = 64 bounds the buffers and does not
    bind (the rounded bonds stay below 40 at tolerance 1e-9)."""
    if N > 12:
        raise ValueError("the dense TT-SVD construction is for N <= 12")
    I = [2] * N
    J = [2] * (N - 1) + [1]
    D = hilbert_submatrix(N)
    return dict(A=tt_svd_operator(D, I, J, tol), k=16, p=16, q=2, seed=seed_omega, tol=1e-9, max_rank=64, dense=D)
