"""Sparse matrix -> MPO conversion, Alg. 4.1 (test infrastructure only).

Alg. 4.1 writes A as a sum over its nonzero I_1 x J_1 blocks X of rank-1 MPOs
E^(d)_{i_d j_d} (x) ... (x) E^(2)_{i_2 j_2} (x) X, where E_{ij} is the unit matrix with a single
1 at (i, j) (Section 4.1, Eq. (4.1) "sumofkron2"); adding them adds ranks, so the MPO rank is the
number of nonzero blocks (Lemma 4.2).

Block form. Because every core but the first is a selection (Section 4.2: "almost all of the
MPO-tensors will be sparse"), the result is stored as
  R        number of blocks,
  X        float64 array, block t at X[t*I1*J1 : (t+1)*I1*J1], column-major I1 x J1
           (this is exactly core A^(1)(0, i1, j1, t) in memory order),
  digits   uint8 array of shape (R, 2*(d-1)): row t holds i_2, j_2, i_3, j_3, ..., i_d, j_d.
Readings the paper leaves open: a block exists when at least one COO entry falls in it (an
explicitly stored zero still creates its block); blocks are ordered by (block-row p, block-col q)
lexicographically, p major; p = i_2 + I_2*(i_3 + ...) is split in mixed radix with i_2 fastest
(Eq. (2.1)), and likewise q. Duplicate (row, col) entries are rejected.
"""

import numpy as np


class ConversionError(ValueError):
    pass


def convert(rows, cols, vals, nrows, ncols, I, J):
    """Alg. 4.1: return (R, X, digits) for the COO matrix (rows, cols, vals)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    d = len(I)
    if len(J) != d or d < 1:
        raise ConversionError("I and J must have the same number d >= 1 of factors")
    if int(np.prod(np.asarray(I, dtype=object))) != nrows or int(np.prod(np.asarray(J, dtype=object))) != ncols:
        raise ConversionError("prod(I) must equal nrows and prod(J) must equal ncols (Section 4.1)")
    if any(int(v) > 256 for v in list(I[1:]) + list(J[1:])):
        raise ConversionError("digit storage is uint8: I_k, J_k <= 256 for k >= 2")
    if rows.size and (rows.min() < 0 or rows.max() >= nrows or cols.min() < 0 or cols.max() >= ncols):
        raise ConversionError("index out of range")
    I1, J1 = int(I[0]), int(J[0])
    nq = ncols // J1
    p, i1 = rows // I1, rows % I1
    q, j1 = cols // J1, cols % J1
    key = p * nq + q
    # Duplicate entries: same (row, col) twice.
    flatpos = rows * ncols + cols
    if np.unique(flatpos).size != flatpos.size:
        raise ConversionError("duplicate (row, col) entry")
    ukeys, t = np.unique(key, return_inverse=True)  # sorted: p major, then q
    R = int(ukeys.size)
    X = np.zeros(R * I1 * J1, dtype=np.float64)
    # "Construct rank-1 MPO T with X": X_t(i1, j1) = value, column-major within the block.
    X[t * I1 * J1 + i1 + I1 * j1] = vals
    digits = np.zeros((R, 2 * (d - 1)), dtype=np.uint8)
    bp, bq = ukeys // nq, ukeys % nq
    for k in range(1, d):  # "Determine d-1 E_ij matrices": digits of p and q, site 2 fastest
        digits[:, 2 * (k - 1)] = bp % int(I[k])
        digits[:, 2 * (k - 1) + 1] = bq % int(J[k])
        bp //= int(I[k])
        bq //= int(J[k])
    return R, X, digits


def block_cores(R, X, digits, I, J):
    """Expand block form into the dense MPO cores of Alg. 4.1 (for small tests).

    Site 1: A1(0, i1, j1, t) = X_t(i1, j1). Sites 2..d-1: A_k(t, i, j, t) = [i = i_{t,k}][j = j_{t,k}].
    Site d: A_d(t, i, j, 0) = [i = i_{t,d}][j = j_{t,d}]. With d = 1 the single core is X itself.
    """
    d = len(I)
    I1, J1 = int(I[0]), int(J[0])
    if d == 1:
        core = np.zeros((1, I1, J1, 1))
        for t in range(R):
            core[0, :, :, 0] += X[t * I1 * J1:(t + 1) * I1 * J1].reshape(I1, J1, order="F")
        return [core]
    cores = [X.reshape(R, J1, I1).transpose(2, 1, 0)[None].copy()]  # (1, I1, J1, R)
    for k in range(1, d):
        last = k == d - 1
        c = np.zeros((R, int(I[k]), int(J[k]), 1 if last else R))
        for t in range(R):
            c[t, digits[t, 2 * (k - 1)], digits[t, 2 * (k - 1) + 1], 0 if last else t] = 1.0
        cores.append(c)
    return cores


def dense_from_blocks(R, X, digits, I, J):
    """Reconstruct the dense matrix directly from block form (sum of Kronecker terms, Eq. (4.1))."""
    d = len(I)
    I1, J1 = int(I[0]), int(J[0])
    nrows = int(np.prod(np.asarray(I, dtype=object)))
    ncols = int(np.prod(np.asarray(J, dtype=object)))
    A = np.zeros((nrows, ncols))
    for t in range(R):
        term = X[t * I1 * J1:(t + 1) * I1 * J1].reshape(I1, J1, order="F")
        for k in range(1, d):
            E = np.zeros((int(I[k]), int(J[k])))
            E[digits[t, 2 * (k - 1)], digits[t, 2 * (k - 1) + 1]] = 1.0
            term = np.kron(E, term)
        A += term
    return A
