"""Writes c5_fd_gradient.txt: the oracle's FP64 central-difference gradient of the differentiable
workload (calls only oracle/ and workloads/; never the CUDA path).

Workload: a 4^12 x 4^12 MPO, d = 12, I = J = 4, interior ranks 16, Gaussian cores (seed 0) scaled by
1/sqrt(I R) and rounded to float32 values; k = 16, p = 16, q = 2, Omega seed 3, fixed ranks
(tol = 0, max_rank = K = 32); loss L = sum of the 16 singular values TNrSVD returns (Alg. 5.4 with
Alg. 5.3, the rounding of Section 5.4). 64 core entries drawn uniformly over all cores (seed 1),
each differentiated by (L(A + h e) - L(A - h e)) / (2 h) with h = 1e-6 on float64 copies.

Run: python tests/golden/make_c5_fd.py [--workers N]   (about 128 oracle forwards of ~10 s each)
"""

import argparse
import multiprocessing as mp
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "c5_fd_gradient.txt")

D, RANK, K_OUT, P_OVER, Q_PI, SEED, N_SV, H, N_ENTRIES = 12, 16, 16, 16, 2, 3, 16, 1e-6, 64


def workload():
    sys.path.insert(0, ROOT)
    import workloads as W

    A = W.gaussian_mpo(0, [4] * D, [4] * D, [1] + [RANK] * (D - 1) + [1],
                       scale=lambda kk, sh: 1.0 / np.sqrt(sh[1] * sh[0]))
    return [c.astype(np.float32).astype(np.float64) for c in A]


def entries(A):
    """64 (core, flat Fortran-order index) pairs, uniform over all core entries."""
    sizes = np.array([c.size for c in A])
    rng = np.random.default_rng(1)
    flat = rng.choice(int(sizes.sum()), size=N_ENTRIES, replace=False)
    starts = np.concatenate([[0], np.cumsum(sizes)])
    out = []
    for f in sorted(int(x) for x in flat):
        c = int(np.searchsorted(starts, f, side="right") - 1)
        out.append((c, f - int(starts[c])))
    return out


def _one(args):
    sys.path.insert(0, ROOT)
    from oracle import gradient as og

    A, ent = args
    return float(og.fd_gradient(A, K_OUT, P_OVER, Q_PI, SEED, N_SV, [ent], h=H, max_rank=K_OUT + P_OVER)[0])


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workers", type=int, default=4)
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    from oracle import tnrsvd as ot

    A = workload()
    ent = entries(A)
    _, S, _ = ot.tnrsvd(A, K_OUT, P_OVER, Q_PI, SEED, tol=0.0, max_rank=K_OUT + P_OVER)
    with mp.get_context("spawn").Pool(args.workers) as pool:
        g = pool.map(_one, [(A, e) for e in ent])
    with open(OUT, "w") as f:
        f.write("# Oracle FP64 central differences (h = 1e-6) of L = sum of the 16 TNrSVD singular values\n")
        f.write("# (Alg. 5.4 with Alg. 5.3 and the rounding of Section 5.4; fixed ranks tol = 0, max_rank = 32)\n")
        f.write("# for the d = 12 differentiable workload; written by tests/golden/make_c5_fd.py (oracle only).\n")
        f.write("# S " + " ".join(f"{v:.17e}" for v in S) + "\n")
        f.write("# core flat_index dL/de\n")
        for (c, e), v in zip(ent, g):
            f.write(f"{c} {e} {v:.17e}\n")


if __name__ == "__main__":
    main()
