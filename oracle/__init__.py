"""Plain FP64 CPU oracle for TNrSVD (Batselier, Yu, Daniel, Wong, arXiv 1707.07803).

TEST INFRASTRUCTURE ONLY. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may import this package. The product path (the CUDA library and its
Python binding) never imports it, and this package never imports the product path.

Every function here is a slow, direct transcription of the paper's definitions and
algorithms in NumPy float64 (LAPACK through ``numpy.linalg`` is used as a step where the
paper calls for a QR or an SVD). No blocking, fusion or reordering beyond what the paper
states. Conventions (Section 2, Eq. (2.1) "multiindex"): multi-indices are column-major,
the first index varies fastest; an MPO core ``A^(k)`` has shape ``(R_k, I_k, J_k, R_{k+1})``
and is indexed logically as ``core[r, i, j, r2]``; flattening to memory uses Fortran order
(``r`` fastest), which makes every reshape the paper performs a free view.

Modules
  mpo       dense expansion, Kronecker form (Thm 3.1), rank bounds (Thm 3.2), leading-site
            merge, MPO x MPO product (Section 5.2), MPO inner products.
  convert   sparse matrix -> MPO (Alg. 4.1) in block form, and its dense-core expansion.
  rng       SplitMix64 counter stream + Box-Muller, and the random MPO of Lemma 5.1.
  rounding  MPO-QR (Alg. 5.2) with the integrated rounding of Section 5.4, MPO-SVD (Alg. 5.3),
            and plain MPO rounding.
  tnrsvd    the randomized MPO subspace iteration (Alg. 5.4) driving Alg. 5.1, and a dense
            rSVD cross-check.
  sparse    the products of Section 5.2 applied straight from the Alg. 4.1 block form (the MPO
            has rank R at every bond, Lemma 4.2), and TNrSVD driven by them.
  gradient  the sum of the top singular values as a function of the cores, its central
            differences, and its closed-form gradient when A is exactly of rank K.

Parity status: every function is pinned by tests under ``tests/test_oracle_*.py`` except the
accuracy of TNrSVD against the true SVD for generic inputs, which the paper does not bound
(Section 5.1 remarks that the MPO test matrix is not Gaussian): "parity unpinned" for that
property only; the algorithm itself is pinned by exact-recovery and dense cross-checks.
"""

from . import mpo, convert, rng, rounding, tnrsvd  # noqa: F401
