"""GB300 (sm_103a) implementation of TNrSVD and sparse -> MPO conversion (arXiv 1707.07803).

The compute path is libtnrsvd.so (hand-written CUDA kernels behind a C ABI, include/tnrsvd.h);
``tnrsvd`` is its thin ctypes binding. Build with ``paper_1707_07803_gb300.build.build()``.
"""

from . import tnrsvd  # noqa: F401
from .tnrsvd import Mpo, SolvePlan, sparse_to_mpo, tnr_mpo_contract, tnr_orthogonalize, tnr_solve  # noqa: F401
