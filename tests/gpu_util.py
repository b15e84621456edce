"""Helpers for the GPU parity tests (marshalling between numpy oracle data and the CUDA path)."""

import numpy as np
import torch

from paper_1707_07803_gb300 import tnrsvd as T


def dev_mpo(cores):
    return T.Mpo.from_numpy(cores)


def host_cores(m):
    return m.to_numpy()


def sv_rel_err(S, S_ref):
    S = np.asarray(S, dtype=np.float64)
    S_ref = np.asarray(S_ref, dtype=np.float64)
    return float(np.linalg.norm(S - S_ref) / np.linalg.norm(S_ref))


def coo_to_device(rows, cols, vals):
    return (torch.from_numpy(np.ascontiguousarray(rows, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(cols, dtype=np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float64)).cuda())
