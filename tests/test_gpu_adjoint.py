"""Adjoint of TNrSVD (tnr_diff_forward / tnr_diff_backward) through the C ABI and the
torch.autograd.Function: the fixed-rank forward matches the oracle's singular values, and the
gradient of L = sum of the leading singular values matches the oracle's central-difference
gradient (FP64, h = 1e-6) and, where the randomized SVD is exact, the closed form U_n V_n^T."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import gradient as og
from oracle import tnrsvd as ot
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import dev_mpo, sv_rel_err

pytestmark = pytest.mark.gpu

GRAD_TOL = 1e-6  # normwise relative error of the sampled gradient entries


def _entries(A, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        c = int(rng.integers(0, len(A)))
        out.append((c, int(rng.integers(0, A[c].size))))
    return out


def _gpu_grad(A_host, k, p, q, seed, n_sv):
    A = dev_mpo(A_host)
    for c in A.cores:
        c.requires_grad_(True)
    S = T.tnrsvd_values(A, k, p, q, seed)
    S[:n_sv].sum().backward()
    torch.cuda.synchronize()
    return S.detach().cpu().numpy(), [c.grad.cpu().numpy() for c in A.cores]


def _pick(grads, entries):
    return np.array([grads[c][e] for c, e in entries])


@pytest.mark.parametrize("case", ["plain", "merge", "power_iterations"])
def test_adjoint_matches_oracle_fd(case):
    if case == "plain":
        A, k, p, q, n_sv = W.gaussian_mpo(3, [6, 3, 2, 2], [5, 4, 2, 2], [1, 3, 4, 2, 1]), 2, 2, 1, 2
    elif case == "merge":  # K = 8 needs the first three 2 x 2 sites merged
        A, k, p, q, n_sv = W.gaussian_mpo(4, [2] * 6, [2] * 6, [1, 2, 3, 3, 2, 2, 1]), 4, 4, 1, 3
    else:
        A, k, p, q, n_sv = W.gaussian_mpo(5, [4, 4, 4], [4, 4, 4], [1, 3, 3, 1]), 3, 3, 2, 3
    seed = 11
    S_gpu, grads = _gpu_grad(A, k, p, q, seed, n_sv)
    K = k + p
    _, S_o, _ = ot.tnrsvd(A, k, p, q, seed, tol=0.0, max_rank=K)
    assert sv_rel_err(S_gpu, S_o) <= 1e-10
    ent = _entries(A, 16, 7)
    fd = og.fd_gradient(A, k, p, q, seed, n_sv, ent)
    got = _pick(grads, ent)
    assert np.linalg.norm(got - fd) <= GRAD_TOL * np.linalg.norm(fd), (got, fd)


def test_adjoint_closed_form_when_exact():
    A, _, _ = W.prescribed_mpo(0, 1, 16, [2, 2, 2], 8, 3, 0.7 ** np.arange(8))
    S_gpu, grads = _gpu_grad(A, 4, 4, 1, 7, 3)
    np.testing.assert_allclose(S_gpu[:4], 0.7 ** np.arange(4), rtol=1e-12)
    ent = _entries(A, 16, 3)
    cf = og.closed_form_exact(A, 3, ent)
    got = _pick(grads, ent)
    assert np.linalg.norm(got - cf) <= GRAD_TOL * np.linalg.norm(cf)


def test_backward_twice_and_free():
    A_host = W.gaussian_mpo(3, [6, 3, 2, 2], [5, 4, 2, 2], [1, 3, 4, 2, 1])
    A = dev_mpo(A_host)
    for c in A.cores:
        c.requires_grad_(True)
    S = T.tnrsvd_values(A, 2, 2, 1, 11)
    g1 = torch.autograd.grad(S.sum(), A.cores, retain_graph=True)
    g2 = torch.autograd.grad(S.sum(), A.cores)
    for a, b in zip(g1, g2):
        assert torch.equal(a, b)


def test_float32_cores_give_the_float64_values_and_rounded_gradients():
    # FP32 Gaussian cores (the shape of the differentiable workload): the forward widens them
    # exactly, so S equals the float64 run's; the gradients are the float64 ones rounded to float32
    A_host = [c.astype(np.float32) for c in W.gaussian_mpo(8, [4] * 4, [4] * 4, [1, 3, 3, 3, 1], scale=0.3)]
    A32 = T.Mpo.from_numpy(A_host, dtype=np.float32)
    A64 = T.Mpo.from_numpy([c.astype(np.float64) for c in A_host])
    for A in (A32, A64):
        for c in A.cores:
            c.requires_grad_(True)
    S32 = T.tnrsvd_values(A32, 4, 4, 1, 5)
    S64 = T.tnrsvd_values(A64, 4, 4, 1, 5)
    assert torch.equal(S32, S64)
    g32 = torch.autograd.grad(S32.sum(), A32.cores)
    g64 = torch.autograd.grad(S64.sum(), A64.cores)
    for a, b in zip(g32, g64):
        assert a.dtype == torch.float32
        torch.testing.assert_close(a, b.to(torch.float32), rtol=1e-6, atol=1e-30)


def _c5_golden():
    """The d = 12 differentiable workload and the oracle's stored central differences (written by
    tests/golden/make_c5_fd.py, which calls only the oracle)."""
    import importlib.util

    from tests.conftest import golden_path

    spec = importlib.util.spec_from_file_location("make_c5_fd", golden_path("make_c5_fd.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    S, ent, fd = None, [], []
    for line in open(golden_path("c5_fd_gradient.txt")):
        if line.startswith("# S "):
            S = np.array([float(x) for x in line.split()[2:]])
        elif not line.startswith("#") and line.strip():
            c, e, g = line.split()
            ent.append((int(c), int(e)))
            fd.append(float(g))
    return mk, mk.workload(), S, ent, np.array(fd)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_full_size_gradient_matches_oracle_central_differences(dtype):
    """d = 12, 4 x 4 sites, rank 16, k = p = 16, q = 2 (512-wide product bonds): the forward's
    singular values equal the oracle's (1e-10) and the adjoint's gradient on the 64 stored entries
    equals the oracle's FP64 central differences (h = 1e-6) to 1e-6 normwise; float32 cores (their
    values are float32 numbers) give the same within the float32 rounding of the gradient."""
    mk, A_host, S_ref, ent, fd = _c5_golden()
    A = T.Mpo.from_numpy(A_host, dtype=dtype)
    for c in A.cores:
        c.requires_grad_(True)
    S = T.tnrsvd_values(A, mk.K_OUT, mk.P_OVER, mk.Q_PI, mk.SEED)
    S[: mk.N_SV].sum().backward()
    torch.cuda.synchronize()
    assert sv_rel_err(S.detach().cpu().numpy(), S_ref) <= 1e-10
    grads = [c.grad.double().cpu().numpy() for c in A.cores]
    got = _pick(grads, ent)
    assert np.linalg.norm(got - fd) <= GRAD_TOL * np.linalg.norm(fd), np.linalg.norm(got - fd) / np.linalg.norm(fd)
