"""GPU parity for the MPO product, MPO-QR/rounding and TNrSVD (FP64), through the C ABI."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import mpo as om
from oracle import rounding as orr
from oracle import tnrsvd as ot
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import dev_mpo, host_cores, sv_rel_err

pytestmark = pytest.mark.gpu

FP64_SV_TOL = 1e-10  # relative singular-value error gate for the FP64 path


@pytest.mark.parametrize("trans", [0, 1])
def test_contract_elementwise(trans):
    I, J = [5, 2, 3, 4], [3, 4, 2, 2]
    A = W.gaussian_mpo(1, I, J, [1, 3, 4, 2, 1])
    rows = J if trans == 0 else I
    X = W.gaussian_mpo(2, rows, [6, 1, 1, 1], [1, 2, 3, 2, 1])
    want = om.contract(A, X, trans=bool(trans))
    Y = T.tnr_mpo_contract(dev_mpo(A), trans, dev_mpo(X))
    got = host_cores(Y)
    for g, w in zip(got, want):
        assert g.shape == w.shape
        np.testing.assert_allclose(g, w, rtol=0, atol=1e-13 * max(1.0, np.abs(w).max()))


@pytest.mark.parametrize("case", ["plain", "wide_sites", "rank_deficient", "single_site", "hundred_wide"])
def test_orthogonalize_invariants_and_ranks(case):
    if case == "plain":
        Y = W.gaussian_mpo(3, [12, 3, 2, 2], [5, 1, 1, 1], [1, 4, 3, 2, 1])
    elif case == "wide_sites":
        Y = W.gaussian_mpo(4, [8, 4, 4], [6, 1, 1], [1, 9, 7, 1])
    elif case == "rank_deficient":
        Y = W.gaussian_mpo(5, [10, 2, 2, 2], [4, 1, 1, 1], [1, 6, 6, 6, 1])  # bonds above Thm 3.2 bounds
    elif case == "hundred_wide":
        # 100-wide bonds: the compression factors 4 x 100, 16 x 100 and 64 x 100 matrices (the
        # last of rank 48, cut by the pivoting), with columns spread unevenly over a cluster
        Y = W.gaussian_mpo(7, [8, 4, 4, 4], [6, 1, 1, 1], [1, 100, 100, 100, 1], scale=0.1)
    else:
        Y = W.gaussian_mpo(6, [40], [9], [1, 1])
    Qo, Ro = orr.orthogonalize(Y, tol=1e-13)
    Yd = dev_mpo(Y)
    Qd, Rd = T.tnr_orthogonalize(Yd, tol=1e-13)
    torch.cuda.synchronize()
    Q = host_cores(Qd)
    R = Rd.cpu().numpy()
    assert Qd.R == orr.ranks(Qo)
    K = Y[0].shape[2]
    DQ, DY = om.dense(Q), om.dense(Y)
    np.testing.assert_allclose(DQ.T @ DQ, np.eye(K), atol=1e-13)
    np.testing.assert_allclose(DQ @ R, DY, atol=1e-11 * np.abs(DY).max())
    # same subspace and the same R up to the signs of its rows
    DQo = om.dense(Qo)
    np.testing.assert_allclose(DQ @ DQ.T, DQo @ DQo.T, atol=1e-12)
    np.testing.assert_allclose(np.abs(R), np.abs(Ro), atol=1e-11 * np.abs(Ro).max())


def test_compression_factors_each_bond_on_a_thread_block_cluster():
    # on GB300 the cooperative launch with clusters is available: each bond's pivoted QR runs on a
    # 8-CTA cluster (distributed shared memory), not the one-CTA fallback
    Y = W.gaussian_mpo(8, [8, 4, 4, 4], [6, 1, 1, 1], [1, 100, 100, 100, 1], scale=0.1)
    Qd, Rd = T.tnr_orthogonalize(dev_mpo(Y), tol=1e-13)
    torch.cuda.synchronize()
    assert T.load().tnr_compress_cluster_size() == 8
    Qo, Ro = orr.orthogonalize(Y, tol=1e-13)
    assert Qd.R == orr.ranks(Qo)
    DQ, DY = om.dense(host_cores(Qd)), om.dense(Y)
    np.testing.assert_allclose(DQ @ Rd.cpu().numpy(), DY, atol=1e-11 * np.abs(DY).max())


def _check_solve(A, k, p, q, seed, tol, max_rank, sv_tol=FP64_SV_TOL, vec_tol=1e-8):
    Uo, So, Vo, info = ot.tnrsvd(A, k, p, q, seed, tol=tol, max_rank=max_rank, return_info=True)
    U, S, V = T.tnr_solve(dev_mpo(A), k, p, q, seed, tol=tol, max_rank=max_rank)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    err = sv_rel_err(S, So)
    assert err <= sv_tol, (err, S, So)
    assert U.R == orr.ranks(Uo) and V.R == orr.ranks(Vo)
    Uh, Vh = host_cores(U), host_cores(V)
    GU = om.inner(Uh, Uo)
    GV = om.inner(Vh, Vo)
    np.testing.assert_allclose(np.abs(np.diag(GU)), 1.0, atol=vec_tol)
    np.testing.assert_allclose(np.abs(np.diag(GV)), 1.0, atol=vec_tol)
    np.testing.assert_allclose(om.inner(Uh, Uh), np.eye(k), atol=1e-12)
    np.testing.assert_allclose(om.inner(Vh, Vh), np.eye(k), atol=1e-12)
    return S, So, err


def test_solve_small_merge_and_power_iterations():
    A = W.gaussian_mpo(0, [4, 4, 4, 4], [4, 4, 4, 4], [1, 3, 3, 3, 1], scale=1 / np.sqrt(12))
    for q in (0, 1, 2):
        _check_solve(A, 5, 5, q, seed=q, tol=1e-14, max_rank=0)


def test_solve_rectangular_and_ragged():
    A = W.gaussian_mpo(7, [6, 5, 3, 2], [4, 3, 5, 2], [1, 4, 5, 3, 1])
    _check_solve(A, 3, 4, 1, seed=11, tol=1e-14, max_rank=0)


def test_solve_single_site_after_merge():
    A = W.gaussian_mpo(8, [4, 4], [4, 4], [1, 3, 1])
    S, So, _ = _check_solve(A, 8, 8, 0, seed=0, tol=0.0, max_rank=0)
    np.testing.assert_allclose(S, np.linalg.svd(om.dense(A), compute_uv=False)[:8], rtol=1e-12)


def test_solve_exact_recovery_prescribed_sigma():
    K = 8
    sigma = 0.7 ** np.arange(K)
    A, _, _ = W.prescribed_mpo(0, 1, 16, [2, 2, 2], K, 3, sigma)
    S, So, _ = _check_solve(A, 4, 4, 1, seed=2, tol=1e-13, max_rank=0)
    np.testing.assert_allclose(S, sigma[:4], rtol=1e-12)


@pytest.mark.parametrize("K", [1, 2, 3, 7, 9, 31, 32, 33, 40])
def test_solve_kxk_svd_sizes(K):
    """The K x K SVD of the MPO-SVD at sizes around its paths: K <= 32 runs on an 8-CTA cluster
    (K < 8: CTAs without product columns; K = 31, 32: the FP32 sweeps' widest one-warp-per-pair
    case), K > 32 on one CTA with the same refinement. A of exact rank K with singular values 0.8^j
    (separated: the refinement accepts), k = K // 2, p = K - k: the singular values equal the
    oracle's and the exact ones."""
    sigma = 0.8 ** np.arange(K)
    A, _, _ = W.prescribed_mpo(K, K + 1, 16, [2, 2, 2], K, 3, sigma)
    k = max(1, K // 2)
    S, So, _ = _check_solve(A, k, K - k, 1, seed=K, tol=1e-13, max_rank=0)
    np.testing.assert_allclose(S, sigma[:k], rtol=1e-12)


def test_solve_rank_deficient_kxk_factor():
    """A of rank 10 solved with K = 16: the K x K factor has six zero singular values, so the
    refinement is skipped (FP32 noise floor) and the FP64 sweeps finish; the leading eight singular
    values are exact."""
    sigma = 0.8 ** np.arange(10)
    A, _, _ = W.prescribed_mpo(50, 51, 16, [2, 2, 2], 10, 3, sigma)
    S, So, _ = _check_solve(A, 8, 8, 1, seed=3, tol=1e-13, max_rank=0)
    np.testing.assert_allclose(S, sigma[:8], rtol=1e-12)


def test_solve_repeated_singular_values_take_the_fp64_sweeps():
    """Prescribed singular values in groups of equal values (1 x3, 0.5 x3, 0.25 x2, then distinct):
    the K x K SVD of B has equal singular values, so its product refinement declines and the FP64
    Jacobi sweeps finish it (on the cluster's first CTA). k = 8 ends at a gap, so the top-k
    subspaces are unique: the singular values match the oracle and the exact ones, and U, V span
    the oracle's subspaces (their cross Gram matrices are orthogonal)."""
    K, k = 16, 8
    sigma = np.array([1, 1, 1, 0.5, 0.5, 0.5, 0.25, 0.25] + [0.1 * 0.7**j for j in range(K - 8)])
    A, _, _ = W.prescribed_mpo(3, 4, 16, [2, 2, 2], K, 3, sigma)
    Uo, So, Vo = ot.tnrsvd(A, k, k, 1, 5, tol=1e-13)
    U, S, V = T.tnr_solve(dev_mpo(A), k, k, 1, 5, tol=1e-13)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    assert sv_rel_err(S, So) <= FP64_SV_TOL
    np.testing.assert_allclose(S, sigma[:k], rtol=1e-12)
    Uh, Vh = host_cores(U), host_cores(V)
    for X, Xo in ((Uh, Uo), (Vh, Vo)):
        np.testing.assert_allclose(om.inner(X, X), np.eye(k), atol=1e-12)
        np.testing.assert_allclose(np.linalg.svd(om.inner(X, Xo), compute_uv=False), 1.0, atol=1e-10)


def test_solve_max_rank_cap():
    A = W.gaussian_mpo(9, [4, 4, 4, 4, 4], [4, 4, 4, 4, 4], [1, 4, 4, 4, 4, 1], scale=0.25)
    _check_solve(A, 4, 4, 1, seed=3, tol=1e-14, max_rank=6)


def test_solve_c1_plain_fp64():
    """4096 x 4096 Gaussian MPO (d=6, 4x4 sites, ranks 3), k=10, p=10, q=1, seed 0."""
    c = W.c1_plain_fp64()
    S, So, err = _check_solve(c["A"], c["k"], c["p"], c["q"], c["seed"], c["tol"], c["max_rank"])
    true = np.linalg.svd(om.dense(c["A"]), compute_uv=False)[: c["k"]]
    assert np.all(S <= true * (1 + 1e-12))


def test_solve_c2_prescribed_fp64():
    """2^20 x 2^20 MPO with sigma_j = 0.7^j (rank 32), k=16, p=16, q=2: exact recovery."""
    c = W.c2_prescribed()
    S, So, err = _check_solve(c["A"], c["k"], c["p"], c["q"], c["seed"], c["tol"], c["max_rank"])
    # FP64 throughout: the prescribed values come back to a few units of rounding (every reduction
    # runs in a fixed order, so this is reproducible); a factor that is off by more than rounding
    # anywhere in the chain (e.g. a QR whose R does not match the Q it was solved with to rounding)
    # shows up here long before the 1e-10 gates
    assert sv_rel_err(S, c["sigma"][:16]) <= 3e-15


def test_rank_deficient_site1_falls_back_to_householder():
    # A of exact rank 3 with K = 8 columns: the site-1 matrices of Y = A Omega and of the later
    # products have rank 3, so their CholeskyQR2 must hand over to the Householder QR
    K = 8
    sigma = np.array([1.0, 0.5, 0.25, 0, 0, 0, 0, 0])
    A, _, _ = W.prescribed_mpo(3, 4, 16, [2, 2, 2], K, 3, sigma)
    T.stats_reset()
    U, S, V = T.tnr_solve(dev_mpo(A), 4, 4, 1, 5, tol=1e-13, max_rank=0)
    torch.cuda.synchronize()
    classes = T.stats_classes()
    householder = T.stats(classes.index("qr_small"))[0] + max(0, T.stats(classes.index("qr"))[0] - 4)
    assert householder >= 1
    S = S.cpu().numpy()
    Uo, So, Vo = ot.tnrsvd(A, 4, 4, 1, 5, tol=1e-13, max_rank=0)
    assert sv_rel_err(S, So) <= FP64_SV_TOL
    np.testing.assert_allclose(S[:3], sigma[:3], rtol=1e-12)
    # the rank-3 part of the singular vectors (the rest spans an arbitrary null direction)
    Uh, Vh = host_cores(U), host_cores(V)
    np.testing.assert_allclose(np.abs(np.diag(om.inner(Uh, Uo)))[:3], 1.0, atol=1e-9)
    np.testing.assert_allclose(np.abs(np.diag(om.inner(Vh, Vo)))[:3], 1.0, atol=1e-9)


def test_wide_bonds_continue_on_the_host_path():
    # product bonds wider than the one-CTA pivoted QR takes (w > 64): the cooperative compression
    # hands the rest of the sweep to the host-driven kernels, and the rounding runs per bond
    A = W.gaussian_mpo(12, [4] * 6, [4] * 6, [1, 8, 8, 8, 8, 8, 1], scale=lambda k, sh: 1.0 / np.sqrt(sh[1] * sh[0]))
    _check_solve(A, 8, 8, 1, seed=7, tol=1e-13, max_rank=16)


def test_bounded_wait_reports_timeout_and_the_context_stays_usable():
    # a grid-barrier wait that nothing satisfies gives up after its poll cap with TNR_ETIMEOUT
    lib = T.load()
    assert lib.tnr_selftest_wait_timeout(1000, T._stream()) == -7
    assert lib.tnr_selftest_wait_timeout(0, T._stream()) == -1
    # the status word is clear again and the next solve is unaffected
    A = W.gaussian_mpo(4, [4, 4, 4, 4], [4, 4, 4, 4], [1, 3, 3, 3, 1], scale=1 / np.sqrt(12))
    _check_solve(A, 4, 4, 1, seed=2, tol=1e-14, max_rank=0)


def test_float32_input_cores_are_widened_exactly():
    # TNR_F32 cores: the solve widens them to float64 on the device, so it equals the solve of the
    # same values held in float64, bit for bit
    A = W.gaussian_mpo(5, [4] * 5, [4] * 5, [1, 4, 4, 4, 4, 1], scale=0.25)
    A32 = [c.astype(np.float32) for c in A]
    for precision in (T.TNR_FP64, T.TNR_MIXED):
        U1, S1, V1 = T.tnr_solve(T.Mpo.from_numpy(A32, dtype=np.float32), 4, 4, 1, 3, tol=1e-13, precision=precision)
        U2, S2, V2 = T.tnr_solve(T.Mpo.from_numpy([c.astype(np.float64) for c in A32]), 4, 4, 1, 3, tol=1e-13,
                                 precision=precision)
        torch.cuda.synchronize()
        assert torch.equal(S1, S2)
        assert all(np.array_equal(a, b) for a, b in zip(host_cores(U1), host_cores(U2)))
    # the persistent batch reads float64 cores only
    pr = dict(A=T.Mpo.from_numpy(A32, dtype=np.float32), k=4, p=4, q=1, seed=3, tol=1e-13, max_rank=8)
    with pytest.raises(T.TnrError):
        T.PersistentBatch([pr], precision=T.TNR_FP64)


def test_run_host_moves_inputs_and_outputs_in_one_copy_each():
    """SolvePlan.run_host: the operator built with flat=True, its host image (Mpo.host_flat) copied
    in one transfer, the outputs (S, then U's and V's cores at their capacities) copied back in one:
    the host copy equals the device outputs of a plain run and S equals the oracle's."""
    A = W.gaussian_mpo(0, [4] * 4, [4] * 4, [1, 3, 3, 3, 1], scale=1 / np.sqrt(12))
    k, p, q, seed = 5, 5, 1, 4
    plan = T.SolvePlan(T.Mpo.from_numpy(A, flat=True), k, p, tol=1e-14)
    assert plan.A.flat is not None and all(c.data_ptr() >= plan.A.flat.data_ptr() for c in plan.A.cores)
    host_in = T.Mpo.host_flat(A)
    host_out = torch.empty(plan.out_flat.numel(), dtype=torch.float64).pin_memory()
    plan.A.flat.zero_()  # the operator must come from host_in
    plan.run_host(host_in, host_out, q, seed)
    torch.cuda.synchronize()
    assert np.array_equal(host_out.numpy(), plan.out_flat.cpu().numpy())
    _, So, _ = ot.tnrsvd(A, k, p, q, seed, tol=1e-14)
    assert sv_rel_err(host_out[:k].numpy(), So) <= FP64_SV_TOL
    ref = T.SolvePlan(T.Mpo.from_numpy(A), k, p, tol=1e-14).run(q, seed)
    torch.cuda.synchronize()
    assert np.array_equal(ref.S.cpu().numpy(), host_out[:k].numpy())
    with pytest.raises(ValueError):
        plan.run_host(host_in[:-1], host_out, q, seed)
