"""Persistent batched TNrSVD (tnr_batch_*): one kernel launch, one CTA per problem, problems
taken from a device work queue. Every problem of a batch of uneven MPOs (d, physical dims,
ranks, k) gives the oracle's singular values and ranks, orthonormal U and V with U^T A V =
diag(S); results do not depend on where the factorisations' work areas live (shared memory or
global scratch: bit-identical); graph replays reproduce the first launch bit for bit; bad
problems are refused at planning; output capacities are checked per problem."""

import ctypes

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

FP64_SV_TOL = 1e-10
# Mixed precision: the persistent batch's products use FP32 operands (about 2^-24 relative per
# term) and its power iteration is rounded at max(tol, 1e-6); the relative singular-value error
# against the FP64 oracle is held to the mixed-mode gate, 1e-6.
MIXED_SV_TOL = 1e-6


def _problems(seed, n, precision, d_range=(4, 7), rank_range=(2, 5), ks=(2, 4), q=1, tol=1e-13):
    probs = W.batched_gaussian(seed, n, d_range=d_range, phys=(2, 4), rank_range=rank_range, ks=ks, q=q, tol=tol)
    return [dict(pr, A=dev_mpo(pr["A"]), A_host=pr["A"], precision=precision) for pr in probs]


def _host(pb, i):
    U, S, V = pb.outputs(i)
    return host_cores(U), S.cpu().numpy().copy(), host_cores(V)


def _check_against_oracle(pr, Uh, S, Vh, sv_tol, check_ranks):
    Uo, So, Vo = ot.tnrsvd(pr["A_host"], pr["k"], pr["p"], pr["q"], pr["seed"], tol=pr["tol"],
                           max_rank=pr["max_rank"])
    err = sv_rel_err(S, So)
    assert err <= sv_tol, (err, S, So)
    if check_ranks:
        assert orr.ranks(Uh) == orr.ranks(Uo) and orr.ranks(Vh) == orr.ranks(Vo)
    k = pr["k"]
    np.testing.assert_allclose(om.inner(Uh, Uh), np.eye(k), atol=1e-12)
    np.testing.assert_allclose(om.inner(Vh, Vh), np.eye(k), atol=1e-12)
    # U^T A V = diag(S): B = Q^T A is exact and W, V come from its SVD (merged operator sites)
    m = om.merge_count(*om.dims(pr["A_host"])[:2], k + pr["p"])
    Am = om.merge_leading(pr["A_host"], m) if m > 1 else pr["A_host"]
    G = om.sandwich(Uh, Am, Vh)
    np.testing.assert_allclose(G, np.diag(S), atol=1e-9 * S[0])


@pytest.mark.parametrize("precision", [T.TNR_FP64, T.TNR_MIXED])
def test_persistent_batch_matches_oracle(precision):
    probs = _problems(31, 12, precision)
    pb = T.PersistentBatch(probs, precision=precision)
    pb.launch()
    assert pb.collect() == 0
    assert pb.statuses() == [0] * len(probs)
    cfg = pb.config()
    assert 1 <= cfg["ctas_per_sm"] <= 4 and 1 <= cfg["grid"] <= len(probs) and cfg["smem_bytes"] >= 16384
    tol = FP64_SV_TOL if precision == T.TNR_FP64 else MIXED_SV_TOL
    for i, pr in enumerate(probs):
        Uh, S, Vh = _host(pb, i)
        _check_against_oracle(pr, Uh, S, Vh, tol, check_ranks=precision == T.TNR_FP64)
    pb.close()


def test_persistent_matches_single_solves_fp64():
    probs = _problems(44, 8, T.TNR_FP64, rank_range=(3, 6), ks=(4,), q=2)
    pb = T.PersistentBatch(probs, precision=T.TNR_FP64, autotune=False, graph=False)
    pb.launch()
    pb.collect()
    for i, pr in enumerate(probs):
        _, S_b, _ = pb.outputs(i)
        _, S_1, _ = T.tnr_solve(pr["A"], pr["k"], pr["p"], pr["q"], pr["seed"], tol=pr["tol"],
                                max_rank=pr["max_rank"], precision=T.TNR_FP64)
        assert sv_rel_err(S_b.cpu().numpy(), S_1.cpu().numpy()) <= 1e-12
    pb.close()


def test_work_areas_in_shared_or_global_memory_are_bit_identical():
    # ranks up to 10 with K = 16: some factorisations fit shared memory only at one CTA per SM
    probs = _problems(52, 6, T.TNR_FP64, d_range=(5, 6), rank_range=(6, 10), ks=(8,), q=1)
    outs = []
    for per_sm in (1, 2):
        pb = T.PersistentBatch(probs, precision=T.TNR_FP64, autotune=False, graph=False, ctas_per_sm=per_sm)
        cfg = pb.config()
        pb.launch()
        assert pb.collect() == 0
        outs.append((cfg, [_host(pb, i) for i in range(len(probs))]))
        pb.close()
    (c1, o1), (c2, o2) = outs
    assert c1["smem_bytes"] > c2["smem_bytes"]
    for (U1, S1, V1), (U2, S2, V2) in zip(o1, o2):
        assert np.array_equal(S1, S2)
        assert all(np.array_equal(a, b) for a, b in zip(U1, U2))
        assert all(np.array_equal(a, b) for a, b in zip(V1, V2))
    for pr, (Uh, S, Vh) in zip(probs, o1):
        _check_against_oracle(pr, Uh, S, Vh, FP64_SV_TOL, check_ranks=True)


def test_graph_replay_is_bit_identical():
    probs = _problems(61, 10, T.TNR_MIXED)
    pb = T.PersistentBatch(probs, precision=T.TNR_MIXED, autotune=True, graph=True)
    pb.launch()
    assert pb.collect() == 0
    first = [_host(pb, i) for i in range(len(probs))]
    for _ in range(3):
        pb.launch()
    assert pb.collect() == 0
    again = [_host(pb, i) for i in range(len(probs))]
    for (U1, S1, V1), (U2, S2, V2) in zip(first, again):
        assert np.array_equal(S1, S2)
        assert all(np.array_equal(a, b) for a, b in zip(U1, U2))
        assert all(np.array_equal(a, b) for a, b in zip(V1, V2))
    pb.close()


def test_edge_cases_single_site_no_power_iteration_no_tolerance_rank_cap():
    cases = []
    # every site merged into one (K = 16 needs both 4 x 4 sites): d = 1 after the merge
    A1 = W.gaussian_mpo(1, [4, 4], [4, 4], [1, 3, 1], scale=0.3)
    cases.append(dict(A=A1, k=8, p=8, q=1, seed=3, tol=1e-13, max_rank=0))
    # q = 0 and tol = 0 (no compression, no certificate)
    A2 = W.gaussian_mpo(2, [2] * 6, [2] * 6, [1, 3, 4, 2, 3, 2, 1], scale=0.5)
    cases.append(dict(A=A2, k=2, p=2, q=0, seed=4, tol=0.0, max_rank=0))
    # a binding rank cap
    A3 = W.gaussian_mpo(3, [4] * 5, [4] * 5, [1, 5, 5, 5, 5, 1], scale=0.25)
    cases.append(dict(A=A3, k=4, p=4, q=1, seed=5, tol=1e-13, max_rank=3))
    # rectangular operator (I != J)
    A4 = W.gaussian_mpo(4, [4, 2, 2, 4], [2, 4, 4, 2], [1, 2, 3, 2, 1], scale=0.4)
    cases.append(dict(A=A4, k=3, p=3, q=2, seed=6, tol=1e-13, max_rank=0))
    probs = [dict(c, A=dev_mpo(c["A"]), A_host=c["A"], precision=T.TNR_FP64) for c in cases]
    pb = T.PersistentBatch(probs, precision=T.TNR_FP64, autotune=False, graph=True)
    pb.launch()
    assert pb.collect() == 0
    for i, pr in enumerate(probs):
        Uh, S, Vh = _host(pb, i)
        _check_against_oracle(pr, Uh, S, Vh, FP64_SV_TOL, check_ranks=True)
    pb.close()


def test_bad_problem_refused_and_capacity_checked_per_problem():
    probs = _problems(71, 4, T.TNR_FP64)
    lib = T.load()
    plans, arr, _ = T._batch_outputs(probs, T.TNR_FP64)
    arr[1].k = 1 << 20  # K = k + p > prod I: refused at planning, nothing launched
    b = ctypes.c_size_t(0)
    assert lib.tnr_batch_workspace(len(probs), arr, ctypes.byref(b)) == -1
    h = ctypes.c_void_p(0)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    assert lib.tnr_batch_create(len(probs), arr, 0, T._ptr(ws), ws.numel(), T._stream(), ctypes.byref(h)) == -1
    assert not h.value
    assert lib.tnr_batch_create(len(probs), arr, 1 << 12, T._ptr(ws), ws.numel(), T._stream(), ctypes.byref(h)) == -1
    # an output capacity too small fails that problem alone, on the device
    plans, arr, _ = T._batch_outputs(probs, T.TNR_FP64)
    plans[2][0].us.cap[0] = 1
    assert lib.tnr_batch_workspace(len(probs), arr, ctypes.byref(b)) == 0
    ws = torch.empty(b.value, dtype=torch.uint8, device="cuda")
    assert lib.tnr_batch_create(len(probs), arr, 0, T._ptr(ws), b.value, T._stream(), ctypes.byref(h)) == 0
    assert lib.tnr_batch_launch(h, T._stream()) == 0
    assert lib.tnr_batch_collect(h, T._stream()) == -5
    st = [arr[i].status for i in range(len(probs))]
    assert st[2] == -5 and [s for j, s in enumerate(st) if j != 2] == [0, 0, 0]
    for j, pr in enumerate(probs):
        if j == 2:
            continue
        sp = plans[j][0]
        _check_against_oracle(pr, host_cores(sp.outputs()[0]), sp.S.cpu().numpy(), host_cores(sp.outputs()[2]),
                              FP64_SV_TOL, check_ranks=True)
    assert lib.tnr_batch_destroy(h) == 0


def test_mixed_batch_on_decaying_spectra_where_the_rounding_truncates():
    """Prescribed-sigma problems (sigma_j = 0.5^j, 16 values, K = 8 < 16): the power iteration's
    rounding at max(tol, 1e-6) truncates real directions; the mixed batch (FP32 products) still
    matches the FP64 oracle within the mixed-mode gate 1e-6, and the FP64 batch within 1e-10."""
    probs = []
    for i in range(6):
        sigma = 0.5 ** np.arange(16) * (1 + 0.1 * i)
        A, _, _ = W.prescribed_mpo(10 + i, 20 + i, 16, [2, 2, 2, 2, 2], 16, 3, sigma)
        probs.append(dict(A=A, k=4, p=4, q=1, seed=i, tol=1e-12, max_rank=8))
    for precision, gate in ((T.TNR_FP64, FP64_SV_TOL), (T.TNR_MIXED, MIXED_SV_TOL)):
        dp = [dict(pr, A=dev_mpo(pr["A"]), A_host=pr["A"], precision=precision) for pr in probs]
        pb = T.PersistentBatch(dp, precision=precision, autotune=False, graph=False)
        pb.launch()
        assert pb.collect() == 0
        for i, pr in enumerate(dp):
            _, S, _ = pb.outputs(i)
            _, So, _ = ot.tnrsvd(pr["A_host"], pr["k"], pr["p"], pr["q"], pr["seed"], tol=pr["tol"],
                                 max_rank=pr["max_rank"])
            assert sv_rel_err(S.cpu().numpy(), So) <= gate
        pb.close()
