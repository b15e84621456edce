"""Batched TNrSVD (tnr_solve_batched) through the C ABI: every problem of a batch of uneven
MPOs (d, physical dims, ranks, k) gives the same singular values as its own tnr_solve and as the
oracle; a bad problem fails alone; worker counts from 1 to more than the batch."""

import numpy as np
import pytest
import torch

import workloads as W
from oracle import tnrsvd as ot
from paper_1707_07803_gb300 import tnrsvd as T
from tests.gpu_util import dev_mpo, sv_rel_err

pytestmark = pytest.mark.gpu

FP64_SV_TOL = 1e-10
# Mixed precision (the single solve's kernels: BF16 x3 products, about 2^-16 relative per term,
# FP32 accumulation; power iteration rounded at max(tol, 1.2e-4)): held to the mixed-mode gate of
# 1e-6 relative singular-value error against the FP64 oracle.
MIXED_SV_TOL = 1e-6


def _problems(seed, n, precision):
    probs = W.batched_gaussian(seed, n, d_range=(4, 7), phys=(2, 4), rank_range=(2, 5), ks=(2, 4), q=1,
                               tol=1e-13)
    return [dict(pr, A=dev_mpo(pr["A"]), A_host=pr["A"], precision=precision) for pr in probs]


@pytest.mark.parametrize("precision,workers", [(T.TNR_FP64, 4), (T.TNR_MIXED, 3), (T.TNR_FP64, 1),
                                               (T.TNR_MIXED, 16)])
def test_batch_matches_single_solves_and_oracle(precision, workers):
    probs = _problems(5 + workers, 9, precision)
    plan = T.BatchPlan(probs, workers=workers, precision=precision)
    plan.run()
    torch.cuda.synchronize()
    assert plan.statuses() == [0] * len(probs)
    tol = FP64_SV_TOL if precision == T.TNR_FP64 else MIXED_SV_TOL
    for i, pr in enumerate(probs):
        _, S_b, _ = plan.outputs(i)
        S_b = S_b.cpu().numpy()
        _, S_1, _ = T.tnr_solve(pr["A"], pr["k"], pr["p"], pr["q"], pr["seed"], tol=pr["tol"],
                                max_rank=pr["max_rank"], precision=precision)
        S_1 = S_1.cpu().numpy()
        # same kernels on the same inputs: equal up to the summation order of split-K GEMMs
        same_tol = 1e-13 if precision == T.TNR_FP64 else 1e-9
        assert sv_rel_err(S_b, S_1) <= same_tol, (i, sv_rel_err(S_b, S_1))
        _, S_o, _ = ot.tnrsvd(pr["A_host"], pr["k"], pr["p"], pr["q"], pr["seed"], tol=pr["tol"],
                              max_rank=pr["max_rank"])
        assert sv_rel_err(S_b, S_o) <= tol, (i, sv_rel_err(S_b, S_o))


def test_bad_problem_fails_alone():
    probs = _problems(21, 5, T.TNR_FP64)
    plan = T.BatchPlan(probs, workers=2, precision=T.TNR_FP64)
    plan.probs[2].k = 1 << 20  # K = k + p > prod I: rejected by that solve's own checks
    rc = plan.run(check=False)
    torch.cuda.synchronize()
    assert rc == -1
    st = plan.statuses()
    assert st[2] == -1 and [s for j, s in enumerate(st) if j != 2] == [0, 0, 0, 0]
    for j, pr in enumerate(probs):
        if j == 2:
            continue
        _, S_o, _ = ot.tnrsvd(pr["A_host"], pr["k"], pr["p"], pr["q"], pr["seed"], tol=pr["tol"],
                              max_rank=pr["max_rank"])
        assert sv_rel_err(plan.outputs(j)[1].cpu().numpy(), S_o) <= FP64_SV_TOL


def test_empty_batch_and_argument_checks():
    lib = T.load()
    ws = torch.empty(256, dtype=torch.uint8, device="cuda")
    assert lib.tnr_solve_batched(0, None, 0, T._ptr(ws), 256, T._stream()) == 0
    probs = _problems(3, 2, T.TNR_FP64)
    plan = T.BatchPlan(probs, workers=2, precision=T.TNR_FP64)
    assert lib.tnr_solve_batched(2, plan.probs, 64, T._ptr(plan.ws), plan.ws_stride, T._stream()) == -1
    assert lib.tnr_solve_batched(2, plan.probs, 2, T._ptr(plan.ws), plan.ws_stride + 8, T._stream()) == -1
    assert plan.run() == 0
