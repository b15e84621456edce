"""The batch split over GPUs (paper_1707_07803_gb300.shard): greedy LPT on estimated work, every
problem assigned exactly once, makespan within the list-scheduling bound (and within 4/3 of the
optimum found by brute force on a small instance), and results gathered on rank 0 in the batch's
order. The gather runs on two gloo ranks on the CPU (no GPU)."""

import itertools
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1707_07803_gb300 import shard  # noqa: E402
import workloads as W  # noqa: E402


def _stated_costs(n=256):
    probs = W.batched_gaussian(0, n, d_range=(8, 20), phys=(2, 4), rank_range=(4, 32), ks=(8, 16, 32))
    out = []
    for pr in probs:
        I = [c.shape[1] for c in pr["A"]]
        J = [c.shape[2] for c in pr["A"]]
        R = [pr["A"][0].shape[0]] + [c.shape[3] for c in pr["A"]]
        out.append(shard.problem_cost(I, J, R, pr["k"], pr["p"], pr["q"], pr["max_rank"]))
    return out


@pytest.mark.parametrize("ranks", [1, 2, 3, 8])
def test_lpt_assigns_every_problem_once_within_the_list_bound(ranks):
    costs = _stated_costs()
    parts, loads = shard.lpt_partition(costs, ranks)
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(costs)))
    for p, load in zip(parts, loads):
        assert load == pytest.approx(sum(costs[i] for i in p))
    lower = max(sum(costs) / ranks, max(costs))  # no schedule beats this
    assert max(loads) <= sum(costs) / ranks + max(costs) * (1 - 1 / ranks) + 1e-6 * lower


def test_lpt_within_four_thirds_of_brute_force_optimum():
    rng = np.random.default_rng(4)
    for trial in range(20):
        costs = list(rng.integers(1, 50, size=9).astype(float))
        for m in (2, 3):
            _, loads = shard.lpt_partition(costs, m)
            best = min(max(sum(c for c, a in zip(costs, assign) if a == r) for r in range(m))
                       for assign in itertools.product(range(m), repeat=len(costs)))
            assert max(loads) <= (4 / 3 - 1 / (3 * m)) * best + 1e-9


def test_cost_grows_with_rank_and_k():
    base = shard.problem_cost([4] * 10, [4] * 10, [1] + [8] * 9 + [1], 8, 8, 1)
    assert shard.problem_cost([4] * 10, [4] * 10, [1] + [16] * 9 + [1], 8, 8, 1) > base
    assert shard.problem_cost([4] * 10, [4] * 10, [1] + [8] * 9 + [1], 16, 16, 1) > base
    assert shard.problem_cost([4] * 10, [4] * 10, [1] + [8] * 9 + [1], 8, 8, 2) > base


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1707_07803_gb300 import shard as sh

    costs = [float(c) for c in range(1, 23)]
    parts, _ = sh.lpt_partition(costs, world)
    # each rank "solves" its problems: result of problem i is (i, [i, i^2])
    local = [(i, [float(i), float(i * i)]) for i in parts[rank]]
    got = sh.gather_in_order(local, parts, rank, world, dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, parts, got))


def test_gather_on_two_gloo_ranks_restores_batch_order():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, parts0, got0), (r1, parts1, got1) = out
    assert parts0 == parts1  # both ranks computed the same split
    assert set(parts0[0]).isdisjoint(parts0[1]) and parts0[0] and parts0[1]
    assert got1 is None
    assert [g[0] for g in got0] == list(range(22))
    assert all(g[1] == [float(i), float(i * i)] for i, g in enumerate(got0))
