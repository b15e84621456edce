"""The multi-GPU path of bench.py is replicas only (a single TNrSVD does not shard): every rank solves
its own copy of the workload and the job rate is all ranks' steps over the slowest rank's time.
Checked here with two gloo ranks on the CPU (no GPU): the MAX reduction, the aggregate rate, and the
reference arm's rank-0-only rule."""

import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    # rank r took 100 (r + 1) ms for its 10 steps
    rate, max_ms = bench.replicas_rate(100.0 * (rank + 1), 10, world, "cpu", dist)
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, rate, max_ms))


def test_replica_rate_is_bounded_by_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for _, rate, max_ms in out:
        assert max_ms == pytest.approx(200.0)
        assert rate == pytest.approx(2 * 10 / 0.2)  # 20 steps over 0.2 s


def test_single_rank_rate_and_reference_arm_rank_rule(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    rate, max_ms = bench.replicas_rate(50.0, 5, 1, "cpu")
    assert (rate, max_ms) == (pytest.approx(100.0), pytest.approx(50.0))

    class Args:
        steps, warmup = 1, 0

    monkeypatch.setenv("RANK", "1")
    assert bench.reference_arm(Args()) == 0  # ranks other than 0 do no work and print nothing
    assert capsys.readouterr().out == ""
