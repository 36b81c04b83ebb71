"""Replica plumbing of bench.py on CPU: two gloo ranks, slowest rank bounds the job."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    local_ms = [100.0, 250.0][rank]
    value, total = bench.replica_rate(local_ms, 64, 10, world, dist, "cpu")
    q.put((rank, value, total))
    dist.barrier()
    dist.destroy_process_group()


def test_replica_rate_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, value, total in got:
        assert total == 250.0                       # max over ranks
        assert abs(value - 2 * 64 * 10 / 0.25) < 1e-9  # both replicas' work / slowest time


def test_reference_arm_nonzero_rank_exits_quietly(capsys, monkeypatch):
    import bench
    monkeypatch.setenv("RANK", "1")
    class A:
        gpus, steps, warmup = 2, 1, 0
    bench.run_reference(A())
    assert capsys.readouterr().out == ""
