"""The N > 1 host logic of bench.py on CPU with two gloo ranks: the timed
interval is the slowest rank's and the throughput counts every rank's
replica; the reference arm runs on rank 0 only."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(0.5 + rank, world)
    v = bench.job_throughput(1000, 10, world, t)
    out.put((rank, t, v, bench.dist_info()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, t, v, info in res:
        assert t == 1.5  # slowest rank
        assert abs(v - 2 * 1000 * 10 / 1.5 / 1e6) < 1e-15
        assert info == (rank, 2, rank)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch, capsys):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class A:
        gpus, steps, warmup = 2, 3, 3

    assert bench.run_reference(A()) == 0
    assert capsys.readouterr().out == ""


def test_ensemble_partition_balances_nodes():
    import bench

    sizes = [96 ** 3, 48 ** 3, 88 ** 3, 56 ** 3, 64 ** 3, 80 ** 3, 72 ** 3, 48 ** 3]
    owner = bench.ensemble_partition(sizes, 2)
    load = [sum(s for s, o in zip(sizes, owner) if o == r) for r in range(2)]
    assert set(owner) == {0, 1}
    assert max(load) - min(load) <= max(sizes)
    assert bench.ensemble_partition(sizes, 1) == [0] * len(sizes)
