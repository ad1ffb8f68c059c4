"""The N > 1 host logic of bench.py on CPU with two gloo ranks: the timed
interval is the slowest rank's and the throughput counts every rank's
replica; the reference arm runs on rank 0 only; ensemble members are shared
out by node count and their records gathered back."""
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


def _stub_member(w):
    """A member's record from a short FP64 oracle run of a reduced box with
    the member's own gradient frames, radius and icosphere level."""
    import oracle as O

    n = (16, 16, 16)
    c = tuple(0.5 * (k - 1) for k in n)
    o = O.OracleSim(n, w.tau, w.frames * 10.0, 3)
    r, t = O.icosphere(min(w.level, 2), min(w.R, 4.0), c)
    o.set_mesh(r, t, w.sigma)
    o.step(4)
    ob = O.observables(o.mesh()[0], t)
    o.close()
    return {"name": w.name, "D": float(ob["D"]), "V": float(ob["V"]), "xc": [float(v) for v in ob["xc"]]}


def _share_worker(rank, world, port, out):
    import torch.distributed as dist

    import bench
    from paper_2403_01161_gb300 import config

    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws = config.ensemble_workloads(6, steps=20)
    recs = bench.run_member_share(ws, rank, world, _stub_member)
    owner = bench.ensemble_partition([w.nodes for w in ws], world)
    out.put((rank, recs, [k for k in range(len(ws)) if owner[k] == rank]))
    dist.barrier()
    dist.destroy_process_group()


def test_member_share_gathers_the_one_rank_result():
    """Two gloo ranks split 6 uneven ensemble members by node count, each runs
    only its own share, and the records gathered on every rank are exactly
    those of one rank running all members."""
    import bench
    from paper_2403_01161_gb300 import config

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_share_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=300) for _ in range(2)), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    one = bench.run_member_share(config.ensemble_workloads(6, steps=20), 0, 1, _stub_member)
    assert sorted(one) == list(range(6))
    shares = [set(r[2]) for r in res]
    assert shares[0] and shares[1] and not (shares[0] & shares[1]) and shares[0] | shares[1] == set(range(6))
    for _, recs, _ in res:
        assert recs == one
