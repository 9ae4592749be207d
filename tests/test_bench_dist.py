"""Multi-rank host logic of bench.py on CPU (gloo, world size 2): every rank
runs its own replica, timings are combined as max over ranks and the value
is the units of all ranks over that time; the reference arm prints on rank 0
only."""
import os
import socket

import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.barrier(world)
        t = 1.0 + rank  # rank 1 is the slow one
        tmax = bench.max_over_ranks(t, world)
        rate = bench.aggregate_rate(1000.0, tmax, world)
        q.put((rank, tmax, rate, bench.dist_info()))
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_aggregate_rate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, tmax, rate, info in res:
        assert tmax == 2.0
        assert rate == 2000.0 / 2.0
        assert info == (rank, world, rank)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    import bench

    class A:
        steps, warmup = 1, 3

    monkeypatch.setenv("RANK", "1")
    assert bench.run_reference(A(), 1, 2) is None
