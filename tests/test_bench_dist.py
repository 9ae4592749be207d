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


def test_reference_sample_shrinks_with_the_step_count():
    import bench
    # 0.2 s per step on the 8^3 box (25 ms on 4^3): up to 750 steps fit 150 s
    # on 8^3, up to 6,000 on 4^3
    assert bench.reference_box(10, 3, 0.2) == 8
    assert bench.reference_box(747, 3, 0.2) == 8
    assert bench.reference_box(1000, 3, 0.2) == 4
    assert bench.reference_box(3000, 3, 0.2) == 4
    assert bench.reference_box(10000, 3, 0.2) == 2
    assert bench.reference_box(10 ** 6, 3, 0.2) == 2  # never below 2^3


def test_reference_arm_line(monkeypatch):
    """The reference arm's JSON line on rank 0: the contract's keys, the
    oracle's rate, and zero host-device bytes."""
    import bench

    class A:
        steps, warmup = 2, 3

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(bench, "REFERENCE_BUDGET_S", 0.0)  # forces the smallest sub-box
    out = bench.run_reference(A(), 0, 1)
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in out, key
    assert out["impl"] == "reference" and out["value"] > 0 and out["steps"] == 2
    assert "2x2x2 elements" in out["config"]["workload"]
    assert out["e2e"]["h2d_bytes_per_step"] == 0 and out["e2e"]["value"] == out["value"]
    assert out["cpu_baseline"]["kind"] == "oracle" and out["cpu_baseline"]["cores"] == 1


def test_clock_log_summary():
    import bench
    lines = ["0, 2070, 2070, 910.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "0, 1980, 2070, 1390.2, 0x0000000000000004, Not Active, Not Active, Not Active, Active\n",
             "0, 2055, 2070, 1200.0, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active\n",
             "0, [N/A], 2070, [N/A], [N/A], [N/A], [N/A], [N/A], [N/A]\n",
             "truncated line, 2070\n"]
    out = bench.parse_clock_log(lines)
    assert out["sm_mhz"] == 2055.0 and out["sm_max_mhz"] == 2070.0
    assert out["reasons"] == ["sw_power_cap"] and out["samples"] == 4
    hot = lines[:1] + ["0, 1500, 2070, 700.0, 0x48, Active, Not Active, Active, Not Active\n"]
    assert bench.parse_clock_log(hot)["reasons"] == ["hw_slowdown", "sw_thermal_slowdown"]
    assert bench.parse_clock_log([]) is None
