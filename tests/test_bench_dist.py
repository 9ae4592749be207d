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


def test_nvml_clock_sample_summary():
    """Median SM clock, the maximum, and every clock-event reason seen in any
    sample (bit masks of NVML's reasons)."""
    import bench
    names = bench.NvmlSampler.REASONS
    out = bench.summarize_clock_samples([(2070.0, 0), (2055.0, 0x4), (2070.0, 0), (1980.0, 0x4 | 0x8)], 2070.0,
                                        names)
    assert out == {"sm_mhz": 2062.5, "sm_max_mhz": 2070.0, "reasons": ["hw_slowdown", "sw_power_cap"],
                   "samples": 4}
    assert bench.summarize_clock_samples([], 2070.0, names) is None


def test_summary_of_the_line():
    """The compact summary at the end of the JSON line carries the PCG times
    and counts, the sweep's GDOF/s and the oracle's rates."""
    import bench
    out = {"value": 0.3, "roofline": {"kernel": "assemble", "frac": 0.7, "peak": 1.2586, "unit": "TFLOP/s"},
           "pcg": {"fp64": {"solve_s": 5.2, "iterations": 1440}, "mixed": {"solve_s": 4.6, "iterations": 1530},
                   "mixed_speedup": 1.13, "mixed_ir": {"solve_s": 1.07}},
           "gradient": {"workload": "c4", "forward_s": 0.39, "adjoint_s": 0.45, "total_s": 0.85,
                        "forward_iterations": 379},
           "sweep_c5": {"p": [2, 4], "assemble_f64_gdofs": [1.0, 1.2], "apply_gdofs": [1.5, 2.5],
                        "backward_gdofs": [0.9, 1.5], "precond_f32_gdofs": [18.0, 18.0]},
           "cpu_baseline": {"value": 2e-3, "cores": 16, "one_core": {"value": 1.8e-4}}}
    s = bench.summary(out)
    assert s["pcg_c3_to_1e-8"] == {"fp64_s": 5.2, "fp64_it": 1440, "mixed_s": 4.6, "mixed_it": 1530,
                                   "mixed_speedup": 1.13, "refinement_s": 1.07}
    assert s["gradient_c4_s"] == {"forward_s": 0.39, "adjoint_s": 0.45, "total_s": 0.85}
    assert s["sweep_c5_gdofs"]["p"] == [2, 4] and s["sweep_c5_gdofs"]["apply"] == [1.5, 2.5]
    assert s["oracle_gdofs"] == {"cores": 16, "all_cores": 2e-3, "one_core": 1.8e-4}
    assert s["roofline"].startswith("assemble 0.700")


def test_host_cores_is_positive():
    import bench
    assert bench.host_cores() >= 1


def test_profile_figures_are_read_only_while_the_sources_match(tmp_path, monkeypatch):
    """bench.read_traffic takes a figure from a committed ncu summary only
    while every source file listed there still has the recorded hash."""
    import hashlib
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel v1")
    prof = tmp_path / "profiles"
    prof.mkdir()
    digest = hashlib.sha256(b"kernel v1").hexdigest()
    (prof / "k_demo_c2_case.md").write_text("traffic_bytes_per_launch: 123\nfp64_pipe_active_fraction: 0.5\n"
                                            "source_sha256: %s k.cu\n" % digest)
    (prof / "k_demo_backward_c2_case.md").write_text("fp64_pipe_active_fraction: 0.9\n"
                                                     "source_sha256: %s k.cu\n" % digest)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.read_traffic("k_demo_c2_") == 123.0
    assert bench.read_traffic("k_demo_c2_", "fp64_pipe_active_fraction") == 0.5
    assert bench.read_traffic("k_demo_backward_c2_", "fp64_pipe_active_fraction") == 0.9
    src.write_text("kernel v2")
    assert bench.read_traffic("k_demo_c2_") is None
