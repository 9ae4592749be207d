#!/usr/bin/env python3
"""Benchmark of the LOR hot path on one GB300 (or N replicas, one per GPU).

One step = one pass of the hot path over the 16^3-element, p = 4 workload
(274,625 DOFs, jittered mesh, lognormal kappa, FP64):
  operator setup (D at the Gauss points) -> LOR assembly into CSR (FP64) ->
  high-order apply -> Chebyshev-Jacobi preconditioner (degree 3, FP64, with
  its diagonal) -> backward of the apply (gx and gkappa).
value = DOFs processed per second over the timed steps (GDOF/s), summed over
ranks.  The PCG time to 1e-8 (FP64 vs mixed precision, and the
mixed-precision refinement whose iterations run an FP32 operator) is
measured on the 32^3-element, p = 6 workload (7,189,057 DOFs) and reported
under "pcg" (with the FP64 and FP32 applies timed alone); the
adjoint gradient dJ/dtheta (forward solve, adjoint solve, gradient kernel) on
the 24^3-element, p = 5 workload under "gradient"; the same step with the
reaction term of the definite Helmholtz problem under "helmholtz"; the
macro-element vs unstructured LOR assembly at ~4M DOFs per degree under
"assembly_comparator"; the discrete gradient and vertex coordinates of the
32^3 p = 6 LOR mesh under "hcurl_topology"; the step's kernels on the same
workload handed over as a general mesh under "general_mesh"; the error of
every mixed-precision result against its FP64 counterpart under
"mixed_precision_errors".

Per kernel ("kernels"): time, GDOF/s and the fraction of the HBM peak; the
kernels whose arithmetic runs in 64-bit fixed point on the integer pipe (the
operator and its backward) report their FP64-equivalent rate (the direct
sum-factorisation count over the FP64 peak, frac_fp64_equiv, which may
exceed 1) and the fraction of the integer multiply-add peak their
mad.wide.s32 instructions take (int_mad_frac), the others frac_fp64: the
flops of the formula they evaluate over the FP64 peak (setup and assembly
form their metric's products in fixed point too, so theirs is also an
FP64-equivalent rate).  The FP64-pipe or issue-slot activity comes from the
committed ncu summaries while their sources are unchanged.

Runs as `python bench.py --gpus N --steps K --warmup W` (torchrun for N > 1:
every rank solves its own replica; no data-path collective).  With
`--impl reference` it times the CPU oracle instead (rank 0 only), each step
on a sub-box of the 16^3 p = 4 recipe sized so the whole run takes about
150 s.
"""
import argparse
import json
import os
import shutil
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "LOR assembly & HO apply GDOF/s (%HBM peak); PCG s to 1e-8, mixed vs FP64"
UNIT = "GDOF/s"
STEP_WORKLOAD = "c2_16x16x16_p4"
PCG_WORKLOAD = "c3_32x32x32_p6"
GRAD_WORKLOAD = "c4_24x24x24_p5"
L2_FLUSH_BYTES = 512 << 20


# ---------------------------------------------------------------- distributed helpers
def dist_info():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(
        os.environ.get("LOCAL_RANK", "0"))


def max_over_ranks(value, world):
    """Max of a float over all ranks (identity for a single process)."""
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(value, world):
    if world == 1:
        return float(value)
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_rate(units_per_rank, max_seconds, world):
    """Whole-job throughput: units processed by all ranks / max-over-ranks time."""
    return sum_over_ranks(units_per_rank, world) / max_seconds


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        if shutil.which("nvidia-smi") is None:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        self.f = open(self.path, "w")
        self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                      "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                     stderr=subprocess.DEVNULL)

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        with open(self.path) as f:
            out = parse_clock_log(f.readlines())
        os.remove(self.path)
        return out


class NvmlSampler:
    """SM clock and clock-event reasons read through NVML (read-only queries of
    libnvidia-ml, no settings changed) every `period` seconds on a background
    thread, so a timed region of a few milliseconds still gets samples.
    start() returns False where NVML cannot be loaded."""
    SM_CLOCK = 1  # NVML_CLOCK_SM
    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown"}

    def __init__(self, gpu_index, period=0.001, uuid=None):
        self.gpu, self.period, self.uuid = gpu_index, period, uuid
        self.samples, self.thread, self.lib = [], None, None

    def start(self):
        import ctypes
        import threading
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                return False
            h = ctypes.c_void_p()
            # the CUDA device by its UUID (NVML numbers every GPU of the machine), else by index
            found = self.uuid is not None and lib.nvmlDeviceGetHandleByUUID(
                ("GPU-" + str(self.uuid)).encode(), ctypes.byref(h)) == 0
            if not found and lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(self.gpu), ctypes.byref(h)) != 0:
                lib.nvmlShutdown()
                return False
            reasons_fn = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                lib.nvmlDeviceGetCurrentClocksThrottleReasons
        except (OSError, AttributeError):
            return False
        self.lib, self.h, self.reasons_fn = lib, h, reasons_fn
        mx = ctypes.c_uint(0)
        lib.nvmlDeviceGetMaxClockInfo(h, self.SM_CLOCK, ctypes.byref(mx))
        self.max_mhz = float(mx.value)
        self.stop_flag = threading.Event()

        def run():
            clk, rs = ctypes.c_uint(0), ctypes.c_ulonglong(0)
            while not self.stop_flag.is_set():
                if lib.nvmlDeviceGetClockInfo(h, self.SM_CLOCK, ctypes.byref(clk)) == 0 and \
                        reasons_fn(h, ctypes.byref(rs)) == 0:
                    self.samples.append((float(clk.value), int(rs.value)))
                time.sleep(self.period)
        self.thread = threading.Thread(target=run, daemon=True)
        self.thread.start()
        return True

    def stop(self):
        if self.thread is None:
            return None
        self.stop_flag.set()
        self.thread.join()
        self.lib.nvmlShutdown()
        out = summarize_clock_samples(self.samples, self.max_mhz, self.REASONS)
        if out is not None:
            out["source"] = "NVML every %g ms during the timed region" % (self.period * 1e3)
        return out


def summarize_clock_samples(samples, max_mhz, names):
    """Median SM clock, the maximum clock and the clock-event reasons seen in
    any sample, from (sm_mhz, reason bit mask) samples (None without one)."""
    if not samples:
        return None
    reasons = sorted({n for _, mask in samples for bit, n in names.items() if mask & bit})
    return {"sm_mhz": statistics.median(c for c, _ in samples), "sm_max_mhz": max_mhz, "reasons": reasons,
            "samples": len(samples)}


def parse_clock_log(lines):
    """Summary of `nvidia-smi --query-gpu=ClockSampler.FIELDS --format=csv,noheader,nounits`
    lines: median SM clock, maximum SM clock, and the throttle reasons seen
    Active in any sample (None without a complete sample)."""
    rows = []
    for line in lines:
        parts = [x.strip() for x in line.split(",")]
        if len(parts) >= 9:
            rows.append(parts)
    if not rows:
        return None
    sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
    mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
            "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- GPU arm
def fixed_point_fields(kind, p, nel, flops, ms):
    """The fields of a kernel whose FP64 arithmetic runs in 64-bit fixed point
    on the integer pipe (the operator and its backward): its FP64-equivalent
    rate (the direct sum-factorisation count over the FP64 peak, which it may
    exceed) and the fraction of the integer multiply-add peak its
    32 x 32 -> 64 bit multiply-adds take."""
    from paper_2210_12253_gb300.perfmodel import (FP64_PEAK_TFLOPS, INT_MAD_PEAK_TOPS, MAD_WIDE_PER_FIXED_MAC,
                                                 fixed_macs)
    mads = MAD_WIDE_PER_FIXED_MAC * fixed_macs(kind, p, nel)
    return {"arith": "int64 fixed point (3 mad.wide.s32 per multiply-add)",
            "gflops_fp64_equiv": flops / (ms * 1e-3) / 1e9,
            "frac_fp64_equiv": flops / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS,
            "int_mad_tops": mads / (ms * 1e-3) / 1e12,
            "int_mad_frac": mads / (ms * 1e-3) / 1e12 / INT_MAD_PEAK_TOPS}


def kernel_roofline(name, ms, work, hbm_peak, hbm_src, p=None, nel=None):
    from paper_2210_12253_gb300.perfmodel import FIXED_POINT_KINDS, FP64_PEAK_TFLOPS
    flops, nbytes = work
    out = {"ms": ms, "gbs": nbytes / (ms * 1e-3) / 1e9}
    if name in FIXED_POINT_KINDS and p is not None:
        out.update(fixed_point_fields(name, p, nel, flops, ms))
    else:
        out["gflops_fp64"] = flops / (ms * 1e-3) / 1e9
        out["frac_fp64"] = out["gflops_fp64"] / (FP64_PEAK_TFLOPS * 1e3)
    out["frac_hbm"] = out["gbs"] / hbm_peak
    return out


def read_traffic(kernel, key="traffic_bytes_per_launch"):
    """Per-launch DRAM bytes (or another `key: value` figure) from the committed
    ncu summary of `kernel`, or None when the summary is missing or was taken
    on a different source file."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles")
    if not os.path.isdir(prof):
        return None
    for fn in sorted(os.listdir(prof)):
        if not fn.startswith(kernel) or not fn.endswith(".md"):
            continue
        txt = open(os.path.join(prof, fn)).read()
        m = re.search(re.escape(key) + r":\s*([0-9.eE+]+)", txt)
        srcs = re.findall(r"source_sha256:\s*([0-9a-f]+)\s+(\S+)", txt)
        if not m or not srcs:
            continue
        for digest, rel in srcs:  # every source the kernel is built from must be unchanged
            src = os.path.join(ROOT, rel)
            if not os.path.exists(src) or hashlib.sha256(open(src, "rb").read()).hexdigest() != digest:
                return None
        return float(m.group(1))
    return None


def run_gpu(args, rank, world, local_rank):
    import numpy as np
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.build import build
    from paper_2210_12253_gb300.inputs import power_start_vector, workload
    from paper_2210_12253_gb300.lor import launch_count
    from paper_2210_12253_gb300.perfmodel import FP64_PEAK_TFLOPS, INT_MAD_PEAK_TOPS, hbm_peak_gbs, kernel_work

    if rank == 0:
        build()
    barrier(world)
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    hbm_peak, hbm_src = hbm_peak_gbs()

    prob = workload(STEP_WORKLOAD)
    p = prob.p
    op = LOR(p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=dev))
    kappa_h = torch.tensor(prob.kappa.reshape(-1)).pin_memory()
    kappa = kappa_h.to(dev)
    rng = np.random.default_rng(100 + rank)
    x_h = torch.tensor(rng.standard_normal(op.ndof)).pin_memory()
    gy_h = torch.tensor(rng.standard_normal(op.ndof)).pin_memory()
    r_h = torch.tensor(prob.rhs).pin_memory()
    x, gy, r = x_h.to(dev), gy_h.to(dev), r_h.to(dev)
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    gx = torch.empty_like(x)
    gk = torch.empty(op.nqpt, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    # one-time setup: pattern (A2, once per mesh) and the smoother's lambda_max
    op.set_coefficient(kappa, check=True)
    op.build_pattern_internal()
    op.assemble_internal(torch.float64)
    lam = op.precond_setup("cheb", torch.float64, degree=3, power_iters=20,
                           v0=torch.tensor(power_start_vector(op.ndof), device=dev))
    names = ["setup", "assemble", "apply", "precond", "backward"]

    def step(ev):
        ev[0].record()
        op.set_coefficient(kappa)
        ev[1].record()
        op.assemble_internal(torch.float64)
        ev[2].record()
        op.apply(x, out=y)
        ev[3].record()
        op.precond_setup("cheb", torch.float64, degree=3, lambda_max=lam)
        op.precond_apply(r, out=z)
        ev[4].record()
        op.apply_backward(x, gy, gx_out=gx, gk_out=gk)
        ev[5].record()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(args.steps)]
    for _ in range(args.warmup):
        flush.zero_()
        step([torch.cuda.Event(enable_timing=True) for _ in range(6)])
    torch.cuda.synchronize()
    clocks = NvmlSampler(local_rank, uuid=getattr(torch.cuda.get_device_properties(dev), "uuid", None))
    if not clocks.start():
        clocks = ClockSampler(local_rank)
        clocks.start()
    launches0 = launch_count()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        flush.zero_()  # L2 flush between steps (outside the step's events)
        step(evs[k])
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    launches = launch_count() - launches0
    clk = clocks.stop()
    per_kernel = {n: [] for n in names}
    step_ms = []
    for ev in evs:
        for i, n in enumerate(names):
            per_kernel[n].append(ev[i].elapsed_time(ev[i + 1]))
        step_ms.append(ev[0].elapsed_time(ev[5]))
    dev_s = sum(step_ms) / 1e3
    max_s = max_over_ranks(dev_s, world)
    value = aggregate_rate(op.ndof * args.steps, max_s, world) / 1e9

    # end to end through the public API: every step's inputs copied in from pinned host memory
    # and every result read back, inside the timed region.  Copies run on a second stream with
    # double-buffered device inputs/outputs, so step k+1's inputs and step k's results move
    # while step k computes; the compute stream waits for each step's inputs by event.
    e2e_steps = max(10, args.steps // 2)
    comp_s = torch.cuda.current_stream()
    copy_s = torch.cuda.Stream()
    ins = [(kappa, x, gy, r)] + [tuple(torch.empty_like(t) for t in (kappa, x, gy, r))]
    outs = [(y, z, gx, gk)] + [tuple(torch.empty_like(t) for t in (y, z, gx, gk))]
    hosts = [tuple(torch.empty(t.numel(), dtype=t.dtype).pin_memory() for t in (y, z, gx, gk))
             for _ in range(2)]
    h_in = (kappa_h, x_h, gy_h, r_h)
    in_ready = [torch.cuda.Event() for _ in range(2)]
    done = [torch.cuda.Event() for _ in range(2)]

    def e2e_step(b):
        kb, xb, gyb, rb = ins[b]
        yb, zb, gxb, gkb = outs[b]
        comp_s.wait_event(in_ready[b])
        op.set_coefficient(kb)
        op.assemble_internal(torch.float64)
        op.apply(xb, out=yb)
        op.precond_setup("cheb", torch.float64, degree=3, lambda_max=lam)
        op.precond_apply(rb, out=zb)
        op.apply_backward(xb, gyb, gx_out=gxb, gk_out=gkb)
        done[b].record(comp_s)

    def h2d(b):
        for dst, src in zip(ins[b], h_in):
            dst.copy_(src, non_blocking=True)
        in_ready[b].record(copy_s)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(comp_s)
    copy_s.wait_stream(comp_s)
    with torch.cuda.stream(copy_s):
        h2d(0)
    for k in range(e2e_steps):
        b = k % 2
        e2e_step(b)
        with torch.cuda.stream(copy_s):
            if k + 1 < e2e_steps:
                copy_s.wait_event(done[1 - b])  # step k-1 no longer reads buffer set 1-b
                h2d(1 - b)
            copy_s.wait_event(done[b])
            for dst, src in zip(hosts[b], outs[b]):
                dst.copy_(src, non_blocking=True)
    comp_s.wait_stream(copy_s)
    e1.record(comp_s)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(e0.elapsed_time(e1) / 1e3, world)
    e2e_value = aggregate_rate(op.ndof * e2e_steps, e2e_s, world) / 1e9
    h2d = 8 * (op.nqpt + 3 * op.ndof)
    d2h = 8 * (3 * op.ndof + op.nqpt)

    kernels = {}
    for n in names:
        ms = statistics.mean(per_kernel[n])
        work = kernel_work(n, p, op.ndof, op.nel, op.nnz, vbytes=8, degree=3)
        kernels[n] = kernel_roofline(n, ms, work, hbm_peak, hbm_src, p, op.nel)
        kernels[n]["gdofs"] = op.ndof / (ms * 1e-3) / 1e9
    # each kernel's committed ncu summary (used only while its sources are unchanged)
    prof = {"setup": "k_setup_c2_", "assemble": "k_assemble_c2_", "apply": "k_apply_c2_",
            "backward": "k_apply_backward_c2_", "precond": "k_stencil_c2_"}
    for n in names:
        # FP64-pipe kernels: FP64-pipe activity; fixed-point ones: issue-slot activity
        if "int_mad_frac" in kernels[n]:
            kernels[n]["issue_active"] = read_traffic(prof[n], "issue_active_fraction")
        else:
            kernels[n]["fp64_pipe_active"] = read_traffic(prof[n], "fp64_pipe_active_fraction")
    dominant = max(names, key=lambda n: kernels[n]["ms"])
    dk = kernels[dominant]
    traffic = read_traffic(prof[dominant])
    if "int_mad_frac" in dk:
        roofline = {"kernel": dominant, "bound": "alu", "achieved": dk["int_mad_tops"], "peak": INT_MAD_PEAK_TOPS,
                    "unit": "T int32 multiply-adds/s", "frac": dk["int_mad_frac"],
                    "peak_source": "derived: 152 SMs x 64 IMAD/clk x 2.07 GHz",
                    "issue_active": dk["issue_active"]}
    else:
        roofline = {"kernel": dominant, "bound": "alu", "achieved": dk["gflops_fp64"] / 1e3,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": dk["gflops_fp64"] / 1e3 / FP64_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (FP64; no FP64 entry in "
                                   "MEASURED_PEAKS.json)",
                    "fp64_pipe_active": dk["fp64_pipe_active"]}
        if dominant in ("assemble", "setup"):
            roofline["numerator"] = ("FP64-equivalent: the flops of the formula the kernel evaluates "
                                     "(perfmodel) over the FP64 peak; the kernel forms the metric's products "
                                     "(and the assembly its block algebra) in 64-bit fixed point on the "
                                     "integer pipe, so the FP64 pipe is busy for part of it (fp64_pipe_active)")
    roofline.update({"traffic": traffic,
                     "hbm": {"achieved_gbs": dk["gbs"], "peak_gbs": hbm_peak, "peak_source": hbm_src,
                             "frac": dk["frac_hbm"]}})

    pcg = None
    if not args.no_pcg:
        pcg = run_pcg(args, dev, rank)
    grad = None
    if not args.no_grad:
        grad = run_gradient(args, dev)
    helm = None
    if not args.no_helmholtz:
        helm = run_helmholtz(args, dev)
    comparator = None
    if not args.no_comparator:
        comparator = run_comparator(args, dev)
    hcurl = None
    if not args.no_hcurl:
        hcurl = run_hcurl(args, dev)
    general = None
    if not args.no_general:
        general = run_general(args, dev)
    precision = None
    if not args.no_precision:
        precision = run_precision(args, dev)
    sweep_c5 = None
    if not args.no_c5:
        sweep_c5 = run_sweep_compact(args, dev)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": max_s * 1e3 / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": STEP_WORKLOAD + ": unit cube 16^3 hexes, p=4, 274,625 DOFs, +-10% h jitter (seed 1),"
                                  " kappa lognormal(0,1) at 6^3 Gauss points/element",
                      "step": "setup(D) + LOR assembly(f64, CSR) + HO apply + Chebyshev-Jacobi deg 3 (f64) + "
                              "apply backward (gx, gkappa)",
                      "ndof": op.ndof, "nnz": op.nnz, "elements": op.nel, "p": p,
                      "l2": "flushed between steps (512 MB write, outside the step events)",
                      "parallelism": "replicas x%d (one independent problem per GPU)" % world,
                      "wall_s": wall},
           "kernels": kernels, "roofline": roofline,
           "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                   "steps": e2e_steps,
                   "copies": "pinned host <-> device on a second stream, double-buffered: step k+1's "
                             "inputs and step k's results move while step k computes"},
           "gpu_launches": int(launches), "clocks": clk, "pcg": pcg, "gradient": grad,
           "helmholtz": helm, "assembly_comparator": comparator, "hcurl_topology": hcurl,
           "general_mesh": general, "mixed_precision_errors": precision, "sweep_c5": sweep_c5}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    out["summary"] = summary(out)
    op.close()
    return out


def summary(out):
    """The line's key results in a few hundred characters, last on the line:
    the dominant kernel's roofline, the PCG times to 1e-8 (32^3 p = 6), the
    gradient solves, the p-sweep's GDOF/s and the oracle's rates."""
    r = out["roofline"]
    s = {"step_gdofs": round(out["value"], 4),
         "roofline": "%s %.3f of %s %s" % (r["kernel"], r["frac"], r["peak"], r["unit"])}
    pc = out.get("pcg")
    if pc:
        s["pcg_c3_to_1e-8"] = {"fp64_s": round(pc["fp64"]["solve_s"], 3), "fp64_it": pc["fp64"]["iterations"],
                               "mixed_s": round(pc["mixed"]["solve_s"], 3), "mixed_it": pc["mixed"]["iterations"],
                               "mixed_speedup": round(pc["mixed_speedup"], 3)}
        if pc.get("mixed_ir"):
            s["pcg_c3_to_1e-8"]["refinement_s"] = round(pc["mixed_ir"]["solve_s"], 3)
    g = out.get("gradient")
    if g:
        s["gradient_c4_s"] = {k: round(v, 4) for k, v in g.items() if k.endswith("_s") and isinstance(v, float)}
    c5 = out.get("sweep_c5")
    if c5:
        s["sweep_c5_gdofs"] = {"p": c5["p"]}
        for k in ("assemble_f64", "apply", "backward", "precond_f32"):
            s["sweep_c5_gdofs"][k] = [round(v, 3) for v in c5[k + "_gdofs"]]
    cb = out.get("cpu_baseline")
    if cb:
        s["oracle_gdofs"] = {"cores": cb["cores"], "all_cores": cb["value"], "one_core": cb["one_core"]["value"]}
    return s


def run_pcg(args, dev, rank):
    """PCG to 1e-8 on the 32^3, p = 6 workload: FP64 vs mixed precision."""
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import power_start_vector, workload

    prob = workload(PCG_WORKLOAD)
    op = LOR(prob.p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=dev))
    b = torch.tensor(prob.rhs, device=dev)
    v0 = torch.tensor(power_start_vector(op.ndof), device=dev)
    res = {"workload": PCG_WORKLOAD + ": 32^3 hexes, p=6, 7,189,057 DOFs, +-10% h jitter (seed 2), kappa "
                                      "lognormal(0,1); Chebyshev-Jacobi deg 3 on [lmax/30, 1.1 lmax], rtol 1e-8 "
                                      "confirmed on the true FP64 residual"}
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    for label, dt in (("fp64", torch.float64), ("mixed", torch.float32)):
        ev[0].record()
        op.set_coefficient(torch.tensor(prob.kappa.reshape(-1), device=dev))
        op.build_pattern_internal()
        ev[1].record()
        op.assemble_internal(dt)
        lam = op.precond_setup("cheb", dt, degree=3, power_iters=20, v0=v0)
        ev[2].record()
        torch.cuda.synchronize()
        op.pcg_solve(b, 1e-8, 3, raise_on_noconv=False)  # warm-up of the solve kernels
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        u, it, rel = op.pcg_solve(b, 1e-8, args.pcg_maxit, raise_on_noconv=args.pcg_maxit >= 20000)
        e1.record()
        torch.cuda.synchronize()
        if label == "fp64":
            u64 = u.clone()
        solve_s = e0.elapsed_time(e1) / 1e3
        res[label] = {"solve_s": solve_s, "wall_s": time.perf_counter() - t0, "iterations": it,
                      "final_rel_residual": rel, "lambda_max": lam,
                      "setup_s": ev[0].elapsed_time(ev[2]) / 1e3,
                      "s_per_iteration": solve_s / max(it, 1)}
    res["mixed_speedup"] = res["fp64"]["solve_s"] / res["mixed"]["solve_s"]
    res.update(run_refinement(args, op, b, res, u64))
    if args.pcg_degrees:
        # supplementary: the Chebyshev degree trade-off (the FP32 smoother is
        # cheap next to the FP64 apply), mixed precision and FP64, same lambda
        lam = res["mixed"]["lambda_max"]
        res["degree_sweep"] = []
        for k in args.pcg_degrees:
            row = {"degree": k}
            for label, dt in (("mixed", torch.float32), ("mixed_ir", torch.float32), ("fp64", torch.float64)):
                op.assemble_internal(dt)
                op.precond_setup("cheb", dt, degree=k, lambda_max=lam)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                if label == "mixed_ir":
                    _, _, it, _ = op.pcg_solve_ir(b, 1e-8, args.ir_inner_rtol, 20000)
                else:
                    _, it, _ = op.pcg_solve(b, 1e-8, 20000)
                e1.record()
                torch.cuda.synchronize()
                row[label] = {"solve_s": e0.elapsed_time(e1) / 1e3, "iterations": it}
            res["degree_sweep"].append(row)
    op.close()
    return res


def run_refinement(args, op, b, res, u64):
    """Mixed-precision iterative refinement on the PCG workload (same FP32 LOR
    matrix and smoother as "mixed"): FP64 outer residuals, inner PCG with the
    FP32-arithmetic operator to inner_rtol; and the FP32 apply kernel against
    the FP64 one (D larger than L2 at this size, so no flush is needed)."""
    import torch

    from paper_2210_12253_gb300.perfmodel import FP32_PEAK_TFLOPS, FP64_PEAK_TFLOPS, hbm_peak_gbs, kernel_work

    out = {}
    hbm, hbm_src = hbm_peak_gbs()
    x = torch.randn(op.ndof, dtype=torch.float64, device=b.device)
    y = torch.empty_like(x)
    kern = {}
    for label, fn, kind in (("apply_f64", op.apply, "apply"), ("apply_f32", op.apply_f32, "apply_f32")):
        fn(x, out=y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 10
        e0.record()
        for _ in range(reps):
            fn(x, out=y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        flops, byts = kernel_work(kind, op.p, op.ndof, op.nel, op.nnz)
        kern[label] = {"ms": ms, "gdofs": op.ndof / (ms * 1e-3) / 1e9, "gbs": byts / (ms * 1e-3) / 1e9,
                       "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm}
        if kind == "apply_f32":
            kern[label].update({"tflops": flops / (ms * 1e-3) / 1e12,
                                "frac_alu": flops / (ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS, "alu": "fp32"})
        else:
            kern[label].update(fixed_point_fields(kind, op.p, op.nel, flops, ms))
    y32 = op.apply_f32(x)
    y64 = op.apply(x)
    kern["apply_f32_max_rel_err"] = ((y32 - y64).abs().max() / y64.abs().max()).item()
    kern["hbm_peak_gbs"] = hbm
    kern["hbm_peak_source"] = hbm_src
    kern["note"] = ("both include the FP64 output initialisation launch; ms per apply, 10 back-to-back "
                    "applies (D: 805 MB FP64 / 403 MB FP32, larger than L2)")
    out["apply_kernels"] = kern

    op.assemble_internal(torch.float32)
    op.precond_setup("cheb", torch.float32, degree=3, lambda_max=res["mixed"]["lambda_max"])
    xs = torch.empty_like(b)
    for scheme in ("replace", "restart"):  # warm-up
        op.pcg_solve_ir(b, 1e-8, args.ir_inner_rtol, 3, x=xs, raise_on_noconv=False, scheme=scheme)
    rows = []
    runs = [("replace", args.ir_inner_rtol), ("restart", args.ir_inner_rtol)]
    runs += [(sch, r) for r in (args.ir_sweep or []) if r != args.ir_inner_rtol for sch in ("replace", "restart")]
    for scheme, inner_rtol in runs:
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        e0.record()
        u, outer, inner, rel = op.pcg_solve_ir(b, 1e-8, inner_rtol, args.pcg_maxit, x=xs, scheme=scheme,
                                               raise_on_noconv=args.pcg_maxit >= 20000)
        e1.record()
        torch.cuda.synchronize()
        solve_s = e0.elapsed_time(e1) / 1e3
        rows.append({"scheme": scheme, "inner_rtol": inner_rtol, "solve_s": solve_s,
                     "wall_s": time.perf_counter() - t0,
                     "outer_iterations": outer, "inner_iterations": inner, "final_rel_residual": rel,
                     "s_per_inner_iteration": solve_s / max(inner, 1),
                     "speedup_vs_fp64": res["fp64"]["solve_s"] / solve_s,
                     "speedup_vs_mixed": res["mixed"]["solve_s"] / solve_s,
                     "solution_vs_fp64_max_rel_diff": ((u - u64).abs().max() / u64.abs().max()).item()})
    out["mixed_ir"] = rows[0]
    out["mixed_ir"]["description"] = (
        "mixed-precision refinement, residual-replacement scheme: one PCG (FP32 LOR Chebyshev deg 3, FP64 "
        "dots/recurrences) on the FP32-arithmetic operator; after each inner_rtol reduction of its recurrence "
        "residual the FP64 residual b - A_p x replaces it; stop on the FP64 residual")
    out["mixed_ir_restart"] = rows[1]
    if len(rows) > 2:
        out["mixed_ir_inner_rtol_sweep"] = rows
    return out


def run_apply_kernels(args, dev):
    """FP64 and FP32 high-order applies on an NEX^3 unit-cube mesh of degree
    P (jitter 10%, lognormal kappa, seed 2): two untimed applies each, then 10
    timed back-to-back (CUDA events)."""
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import make_problem
    from paper_2210_12253_gb300.perfmodel import hbm_peak_gbs, kernel_work

    nex, p = args.apply_kernels
    prob = make_problem("apply", nex, nex, nex, p, seed=2, jitter=0.1, kappa="lognormal", rhs="normal")
    op = LOR(p, nex, nex, nex, torch.tensor(prob.vertices, device=dev))
    op.set_coefficient(torch.tensor(prob.kappa.reshape(-1), device=dev))
    x = torch.randn(op.ndof, dtype=torch.float64, device=dev)
    y = torch.empty_like(x)
    hbm, _ = hbm_peak_gbs()
    out = {"workload": "%d^3 elements, p=%d, %d DOFs" % (nex, p, op.ndof)}
    for label, fn, kind in (("apply_f32", op.apply_f32, "apply_f32"), ("apply_f64", op.apply, "apply")):
        for _ in range(2):
            fn(x, out=y)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(10):
            fn(x, out=y)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 10
        _, byts = kernel_work(kind, p, op.ndof, op.nel, op.nnz)
        out[label] = {"ms": ms, "gdofs": op.ndof / (ms * 1e-3) / 1e9, "frac_hbm": byts / (ms * 1e-3) / 1e9 / hbm}
    op.close()
    return out


def run_gradient(args, dev):
    """dJ/dtheta on the 24^3, p = 5 workload (1,771,561 DOFs): forward PCG
    solve, adjoint PCG solve with the same preconditioner, and the gradient
    kernel, each timed with CUDA events (rtol 1e-8, FP64)."""
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import power_start_vector, workload

    prob = workload(GRAD_WORKLOAD)
    op = LOR(prob.p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=dev))
    b = torch.tensor(prob.rhs, device=dev)
    v0 = torch.tensor(power_start_vector(op.ndof), device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(6)]
    theta = torch.tensor(prob.theta.reshape(-1), device=dev)
    kstar = torch.exp(torch.tensor(prob.theta_star.reshape(-1), device=dev))
    op.set_coefficient(kstar)
    op.build_pattern_internal()
    op.assemble_internal(torch.float64)
    op.precond_setup("cheb", torch.float64, degree=3, power_iters=20, v0=v0)
    ustar, _, _ = op.pcg_solve(b, 1e-8, 20000)
    # output buffers allocated, and the gradient kernel launched once, before
    # the events (device allocation would otherwise sit inside them)
    kappa = torch.empty_like(theta)
    gk = torch.empty_like(theta)
    grad = torch.empty_like(theta)
    resid = torch.empty_like(b)
    op.apply_backward(ustar, b, want_gx=False, gk_out=gk)
    # first use of each elementwise torch op outside the events too (a fresh
    # process pays a one-time load of the op's kernel, ~1 s measured)
    torch.exp(theta, out=kappa)
    torch.sub(ustar, ustar, out=resid)
    torch.mul(kappa, gk, out=grad).neg_()
    torch.cuda.synchronize()
    ev[0].record()
    torch.exp(theta, out=kappa)
    op.set_coefficient(kappa)
    op.assemble_internal(torch.float64)
    op.precond_setup("cheb", torch.float64, degree=3, power_iters=20, v0=v0)
    ev[1].record()
    u, it_f, _ = op.pcg_solve(b, 1e-8, 20000)
    ev[2].record()
    torch.sub(u, ustar, out=resid)
    lam, it_a, _ = op.pcg_solve(resid, 1e-8, 20000)
    ev[3].record()
    op.apply_backward(u, lam, want_gx=False, gk_out=gk)
    torch.mul(kappa, gk, out=grad).neg_()
    ev[4].record()
    torch.cuda.synchronize()
    res = {"workload": GRAD_WORKLOAD + ": 24^3 hexes, p=5, 1,771,561 DOFs, +-10% h jitter (seed 3), "
                                       "theta ~ N(0, 0.5^2), J = |u - u*|^2 / 2, PCG rtol 1e-8 (FP64)",
           "setup_s": ev[0].elapsed_time(ev[1]) / 1e3, "forward_s": ev[1].elapsed_time(ev[2]) / 1e3,
           "adjoint_s": ev[2].elapsed_time(ev[3]) / 1e3, "gradient_kernel_ms": ev[3].elapsed_time(ev[4]),
           "forward_iterations": it_f, "adjoint_iterations": it_a,
           "total_s": ev[0].elapsed_time(ev[4]) / 1e3, "grad_norm": float(grad.norm())}
    op.close()
    return res


def run_helmholtz(args, dev):
    """The bench step with the reaction term of the definite Helmholtz
    problem (Section 4.1) on the 16^3, p = 4 workload: beta = exp(N(0,1)) at
    the Gauss points (seeded), then setup (D and beta w detJ), LOR assembly
    with the sub-hex mass blocks (FP64), HO apply, Chebyshev-Jacobi degree 3
    (FP64) and the backward; CUDA-event timed per kernel, L2 flushed between
    steps.  Reported next to the diffusion-only step."""
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import power_start_vector, reaction_coefficient, workload
    from paper_2210_12253_gb300.perfmodel import FP64_PEAK_TFLOPS, hbm_peak_gbs, kernel_work

    prob = workload(STEP_WORKLOAD)
    p, q = prob.p, prob.q
    op = LOR(p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=dev))
    kappa = torch.tensor(prob.kappa.reshape(-1), device=dev)
    beta = torch.tensor(reaction_coefficient(op.nel, q).reshape(-1), device=dev)
    g = torch.Generator().manual_seed(5)
    x = torch.randn(op.ndof, generator=g, dtype=torch.float64).to(dev)
    gy = torch.randn(op.ndof, generator=g, dtype=torch.float64).to(dev)
    r = torch.tensor(prob.rhs, device=dev)
    y, z, gx = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    gk = torch.empty(op.nqpt, dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    op.set_coefficient(kappa, check=True)
    op.set_reaction(beta, check=True)
    op.build_pattern_internal()
    op.assemble_internal(torch.float64)
    lam = op.precond_setup("cheb", torch.float64, degree=3, power_iters=20,
                           v0=torch.tensor(power_start_vector(op.ndof), device=dev))
    names = ["setup", "reaction_setup", "assemble_helmholtz", "apply_helmholtz", "precond", "backward_helmholtz"]

    def step(ev):
        ev[0].record()
        op.set_coefficient(kappa)
        ev[1].record()
        op.set_reaction(beta)
        ev[2].record()
        op.assemble_internal(torch.float64)
        ev[3].record()
        op.apply(x, out=y)
        ev[4].record()
        op.precond_setup("cheb", torch.float64, degree=3, lambda_max=lam)
        op.precond_apply(r, out=z)
        ev[5].record()
        op.apply_backward(x, gy, gx_out=gx, gk_out=gk)
        ev[6].record()

    steps = max(10, args.steps // 10)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(7)] for _ in range(steps)]
    for _ in range(max(3, args.warmup)):
        flush.zero_()
        step([torch.cuda.Event(enable_timing=True) for _ in range(7)])
    torch.cuda.synchronize()
    for k in range(steps):
        flush.zero_()
        step(evs[k])
    torch.cuda.synchronize()
    hbm_peak, hbm_src = hbm_peak_gbs()
    kernels = {}
    for i, n in enumerate(names):
        ms = statistics.mean(ev[i].elapsed_time(ev[i + 1]) for ev in evs)
        work = kernel_work(n, p, op.ndof, op.nel, op.nnz, vbytes=8, degree=3)
        kernels[n] = kernel_roofline(n, ms, work, hbm_peak, hbm_src, p, op.nel)
        kernels[n]["gdofs"] = op.ndof / (ms * 1e-3) / 1e9
    step_ms = statistics.mean(ev[0].elapsed_time(ev[6]) for ev in evs)
    op.close()
    return {"workload": STEP_WORKLOAD + " with beta = exp(N(0,1)) per Gauss point (seed 777)",
            "steps": steps, "ms_per_step": step_ms, "gdofs": op.ndof / (step_ms * 1e-3) / 1e9,
            "fp64_peak_tflops": FP64_PEAK_TFLOPS, "kernels": kernels}


def run_comparator(args, dev):
    """Macro-element vs unstructured LOR assembly (Section 4.2's comparison)
    at about 4M DOFs for p = 1, 2, 3, 4, 6, 8 (jittered mesh, lognormal
    kappa, seed 4, FP64 values).  macro = lor_assemble; unstructured =
    lor_assemble_unstructured on the LOR mesh given as E-vectors (built once
    by lor_lor_mesh, whose time is reported separately: the paper notes that
    building the LOR mesh and its restriction dominates the unstructured
    path).  Median of 5 event-timed launches after one warm-up, L2 flushed
    before each."""
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import make_problem

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed(fn, reps=5):
        fn()
        out = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    rows = []
    for p in (1, 2, 3, 4, 6, 8):
        ne = max(1, round(4e6 ** (1 / 3) / p))
        prob = make_problem("cmp_p%d" % p, ne, ne, ne, p, seed=4, kappa="lognormal", rhs=None)
        op = LOR(p, ne, ne, ne, torch.tensor(prob.vertices, device=dev))
        op.set_coefficient(torch.tensor(prob.kappa.reshape(-1), device=dev))
        rp, ci = op.build_pattern()
        op.build_pattern_internal()
        vals = torch.empty(op.nnz, dtype=torch.float64, device=dev)
        ms_macro = timed(lambda: op.assemble(torch.float64, out=vals))
        mesh_box = {}

        def build_mesh():
            mesh_box["m"] = op.lor_mesh()

        ms_mesh = timed(build_mesh, reps=3)
        corners, dofs, ks, _, ess = mesh_box["m"]
        ms_uns = timed(lambda: op.assemble_unstructured(corners, dofs, ks, rp, ci, op.ndof, ess=ess, out=vals))
        op.check()
        rows.append({"p": p, "elements": op.nel, "ndof": op.ndof, "nnz": op.nnz, "macro_ms": ms_macro,
                     "unstructured_ms": ms_uns, "lor_mesh_ms": ms_mesh,
                     "macro_gdofs": op.ndof / (ms_macro * 1e-3) / 1e9,
                     "unstructured_gdofs": op.ndof / (ms_uns * 1e-3) / 1e9,
                     "ratio": ms_uns / ms_macro, "ratio_with_mesh": (ms_uns + ms_mesh) / ms_macro})
        del corners, dofs, ks, ess, mesh_box, vals, rp, ci
        op.close()
        torch.cuda.empty_cache()
    return {"workload": "~4M DOFs per degree, +-10% jitter, kappa lognormal(0,1), seed 4, FP64 values",
            "rows": rows}


def run_hcurl(args, dev):
    """The LOR mesh's H(curl) topology on the 32^3, p = 6 mesh (7.19M vertices,
    21.5M edges): the discrete gradient (Algorithm 1) and the deduplicated
    vertex coordinates; median of 5 event-timed launches after one warm-up,
    L2 flushed before each.  Both are HBM-bound writes: 32 bytes per edge
    (row pointer 8, two int32 columns 8, two f64 values 16) and 24 bytes per
    vertex."""
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import workload
    from paper_2210_12253_gb300.perfmodel import hbm_peak_gbs

    prob = workload(PCG_WORKLOAD)
    op = LOR(prob.p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=dev))
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    ne = op.edge_count()
    rp = torch.empty(ne + 1, dtype=torch.int64, device=dev)
    ci = torch.empty(2 * ne, dtype=torch.int32, device=dev)
    vals = torch.empty(2 * ne, dtype=torch.float64, device=dev)
    xyz = torch.empty(3 * op.ndof, dtype=torch.float64, device=dev)
    from paper_2210_12253_gb300.lor import _ptr

    def timed(fn):
        fn()
        out = []
        for _ in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    ms_g = timed(lambda: op._call("lor_discrete_gradient", _ptr(rp), _ptr(ci), _ptr(vals), None))
    ms_x = timed(lambda: op._call("lor_vertex_coordinates", _ptr(xyz)))
    peak, src = hbm_peak_gbs()
    bg, bx = 32 * ne + 8, 24 * op.ndof
    op.close()
    return {"workload": PCG_WORKLOAD + " mesh (topology only)", "edges": ne, "vertices": op.ndof,
            "discrete_gradient": {"ms": ms_g, "gbs": bg / (ms_g * 1e-3) / 1e9,
                                  "frac_hbm": bg / (ms_g * 1e-3) / 1e9 / peak, "bytes": bg},
            "vertex_coordinates": {"ms": ms_x, "gbs": bx / (ms_x * 1e-3) / 1e9,
                                   "frac_hbm": bx / (ms_x * 1e-3) / 1e9 / peak, "bytes": bx},
            "hbm_peak_gbs": peak, "peak_source": src}


def run_general(args, dev):
    """The 16^3 p=4 step workload handed over as a general mesh (corners,
    element-to-DOF map, essential mask; natural numbering, no rotation):
    pattern build (count/scan/fill/sort on the GPU), setup, FP64 assembly
    (CSR positions by search), apply, backward and the FP64 Chebyshev step
    on the explicit pattern, each next to the structured path's time.  Median
    of 5 event-timed launches after one warm-up, L2 flushed before each."""
    import numpy as np
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import boundary_mask, power_start_vector, workload

    prob = workload(STEP_WORKLOAD)
    p, n = prob.p, prob.p + 1
    nex, ney, nez = prob.nex, prob.ney, prob.nez
    V = prob.vertices.reshape(nez + 1, ney + 1, nex + 1, 3)
    ez, ey, ex = np.meshgrid(np.arange(nez), np.arange(ney), np.arange(nex), indexing="ij")
    corners = np.stack([V[ez + (c >> 2), ey + ((c >> 1) & 1), ex + (c & 1)] for c in range(8)], axis=3)
    corners = corners.reshape(-1, 8, 3)
    k, j, i = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    nx, ny = nex * p + 1, ney * p + 1
    edofs = ((ex.reshape(-1, 1) * p + i.reshape(1, -1)) +
             nx * ((ey.reshape(-1, 1) * p + j.reshape(1, -1)) + ny * (ez.reshape(-1, 1) * p + k.reshape(1, -1))))
    ess = boundary_mask(nex, ney, nez, p).astype(np.uint8)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def timed(fn, reps=5):
        fn()
        out = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            out.append(e0.elapsed_time(e1))
        return statistics.median(out)

    t_c, t_d, t_e = (torch.tensor(a, device=dev) for a in (corners, edofs, ess))
    t0 = time.perf_counter()
    g = LOR.general(p, t_c, t_d, int(ess.size), t_e)
    create_s = time.perf_counter() - t0
    s = LOR(p, nex, ney, nez, torch.tensor(prob.vertices, device=dev))
    kappa = torch.tensor(prob.kappa.reshape(-1), device=dev)
    x = torch.tensor(np.random.default_rng(5).standard_normal(g.ndof), device=dev)
    r = torch.tensor(prob.rhs, device=dev)
    out = {"workload": STEP_WORKLOAD + " as a general mesh (natural numbering)", "create_s": create_s,
           "nnz": g.nnz}
    for name, op in (("general", g), ("structured", s)):
        y, z, gx = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
        gk = torch.empty(op.nqpt, dtype=torch.float64, device=dev)
        op.set_coefficient(kappa, check=True)
        op.build_pattern_internal()
        op.assemble_internal(torch.float64)
        lam = op.precond_setup("cheb", torch.float64, degree=3, power_iters=20,
                               v0=torch.tensor(power_start_vector(op.ndof), device=dev))
        out[name] = {
            "setup_ms": timed(lambda: op.set_coefficient(kappa)),
            "assemble_ms": timed(lambda: op.assemble_internal(torch.float64)),
            "apply_ms": timed(lambda: op.apply(x, out=y)),
            "backward_ms": timed(lambda: op.apply_backward(x, x, gx_out=gx, gk_out=gk)),
            "precond_ms": timed(lambda: op.precond_apply(r, out=z)),
            "lambda_max": lam}
    g.close()
    s.close()
    return out


def run_precision(args, dev):
    """Error of every mixed-precision result against its FP64 counterpart on
    the 16^3 p=4 workload (the FP64 path matches the FP64 oracle to 1e-12,
    see the parity tests): LOR values (max relative error per row maximum),
    SpMV, the Chebyshev-Jacobi preconditioned vector, the PCG solution to
    1e-8 (relative max-norm difference and the true FP64 residual of each);
    the FP32-arithmetic apply and the refinement solver's solution (both
    schemes) likewise."""
    import numpy as np
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import power_start_vector, workload

    prob = workload(STEP_WORKLOAD)
    op = LOR(prob.p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=dev))
    op.set_coefficient(torch.tensor(prob.kappa.reshape(-1), device=dev), check=True)
    rp, _ = op.build_pattern()
    op.build_pattern_internal()
    v64 = op.assemble(torch.float64)
    v32 = op.assemble(torch.float32).double()
    rows = torch.repeat_interleave(torch.arange(op.ndof, device=dev), rp[1:] - rp[:-1])
    rowmax = torch.zeros(op.ndof, dtype=torch.float64, device=dev).scatter_reduce(0, rows, v64.abs(), "amax")
    val_err = float(((v32 - v64).abs() / rowmax[rows]).max())
    x = torch.tensor(np.random.default_rng(8).standard_normal(op.ndof), device=dev)
    b = torch.tensor(prob.rhs, device=dev)
    v0 = torch.tensor(power_start_vector(op.ndof), device=dev)
    out = {"workload": STEP_WORKLOAD, "lor_values_f32_max_rel_err": val_err}
    res = {}
    for dt in (torch.float64, torch.float32):
        op.assemble_internal(dt)
        lam = op.precond_setup("cheb", dt, degree=3, power_iters=20, v0=v0)
        res[dt] = {"lam": lam, "spmv": op.spmv(x, dt), "z": op.precond_apply(b)}
        u, it, rel = op.pcg_solve(b, 1e-8, 20000)
        true_rel = float((b - op.apply(u)).norm() / b.norm())
        res[dt].update(u=u, it=it, true_rel=true_rel)
    rel = lambda a, r: float((a - r).abs().max() / r.abs().max())
    out.update({
        "lambda_max_f32_rel_err": abs(res[torch.float32]["lam"] - res[torch.float64]["lam"]) / res[torch.float64]["lam"],
        "spmv_f32_max_rel_err": rel(res[torch.float32]["spmv"], res[torch.float64]["spmv"]),
        "precond_f32_max_rel_err": rel(res[torch.float32]["z"], res[torch.float64]["z"]),
        "pcg_iterations_f64_mixed": [res[torch.float64]["it"], res[torch.float32]["it"]],
        "pcg_true_rel_residual_f64_mixed": [res[torch.float64]["true_rel"], res[torch.float32]["true_rel"]],
        "pcg_solution_mixed_vs_f64_max_rel_diff": rel(res[torch.float32]["u"], res[torch.float64]["u"])})
    # the FP32 operator and the refinement (FP32 LOR smoother, as "mixed")
    out["apply_f32_max_rel_err"] = rel(op.apply_f32(x), op.apply(x))
    for scheme in ("replace", "restart"):
        u, outer, inner, _ = op.pcg_solve_ir(b, 1e-8, 1e-4, 20000, scheme=scheme)
        out["refinement_%s" % scheme] = {
            "inner_iterations": inner, "fp64_residuals": outer,
            "true_rel_residual": float((b - op.apply(u)).norm() / b.norm()),
            "solution_vs_f64_max_rel_diff": rel(u, res[torch.float64]["u"])}
    op.close()
    return out


SWEEP_KERNELS = ("setup", "assemble_f64", "assemble_f32", "apply", "apply_f32", "backward", "precond_f32")


def sweep_degree(name, dev, reps, flush, kernels=SWEEP_KERNELS, pcg=True):
    """Per-kernel timings on one p-sweep workload (about 20M DOFs): each kernel
    CUDA-event timed, median of `reps` after one warm-up, L2 flushed before
    each launch; with pcg, the time per PCG iteration (30 iterations, the
    faster of two runs) in mixed precision, in FP64 and in the refinement
    solver's inner iterations (FP32 operator)."""
    import numpy as np
    import torch

    from paper_2210_12253_gb300 import LOR
    from paper_2210_12253_gb300.inputs import workload
    from paper_2210_12253_gb300.perfmodel import FP32_PEAK_TFLOPS, FP64_PEAK_TFLOPS, hbm_peak_gbs, kernel_work

    hbm_peak, _ = hbm_peak_gbs()
    prob = workload(name)
    p = prob.p
    op = LOR(p, prob.nex, prob.ney, prob.nez, torch.tensor(prob.vertices, device=dev))
    kappa = torch.tensor(prob.kappa.reshape(-1), device=dev)
    prob.kappa = None
    x = torch.tensor(np.random.default_rng(5).standard_normal(op.ndof), device=dev)
    y, z, gx = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    gk = torch.empty(op.nqpt, dtype=torch.float64, device=dev)
    op.set_coefficient(kappa, check=True)
    op.build_pattern_internal()
    op.assemble_internal(torch.float32)
    lam = op.precond_setup("cheb", torch.float32, degree=3, power_iters=20)
    calls = {
        "setup": lambda: op.set_coefficient(kappa),
        "assemble_f64": lambda: op.assemble_internal(torch.float64),
        "assemble_f32": lambda: op.assemble_internal(torch.float32),
        "apply": lambda: op.apply(x, out=y),
        "apply_f32": lambda: op.apply_f32(x, out=y),
        "backward": lambda: op.apply_backward(x, x, gx_out=gx, gk_out=gk),
        "precond_f32": lambda: op.precond_apply(x, out=z),
    }
    res = {"p": p, "elements": op.nel, "ndof": op.ndof, "nnz": op.nnz, "lambda_max": lam}
    for kname in kernels:
        fn = calls[kname]
        fn()
        times = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = statistics.median(times)
        kind = {"assemble_f64": "assemble", "assemble_f32": "assemble", "precond_f32": "precond"}.get(kname, kname)
        vb = 4 if kname.endswith("f32") else 8
        flops, nbytes = kernel_work(kind, p, op.ndof, op.nel, op.nnz, vbytes=vb, degree=3)
        res[kname] = {"ms": ms, "gdofs": op.ndof / (ms * 1e-3) / 1e9,
                      "frac_hbm": nbytes / (ms * 1e-3) / 1e9 / hbm_peak}
        if kname.endswith("f32") and kname != "precond_f32":  # FP32 flops against the FP32 peak
            res[kname]["frac_fp32"] = flops / (ms * 1e-3) / 1e12 / FP32_PEAK_TFLOPS
        elif kind in ("apply", "backward"):
            res[kname].update(fixed_point_fields(kind, p, op.nel, flops, ms))
        else:
            res[kname]["frac_fp64"] = flops / (ms * 1e-3) / 1e12 / FP64_PEAK_TFLOPS
    if pcg:
        # PCG per iteration (30 iterations from x0 = 0, fixed count), mixed
        # precision and FP64, with the same lambda_max
        b = torch.tensor(prob.rhs, device=dev)
        for tag, dt in (("pcg_mixed", torch.float32), ("pcg_f64", torch.float64), ("pcg_ir", torch.float32)):
            op.precond_setup("cheb", dt, degree=3, lambda_max=lam)
            if tag == "pcg_ir":
                def solve(k):
                    _, _, inner, _ = op.pcg_solve_ir(b, 1e-30, 1e-4, k, raise_on_noconv=False)
                    return inner
            else:
                def solve(k):
                    return op.pcg_solve(b, 1e-30, k, raise_on_noconv=False)[1]
            solve(3)
            ms_it = float("inf")
            for _ in range(2):  # the faster of two runs (a one-off stall of ~0.2 s was seen once per process)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                its = solve(30)
                e1.record()
                torch.cuda.synchronize()
                ms_it = min(ms_it, e0.elapsed_time(e1) / its)
            res[tag] = {"ms_per_iteration": ms_it, "gdofs_iterations": op.ndof / (ms_it * 1e-3) / 1e9}
        del b
    op.close()
    del op, kappa, x, y, z, gx, gk
    torch.cuda.empty_cache()
    return res


def run_sweep(args, dev):
    """Per-kernel GDOF/s versus p at about 20M DOFs (p = 2..10, seed 4): one
    JSON object per degree (setup, FP64 and FP32 assembly, apply, backward
    (the kappa-gradient kernel), one FP32 Chebyshev-Jacobi degree-3
    application), CUDA-event timed, median of `--sweep-reps` after one
    warm-up, L2 flushed before each launch, and the FP32-arithmetic apply;
    then the time per PCG iteration (30 iterations, the faster of two runs)
    in mixed precision, in FP64 and in the refinement solver's inner
    iterations (FP32 operator)."""
    import torch

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    out = []
    for name in args.sweep_workloads or ["c5_p%d" % p for p in args.sweep_p]:
        res = sweep_degree(name, dev, args.sweep_reps, flush)
        print(json.dumps(res), flush=True)
        out.append(res)
    return out


def run_sweep_compact(args, dev):
    """The p-sweep's kernels (no PCG) at p = --c5-p (default 2, 4, 6, 8, 10),
    each about 20M DOFs, 3 timed launches per kernel: GDOF/s per kernel and
    degree, and the FP64 kernels' fraction of the FP64 peak."""
    import torch

    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    rows = [sweep_degree("c5_p%d" % p, dev, 3, flush, pcg=False) for p in args.c5_p]
    del flush
    torch.cuda.empty_cache()
    out = {"workloads": "c5 p-sweep: unit cube, n_e = round(20e6^(1/3)/p) per axis (19.9-20.6M DOFs), "
                        "+-10% h jitter (seed 4), kappa lognormal(0,1); median of 3 launches, L2 flushed",
           "p": [r["p"] for r in rows], "ndof": [r["ndof"] for r in rows]}
    for k in SWEEP_KERNELS:
        out[k + "_gdofs"] = [round(r[k]["gdofs"], 4) for r in rows]
    out["assemble_f64_frac_fp64"] = [round(r["assemble_f64"]["frac_fp64"], 3) for r in rows]
    for k in ("apply", "backward"):
        out[k + "_int_mad_frac"] = [round(r[k]["int_mad_frac"], 3) for r in rows]
        out[k + "_frac_fp64_equiv"] = [round(r[k]["frac_fp64_equiv"], 3) for r in rows]
    out["precond_f32_frac_hbm"] = [round(r["precond_f32"]["frac_hbm"], 3) for r in rows]
    return out


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)
REFERENCE_BUDGET_S = 150.0  # the whole --impl reference run (warm-up and timed steps)


def sample_desc(ne):
    n = 4 * ne + 1
    return ("%dx%dx%d elements, p=4 (%s DOFs): the 16^3 p=4 workload's recipe on a sub-box of %d^3 elements "
            "(seed 1)" % (ne, ne, ne, format(n ** 3, ","), ne))


def oracle_step(sample):
    """One pass of the oracle over the sample: LOR assembly (which also forms
    the geometry), high-order apply, Chebyshev-Jacobi (degree 3) and the
    backward of the apply.  Returns DOFs processed."""
    import oracle
    prob, mesh, x, gy, lam = sample
    p, q = prob.p, prob.q
    csr = oracle.lor_assemble(mesh, p, q, prob.kappa, True)
    oracle.ho_apply(mesh, p, q, prob.kappa, x)
    oracle.chebyshev(*csr, prob.rhs, 3, lam / 30, 1.1 * lam)
    oracle.ho_apply_backward(mesh, p, q, prob.kappa, x, gy)
    return prob.ndof


def make_sample(ne=8, seed=1):
    import numpy as np

    import oracle
    from paper_2210_12253_gb300.inputs import make_problem
    prob = make_problem("sample", ne, ne, ne, 4, seed=seed, kappa="lognormal", rhs="normal")
    mesh = oracle.Mesh(ne, ne, ne, prob.vertices)
    rng = np.random.default_rng(100)
    x, gy = rng.standard_normal(prob.ndof), rng.standard_normal(prob.ndof)
    csr = oracle.lor_assemble(mesh, prob.p, prob.q, prob.kappa, True)
    lam = oracle.power_lambda_max(*csr, np.ones(prob.ndof), 20)
    return prob, mesh, x, gy, lam


def reference_box(steps, warmup, step_s, ne=8, budget_s=None):
    """Edge (in elements) of the sub-box each reference step processes: the
    largest of ne, ne/2, ... (at least 2) whose estimated run, (steps +
    warmup) steps at step_s measured on the ne^3 box and scaled by the
    element count, fits the budget (REFERENCE_BUDGET_S by default)."""
    budget_s = REFERENCE_BUDGET_S if budget_s is None else budget_s
    while ne > 2 and (steps + warmup) * step_s > budget_s:
        nxt = max(2, ne // 2)
        step_s *= (nxt / ne) ** 3
        ne = nxt
    return ne


_BARRIER = None


def _pool_init(barrier):
    global _BARRIER
    _BARRIER = barrier


def _oracle_worker(args):
    """One process of the all-cores leg: its own sub-box of the recipe (seed
    1 + w), the oracle's step repeated for `seconds` after all workers met."""
    w, seconds = args
    sample = make_sample(8, seed=1 + w)
    _BARRIER.wait()
    t0 = time.perf_counter()
    dofs = n = 0
    while True:
        dofs += oracle_step(sample)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return dofs, time.perf_counter() - t0, n


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_kernel_rates(seconds_each=2.0):
    """The oracle's rate per kernel on one core, on a 6^3-element sub-box of
    the 32^3 p = 6 PCG workload's recipe (seed 2): LOR assembly, high-order
    apply, and one PCG iteration (FP64 operator, Chebyshev-Jacobi degree 3);
    each repeated for at least `seconds_each`.  The PCG rate is also given as
    the implied seconds per iteration at 7,189,057 DOFs (scaled by the DOF
    count from the sub-box, where the oracle's per-iteration work is linear)."""
    import numpy as np

    import oracle
    from paper_2210_12253_gb300.inputs import make_problem
    ne, p = 6, 6
    prob = make_problem("sample_c3", ne, ne, ne, p, seed=2, kappa="lognormal", rhs="normal")
    mesh = oracle.Mesh(ne, ne, ne, prob.vertices)
    q = p + 2
    x = np.random.default_rng(101).standard_normal(prob.ndof)
    csr = oracle.lor_assemble(mesh, p, q, prob.kappa, True)
    lam = oracle.power_lambda_max(*csr, np.ones(prob.ndof), 20)

    def rate(fn):
        t0 = time.perf_counter()
        n = 0
        while True:
            units = fn()
            n += units
            if time.perf_counter() - t0 >= seconds_each:
                break
        return n / (time.perf_counter() - t0)

    def pcg_iters():
        _, it, _, _ = oracle.pcg(mesh, p, q, prob.kappa, csr, prob.rhs, 1e-30, 3, oracle.PRECOND_CHEB, 3,
                                 lam / 30, 1.1 * lam, raise_on_noconv=False)
        return it
    asm = rate(lambda: (oracle.lor_assemble(mesh, p, q, prob.kappa, True), prob.ndof)[1])
    app = rate(lambda: (oracle.ho_apply(mesh, p, q, prob.kappa, x), prob.ndof)[1])
    its = rate(pcg_iters)
    return {"sample": "%d^3 elements, p=%d (%s DOFs), the 32^3 p=6 recipe (seed 2); one core" %
                      (ne, p, format(prob.ndof, ",")),
            "lor_assemble_gdofs": asm / 1e9, "ho_apply_gdofs": app / 1e9,
            "pcg_iteration_gdofs": its * prob.ndof / 1e9,
            "pcg_s_per_iteration_at_7189057_dofs": 7189057 / (its * prob.ndof)}


def cpu_baseline(seconds):
    """The oracle timed on the host: its step (LOR assembly, apply,
    Chebyshev-Jacobi, backward) on an 8^3-element sub-box of the step
    workload's recipe, on one core and then on every core the process may
    use (one independent sub-box per core in a spawned process pool, started
    together; value = all DOFs / the slowest worker's time), plus the
    per-kernel rates of oracle_kernel_rates."""
    import multiprocessing as mp
    sample = make_sample()
    t0 = time.perf_counter()
    dofs = 0
    n = 0
    while True:
        dofs += oracle_step(sample)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    one = {"value": dofs / dt / 1e9, "cores": 1, "steps": n, "seconds": dt}
    cores = host_cores()
    ctx = mp.get_context("spawn")  # after GPU work: never fork this process
    barrier = ctx.Barrier(cores)
    with ctx.Pool(cores, initializer=_pool_init, initargs=(barrier,)) as pool:
        res = pool.map(_oracle_worker, [(w, seconds) for w in range(cores)])
    all_dofs = sum(r[0] for r in res)
    slowest = max(r[1] for r in res)
    return {"value": all_dofs / slowest / 1e9, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": sample_desc(8) + "; on %d cores: one independent sub-box per core (spawned process pool, "
                      "seeds 1..%d), %d oracle steps in %.1f s (slowest worker), single-threaded FP64 C per "
                      "process" % (cores, cores, sum(r[2] for r in res), slowest),
            "one_core": one, "kernels": oracle_kernel_rates()}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    sample = make_sample(8)
    t0 = time.perf_counter()
    oracle_step(sample)  # the first warm-up step, timed to size the sample
    ne = reference_box(args.steps, args.warmup, time.perf_counter() - t0)
    warm = args.warmup - 1
    if ne != 8:
        sample, warm = make_sample(ne), args.warmup
    for _ in range(warm):
        oracle_step(sample)
    t0 = time.perf_counter()
    dofs = 0
    for _ in range(args.steps):
        dofs += oracle_step(sample)
    dt = time.perf_counter() - t0
    value = dofs / dt / 1e9
    desc = sample_desc(ne)
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": STEP_WORKLOAD + " recipe, bounded sample: " + desc,
                       "step": "oracle: LOR assembly + HO apply + Chebyshev-Jacobi deg 3 + apply backward"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": desc + "; the sub-box is the largest of 8^3, 4^3, 2^3 elements whose "
                                              "%d steps fit about %d s" % (args.steps + args.warmup,
                                                                           REFERENCE_BUDGET_S)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["liblor", "reference"], default="liblor")
    ap.add_argument("--no-pcg", action="store_true", help="skip the 32^3 p=6 PCG comparison")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-grad", action="store_true", help="skip the 24^3 p=5 adjoint-gradient timing")
    ap.add_argument("--no-hcurl", action="store_true", help="skip the discrete-gradient / vertex-coordinate timing")
    ap.add_argument("--no-general", action="store_true", help="skip the general-mesh (element-restriction) timing")
    ap.add_argument("--no-precision", action="store_true", help="skip the mixed-precision error report")
    ap.add_argument("--no-comparator", action="store_true",
                    help="skip the macro-element vs unstructured LOR assembly comparison")
    ap.add_argument("--no-helmholtz", action="store_true",
                    help="skip the definite Helmholtz (reaction term) step on the 16^3 p=4 workload")
    ap.add_argument("--cpu-seconds", type=float, default=8.0,
                    help="seconds of each oracle leg (one core, then all cores)")
    ap.add_argument("--no-c5", action="store_true", help="skip the compact p-sweep (kernels only) at ~20M DOFs")
    ap.add_argument("--c5-p", type=int, nargs="*", default=[2, 4, 6, 8, 10],
                    help="degrees of the compact p-sweep in the default line")
    ap.add_argument("--pcg-maxit", type=int, default=20000,
                    help="iteration cap of the PCG comparison (a small cap is for profiling only)")
    ap.add_argument("--pcg-only", action="store_true", help="run only the PCG comparison (profiling)")
    ap.add_argument("--ir-inner-rtol", type=float, default=1e-4,
                    help="inner tolerance of the mixed-precision iterative refinement")
    ap.add_argument("--ir-sweep", type=float, nargs="*", default=None,
                    help="also time the refinement at these inner tolerances")
    ap.add_argument("--pcg-degrees", type=int, nargs="*", default=None,
                    help="also solve with these Chebyshev degrees (supplementary degree trade-off)")
    ap.add_argument("--sweep", action="store_true", help="per-kernel throughput versus p at ~20M DOFs")
    ap.add_argument("--sweep-p", type=int, nargs="*", default=list(range(2, 11)))
    ap.add_argument("--sweep-reps", type=int, default=5)
    ap.add_argument("--sweep-workloads", nargs="*", default=None,
                    help="run the sweep's kernel set on these named workloads instead (e.g. c4_24x24x24_p5)")
    ap.add_argument("--apply-kernels", type=int, nargs=2, default=None, metavar=("NEX", "P"),
                    help="time only the FP64 and FP32 high-order applies on an NEX^3 cube of degree P "
                         "(a small case for kernel profiling)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    rank, world, local_rank = dist_info()
    if args.impl == "reference":
        out = run_reference(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return 0
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    if args.sweep:
        import torch
        from paper_2210_12253_gb300.build import build
        build()
        torch.cuda.set_device(local_rank)
        run_sweep(args, torch.device("cuda", local_rank))
        return 0
    if args.apply_kernels:
        import torch
        from paper_2210_12253_gb300.build import build
        build()
        torch.cuda.set_device(local_rank)
        print(json.dumps(run_apply_kernels(args, torch.device("cuda", local_rank))))
        return 0
    if args.pcg_only:
        import torch
        from paper_2210_12253_gb300.build import build
        build()
        torch.cuda.set_device(local_rank)
        print(json.dumps({"pcg": run_pcg(args, torch.device("cuda", local_rank), rank)}))
        return 0
    out = run_gpu(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
