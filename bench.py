#!/usr/bin/env python3
"""Benchmark of the spline hot path on GB300: fit + uniform-grid evaluation.

Workload (one step): one instance of n = M = 10^7 knots/queries, the benchmark curve of
arXiv 2001.09253 section "Curve Interpolation" (seed 1; see paper_2001_09253_gb300/synth.py),
natural ends, FP64 on the GPU.  Inputs and outputs (320 MB) exceed the 129 MB L2, so no
explicit flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own instance (instance id = rank): weak scaling, no
collective on the data path (a barrier and a max-reduction of the timings only).
`--impl reference` times the FP64 CPU oracle on the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "instances/sec and GB/s (% roofline) at fixed oracle error; p50/p99 latency"
N_POINTS = 10_000_000
SEED = 1
# Algorithmic work per point (knot and query, M = n), from the paper's own operation counts:
#   fit, forward row ("Implementation" listing): 14 flops incl. 2 divisions; back substitution: 2;
#   query position x_0 + k*step: 2;  newint ("Fast Interpolation"): 19 flops + 1 division.
FLOPS_PER_POINT = 14 + 2 + 2 + 20
# Algorithmic bytes per point: read x, y (16 B), write y'' and S(x_k) (16 B).
BYTES_PER_POINT = 32
# FP64 peak from the unit counts: the nominal 1.25 TFLOP/s of GB300 is 2 FP64 lanes/clk/SM x
# 152 SMs x 2.07 GHz with an FMA counted as 2 flops.  The path's operations are mostly separate
# adds and multiplies, so the roofline counts FP64 operations at one per lane per clock:
# 2 x 152 x 2.07e9 = 0.629e12 op/s (an FMA-counted peak would cap this algorithm near 55%).
PEAK_FP64_OPS_T = 2 * 152 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 1.25
KERNEL_SRC = os.path.join(ROOT, "paper_2001_09253_gb300", "csrc", "spl_fused_f64.cu")
PROFILE = os.path.join(ROOT, "profiles", "fused_f64_n1e7.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--n", type=int, default=N_POINTS, help="knots = queries per instance (profiling runs)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_hash() -> str:
    with open(KERNEL_SRC, "rb") as f:
        h = hashlib.sha256(f.read())
    with open(os.path.join(ROOT, "paper_2001_09253_gb300", "csrc", "spl_device.cuh"), "rb") as f:
        h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic():
    """DRAM bytes per launch of the dominant kernel from the committed ncu summary, or None
    when the summary is absent or was taken on a different version of the kernel source."""
    try:
        text = open(PROFILE).read()
    except OSError:
        return None
    mh = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    mb = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", text)
    if not mh or not mb or mh.group(1) != kernel_hash():
        return None
    return float(mb.group(1))


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.25)

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [v.strip() for v in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out = {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                   "samples": len(sm)}
        return out


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_max(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if torch.cuda.is_available() else torch.device("cpu")
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_oracle_rate(min_seconds=10.0, max_reps=30):
    """The FP64 oracle, as it stands, single-threaded on this host, on the same instance."""
    import oracle
    from paper_2001_09253_gb300 import synth
    x, y = synth.curve(SEED, N_POINTS)
    oracle.fit_eval(x[:1000], y[:1000])  # build/load outside the timing
    reps, t0 = 0, time.perf_counter()
    while True:
        r = oracle.fit_eval(x, y, oracle.NATURAL, oracle.NATURAL, N_POINTS)
        assert r["status"] == oracle.OK
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds or reps >= max_reps:
            break
    return reps / el, reps, el


def run_reference(args, world, rank):
    if rank != 0:
        return
    warm, steps = max(args.warmup, 0), max(args.steps, 1)
    import oracle
    from paper_2001_09253_gb300 import synth
    x, y = synth.curve(SEED, N_POINTS)
    for _ in range(min(warm, 1)):
        oracle.fit_eval(x, y, oracle.NATURAL, oracle.NATURAL, N_POINTS)
    # each step is one full instance; capped so the run stays within a few minutes
    steps = min(steps, 60)
    t0 = time.perf_counter()
    for _ in range(steps):
        r = oracle.fit_eval(x, y, oracle.NATURAL, oracle.NATURAL, N_POINTS)
        assert r["status"] == oracle.OK
    el = time.perf_counter() - t0
    v = steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "instances/s", "n_gpus": args.gpus,
        "steps": steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fit+eval, n=M=1e7, seed 1, natural ends", "n": N_POINTS, "m": N_POINTS,
                   "instances_per_step": 1},
        "cpu_baseline": {"value": v, "unit": "instances/s", "cores": 1, "kind": "oracle",
                         "sample": "%d full n=1e7 instances, single thread" % steps},
        "e2e": {"value": v, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "points_per_s": v * N_POINTS, "ns_per_point": 1e9 / (v * N_POINTS),
    }
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local):
    import torch
    from paper_2001_09253_gb300 import spl
    assert torch.cuda.is_available(), "the benchmark needs a CUDA device"
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    K, W = max(args.steps, 1), max(args.warmup, 3)
    n = m = int(args.n)
    window = 64
    ring = 160 << 20  # per-launch scratch bound (the FP64 ring is ~80 MB on 152 SMs)
    arena = (min(window, K) + 2) * ring
    if not args.no_e2e:
        arena += 10 * (32 * n + ring)  # host-buffer leg: staged inputs/outputs, 8 in flight
    ctx = spl.Context(device=local, stream=stream, arena_bytes=int(arena), max_slots=4096)
    plan = ctx.plan(max_n=n, precision=spl.PREC_F64)
    with torch.cuda.stream(stream):
        x, y = spl.generate_curve(SEED, n, instance=rank, device=local, stream=stream)
        ypp = torch.empty(n, dtype=torch.float64, device=dev)
        yq = torch.empty(m, dtype=torch.float64, device=dev)
    stream.synchronize()

    def step():
        return ctx.submit(plan, x, y, spl.NATURAL, spl.NATURAL, m, ypp, yq)

    for _ in range(W):
        s, _ = ctx.wait(step(), 120.0)
        assert s == spl.OK, spl.status_str(s)
    clocks = Clocks(local)
    st0 = ctx.stats()
    barrier(world)
    torch.cuda.synchronize(dev)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    pending, dev_ms = [], []
    for _ in range(K):
        pending.append(step())
        if len(pending) >= window:
            s, r = ctx.wait(pending.pop(0), 120.0)
            assert s == spl.OK
            dev_ms.append(r.device_ms)
    e1.record(stream)
    for t in pending:
        s, r = ctx.wait(t, 120.0)
        assert s == spl.OK
        dev_ms.append(r.device_ms)
    torch.cuda.synchronize(dev)
    ck = clocks.stop()
    st1 = ctx.stats()
    barrier(world)
    t_ms = reduce_max(world, e0.elapsed_time(e1))
    launches = st1["kernel_launches"] - st0["kernel_launches"]
    value = world * K / (t_ms / 1e3)
    ms_step = t_ms / K
    achieved_tflops = FLOPS_PER_POINT * n / (ms_step * 1e-3) / 1e12
    gbs = BYTES_PER_POINT * n / (ms_step * 1e-3) / 1e9

    if args.no_e2e:
        if rank == 0:
            print(json.dumps({"profile_run": True, "n": n, "steps": K, "ms_per_step": ms_step,
                              "roofline_frac": achieved_tflops / PEAK_FP64_OPS_T, "gpu_launches": int(launches)}))
        ctx.close()
        return
    # end to end through the C ABI with pinned host buffers: H2D of x, y and D2H of y'', S(x_k)
    hx = x.cpu().pin_memory()
    hy = y.cpu().pin_memory()
    hypp = torch.empty(n, dtype=torch.float64).pin_memory()
    hyq = torch.empty(m, dtype=torch.float64).pin_memory()
    Ke = min(K, 100)
    for _ in range(2):
        s, _ = ctx.wait(ctx.submit(plan, hx, hy, spl.NATURAL, spl.NATURAL, m, hypp, hyq), 120.0)
        assert s == spl.OK
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    pend = []
    for _ in range(Ke):
        pend.append(ctx.submit(plan, hx, hy, spl.NATURAL, spl.NATURAL, m, hypp, hyq))
        if len(pend) >= 8:
            s, _ = ctx.wait(pend.pop(0), 120.0)
            assert s == spl.OK
    for t in pend:
        s, _ = ctx.wait(t, 120.0)
        assert s == spl.OK
    torch.cuda.synchronize(dev)
    te = reduce_max(world, time.perf_counter() - t0)
    e2e_value = world * Ke / te

    if rank != 0:
        ctx.close()
        return
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        rate, reps, el = cpu_oracle_rate()
        cpu = {"value": rate, "unit": "instances/s", "cores": 1, "kind": "oracle",
               "sample": "%d full n=1e7 instances (%.1f s), single thread" % (reps, el)}
    pk = measured_peaks()
    lat = sorted(dev_ms)
    line = {
        "metric": METRIC, "value": value, "unit": "instances/s", "n_gpus": world, "steps": K, "warmup": W,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "fit+eval, n=M=1e7, seed 1, natural ends, plain FP64", "n": n, "m": m,
                   "instances_per_step": 1, "l2": "inputs+outputs 320 MB > 129 MB L2, no flush",
                   "parallelism": "one instance per GPU"},
        "points_per_s": value * n, "gb_per_s": gbs,
        "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                       "what": "device time per step (events around each launch, %d in flight)" % window},
        "roofline": {"bound": "alu", "achieved": achieved_tflops, "peak": PEAK_FP64_OPS_T, "unit": "TFLOP/s",
                     "frac": achieved_tflops / PEAK_FP64_OPS_T, "traffic": profiled_traffic(),
                     "what": ("FP64 pipe: %d algorithmic FP64 ops/point (paper's counts, a division = 1) per second; "
                              "peak = 2 FP64 ops/clk/SM x 152 SMs x 2.07 GHz (one op per lane per clock)"
                              % FLOPS_PER_POINT),
                     "frac_of_fma_counted_peak": achieved_tflops / PEAK_FP64_TFLOPS,
                     "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / pk["hbm_gbs"] if pk.get("hbm_gbs") else None},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": "instances/s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 16 * n + 4},
        "gpu_launches": int(launches),
        "clocks": ck,
    }
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    args = parse()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
