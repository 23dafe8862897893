#!/usr/bin/env python3
"""Benchmark of the spline hot path on GB300: fit + uniform-grid evaluation.

Main line (one step): one instance of n = M = 10^7 knots/queries, the benchmark curve of
arXiv 2001.09253 section "Curve Interpolation" (seed 1; see paper_2001_09253_gb300/synth.py),
natural ends, plain FP64 on the GPU.  Inputs and outputs (320 MB) exceed the 129 MB L2, so no
explicit flush is needed between steps.  The same JSON line also carries, under
"other_configs", the mixed-precision path on the same instance (binary32 solve and cubic,
without and with one refinement step) and the batched workload (4096 instances, sizes
log-uniform in [1e2, 1e5], seed 2, one persistent launch replayed from a CUDA graph), and,
in the CPU-baseline leg, the error of every GPU result against the FP64 oracle.

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
WORKLOAD = "fit+eval, n=M=1e7, seed 1, natural ends, plain FP64"
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
TOL = {"f64": 1e-12, "mixed": 1e-5}
CSRC = os.path.join(ROOT, "paper_2001_09253_gb300", "csrc")
PROFILES = {
    "f64": (os.path.join(ROOT, "profiles", "fused_f64_n1e7.md"), ["spl_fused_f64.cu", "spl_device.cuh"]),
    "mixed": (os.path.join(ROOT, "profiles", "mixed_scan_n1e7.md"),
              ["spl_mixed_scan.cu", "spl_mixed_math.cuh", "spl_device.cuh", "spl_numeric.h"]),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--only", default="", choices=["", "f64", "mixed", "mixed-refine", "batched", "variants", "dfma", "serving", "latency",
                                                   "schedule", "n1000", "noalloc"],
                    help="time one path only and print a short line (profiling runs)")
    ap.add_argument("--n", type=int, default=N_POINTS, help="knots = queries per instance (profiling runs)")
    ap.add_argument("--no-serving", action="store_true",
                    help="skip the serving leg (launch-list captures: its persistent loop waits on the host, "
                         "which a profiler that serialises launches would stall)")
    return ap.parse_args()


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def kernel_hash(files) -> str:
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(CSRC, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_field(which: str, key: str):
    """A number recorded as `key: value` in the kernel's committed ncu summary, or None when the
    summary is absent, lacks it, or was taken on a different version of the kernel sources."""
    path, files = PROFILES[which]
    try:
        text = open(path).read()
    except OSError:
        return None
    mh = re.search(r"kernel_source_hash:\s*([0-9a-f]+)", text)
    mv = re.search(r"^" + re.escape(key) + r":\s*([0-9.eE+-]+)", text, re.M)
    if not mh or not mv or mh.group(1) != kernel_hash(files):
        return None
    try:
        return float(mv.group(1))
    except ValueError:
        return None


def profiled_traffic(which: str):
    """DRAM bytes per launch of the kernel (ncu: dram__bytes_read.sum + dram__bytes_write.sum)."""
    return profiled_field(which, "dram_bytes_per_launch_full_size")


def profiled_fraction(which: str, key: str):
    """A percentage counter of the committed ncu summary as a fraction, or None."""
    v = profiled_field(which, key)
    return None if v is None else v / 100.0


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


def pct(vals, q):
    s = sorted(vals)
    return s[min(len(s) - 1, int(q * len(s)))] if s else None


def dist_summary(a):
    """A timing distribution as the paper reports its own (section "Curve Interpolation": no single
    central value describes such timings): median with the 16th/84th percentiles, the tail, the
    10 % trimmed mean."""
    a = np.asarray(a, dtype=np.float64)
    if a.size == 0:
        return None
    lo_, hi_ = np.quantile(a, [0.1, 0.9])
    trimmed = a[(a >= lo_) & (a <= hi_)]
    return {"count": int(a.size), "min": float(a.min()), "p16": float(np.quantile(a, 0.16)),
            "median": float(np.median(a)), "p84": float(np.quantile(a, 0.84)), "p99": float(np.quantile(a, 0.99)),
            "trimmed_mean_10": float(trimmed.mean()), "mean": float(a.mean()), "std": float(a.std())}


# ------------------------------------------------------------------ reference arm (oracle)

def run_reference(args, world, rank):
    if rank != 0:
        return
    warm, steps = max(args.warmup, 0), max(args.steps, 1)
    import oracle
    from paper_2001_09253_gb300 import synth
    x, y = synth.curve(SEED, N_POINTS)
    for _ in range(min(warm, 1)):
        oracle.fit_eval(x, y, oracle.NATURAL, oracle.NATURAL, N_POINTS)
    steps = min(steps, 60)  # each step is one full instance; keeps the run within a few minutes
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
        "config": {"workload": WORKLOAD, "n": N_POINTS, "m": N_POINTS, "instances_per_step": 1,
                   "l2": "inputs+outputs 320 MB > 129 MB L2, no flush", "parallelism": "one instance per GPU"},
        "cpu_baseline": {"value": v, "unit": "instances/s", "cores": 1, "kind": "oracle",
                         "sample": "%d full n=1e7 instances, single thread" % steps},
        "e2e": {"value": v, "unit": "instances/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "points_per_s": v * N_POINTS, "ns_per_point": 1e9 / (v * N_POINTS),
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

class Runner:
    def __init__(self, args, world, rank, local):
        import torch
        from paper_2001_09253_gb300 import spl
        assert torch.cuda.is_available(), "the benchmark needs a CUDA device"
        self.torch, self.spl = torch, spl
        self.args, self.world, self.rank, self.local = args, world, rank, local
        torch.cuda.set_device(local)
        self.dev = torch.device("cuda", local)
        self.stream = torch.cuda.Stream(self.dev)
        self.K, self.W = max(args.steps, 1), max(args.warmup, 3)
        self.n = int(args.n)
        self.window = 16  # launches in flight: enough to keep the device busy
        ring = 512 << 20  # per-launch scratch bound (FP64 tile scratch ~330 MB at n = 1e7, binary32 scratch less)
        arena = (min(self.window, self.K) + 2) * (ring + 4 * self.n)
        if not args.no_e2e:
            arena += 10 * (32 * self.n + ring)  # host-buffer leg: staged inputs/outputs, 8 in flight
        if not args.only or args.only in ("batched", "serving"):
            arena += 2 << 30  # batched workload and serving scratch
        self.ctx = spl.Context(device=local, stream=self.stream, arena_bytes=int(arena), max_slots=8192)
        with torch.cuda.stream(self.stream):
            self.x, self.y = spl.generate_curve(SEED, self.n, instance=rank, device=local, stream=self.stream)
        self.stream.synchronize()

    def plan(self, precision, refine=0, max_n=None):
        return self.ctx.plan(max_n=max_n or self.n, precision=precision, refine_steps=refine)

    def time_single(self, plan, with_clocks=False):
        """K steps of one instance on the device, W untimed warm-ups; events on the launch stream."""
        torch, spl = self.torch, self.spl
        n = m = self.n
        ypp = torch.empty(n, dtype=torch.float64, device=self.dev)
        yq = torch.empty(m, dtype=torch.float64, device=self.dev)

        def step():
            return self.ctx.submit(plan, self.x, self.y, spl.NATURAL, spl.NATURAL, m, ypp, yq)

        for _ in range(self.W):
            s, _ = self.ctx.wait(step(), 120.0)
            assert s == spl.OK, spl.status_str(s)
        clocks = Clocks(self.local) if with_clocks else None
        st0 = self.ctx.stats()
        barrier(self.world)
        torch.cuda.synchronize(self.dev)
        if clocks:
            clocks.start()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        pending, dev_ms = [], []
        for _ in range(self.K):
            pending.append(step())
            if len(pending) >= self.window:
                s, r = self.ctx.wait(pending.pop(0), 120.0)
                assert s == spl.OK
                dev_ms.append(r.device_ms)
        e1.record(self.stream)
        for t in pending:
            s, r = self.ctx.wait(t, 120.0)
            assert s == spl.OK
            dev_ms.append(r.device_ms)
        torch.cuda.synchronize(self.dev)
        ck = clocks.stop() if clocks else None
        st1 = self.ctx.stats()
        barrier(self.world)
        t_ms = reduce_max(self.world, e0.elapsed_time(e1))
        return {"ms_per_step": t_ms / self.K, "value": self.world * self.K / (t_ms / 1e3),
                "launches": st1["kernel_launches"] - st0["kernel_launches"],
                "p50_ms": pct(dev_ms, 0.5), "p99_ms": pct(dev_ms, 0.99), "clocks": ck,
                "ypp": ypp, "yq": yq}

    def time_e2e(self, plan):
        """Same metric through the C ABI with pinned host buffers (H2D of x, y and D2H of
        y'' and S(x_k) inside the timed region), host wall clock."""
        torch, spl = self.torch, self.spl
        n = m = self.n
        hx = self.x.cpu().pin_memory()
        hy = self.y.cpu().pin_memory()
        hypp = torch.empty(n, dtype=torch.float64).pin_memory()
        hyq = torch.empty(m, dtype=torch.float64).pin_memory()
        Ke = min(self.K, 100)
        for _ in range(2):
            s, _ = self.ctx.wait(self.ctx.submit(plan, hx, hy, spl.NATURAL, spl.NATURAL, m, hypp, hyq), 120.0)
            assert s == spl.OK
        barrier(self.world)
        torch.cuda.synchronize(self.dev)
        t0 = time.perf_counter()
        pend = []
        for _ in range(Ke):
            pend.append(self.ctx.submit(plan, hx, hy, spl.NATURAL, spl.NATURAL, m, hypp, hyq))
            if len(pend) >= 8:
                s, _ = self.ctx.wait(pend.pop(0), 120.0)
                assert s == spl.OK
        for t in pend:
            s, _ = self.ctx.wait(t, 120.0)
            assert s == spl.OK
        torch.cuda.synchronize(self.dev)
        te = reduce_max(self.world, time.perf_counter() - t0)
        return {"value": self.world * Ke / te, "unit": "instances/s", "h2d_bytes_per_step": 16 * n,
                "d2h_bytes_per_step": 16 * n + 4, "steps": Ke}

    def batched(self, count=4096, lo=1e2, hi=1e5, seed=2, steps=None):
        """4096 independent instances, one persistent launch per step replayed from a CUDA graph."""
        torch, spl = self.torch, self.spl
        from paper_2001_09253_gb300 import synth
        sizes = synth.sizes_loguniform(seed, count, lo, hi)
        total = int(sizes.sum())
        off = np.concatenate([[0], np.cumsum(sizes)])
        X = torch.empty(total, dtype=torch.float64, device=self.dev)
        Y = torch.empty(total, dtype=torch.float64, device=self.dev)
        P = torch.empty(total, dtype=torch.float64, device=self.dev)
        Q = torch.empty(total, dtype=torch.float64, device=self.dev)
        nbytes = int(self.ctx.lib.spl_generate_scratch_bytes(int(sizes.max())))
        scratch = torch.empty(max(nbytes, 8), dtype=torch.uint8, device=self.dev)
        for i, nn in enumerate(sizes):
            s = self.ctx.lib.spl_generate_curve(seed, self.rank * count + i, int(nn), X[off[i]:].data_ptr(),
                                                Y[off[i]:].data_ptr(), scratch.data_ptr(), nbytes,
                                                self.stream.cuda_stream)
            assert s == 0
        self.stream.synchronize()
        plan = self.plan(spl.PREC_F32_REFINE, 1, max_n=int(sizes.max()))
        reqs = []
        for i, nn in enumerate(sizes):
            o = int(off[i])
            reqs.append(spl.make_request(X[o:o + nn], Y[o:o + nn], spl.NATURAL, spl.NATURAL, int(nn), P[o:o + nn],
                                         Q[o:o + nn]))
        b = self.ctx.batch(plan, reqs, keep=(X, Y, P, Q))
        K = steps or max(10, min(self.K, 100))
        for _ in range(3):
            b.launch()
            assert (b.wait() == 0).all()
        st0 = self.ctx.stats()
        barrier(self.world)
        torch.cuda.synchronize(self.dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(self.stream)
        for _ in range(K):
            b.launch()
        e1.record(self.stream)
        st = b.wait()
        torch.cuda.synchronize(self.dev)
        assert (st == 0).all()
        st1 = self.ctx.stats()
        t_ms = reduce_max(self.world, e0.elapsed_time(e1))
        res = {"workload": "4096 instances, n log-uniform in [1e2, 1e5], seed 2, natural ends, M = n, "
                           "binary32 + 1 refinement step, one persistent launch pair per step from a CUDA graph",
               "instances_per_step": count, "points_per_step": total, "steps": K,
               "ms_per_step": t_ms / K, "value": self.world * count * K / (t_ms / 1e3), "unit": "instances/s",
               "gb_per_s": BYTES_PER_POINT * total / (t_ms / K * 1e-3) / 1e9,
               "gpu_launches": st1["kernel_launches"] - st0["kernel_launches"],
               "graph_launches": st1["graph_launches"] - st0["graph_launches"]}
        b.close()
        return res, (sizes, off, X, Y, P, Q)

    def _timed_submit(self, plan, m, yq, jq=None, xq=None, ypp_in=None, x=None, y=None, ypp_out=None,
                      detail=False):
        """One request bracketed by CUDA events on the context's stream; returns device ms (with
        detail: also the library's own device time of the request, from its first copy to its
        last operation, and the host wall time of submit + wait)."""
        torch, spl = self.torch, self.spl
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        w0 = time.perf_counter()
        e0.record(self.stream)
        t = self.ctx.submit(plan, self.x if x is None else x, self.y if y is None else y, spl.NATURAL,
                            spl.NATURAL, m, ypp_out, yq, jq, xq=xq, ypp_in=ypp_in)
        e1.record(self.stream)
        s, res = self.ctx.wait(t, 120.0)
        assert s == spl.OK, spl.status_str(s)
        e1.synchronize()
        wall = (time.perf_counter() - w0) * 1e3
        if detail:
            return e0.elapsed_time(e1), float(res.device_ms), wall
        return e0.elapsed_time(e1)

    def config1(self, reps=200):
        """The smallest configuration: n = M = 1,000 (seed 0), natural and clamped (-1, 1) ends,
        one request at a time through spl_submit + spl_wait, FP64 and binary32 with one refinement
        step.  Latency per request: device (the library's CUDA events around the request's stream
        work: for one instance in device memory the kernel(s) alone, the descriptor passed as a
        kernel parameter and the status written by the kernel into pinned host memory) and wall
        (host clock around the Python submit and wait), as distributions over `reps` requests after
        warm-up."""
        torch, spl = self.torch, self.spl
        from paper_2001_09253_gb300 import synth
        n = 1000
        hx, hy = synth.curve(0, n)
        x = torch.from_numpy(hx).to(self.dev)
        y = torch.from_numpy(hy).to(self.dev)
        ypp = torch.empty(n, dtype=torch.float64, device=self.dev)
        yq = torch.empty(n, dtype=torch.float64, device=self.dev)
        out = {}
        for label, prec, refine in (("f64", spl.PREC_F64, 0), ("mixed_refine1", spl.PREC_F32_REFINE, 1)):
            plan = self.ctx.plan(n, prec, refine_steps=refine)
            for bcl, (a, b) in (("natural", (spl.NATURAL, spl.NATURAL)), ("clamped", (-1.0, 1.0))):
                dev_ms, wall_ms = [], []
                for r in range(self.W + reps):
                    w0 = time.perf_counter()
                    t = self.ctx.submit(plan, x, y, a, b, n, ypp, yq)
                    st, res = self.ctx.wait(t, 60.0)
                    wl = (time.perf_counter() - w0) * 1e3
                    assert st == spl.OK, spl.status_str(st)
                    if r >= self.W:
                        dev_ms.append(float(res.device_ms))
                        wall_ms.append(wl)
                out["%s/%s" % (label, bcl)] = {"device_ms": dist_summary(dev_ms), "wall_ms": dist_summary(wall_ms)}
        return {"workload": "n = M = 1000, seed 0, natural and clamped (-1, 1) ends, one request at a time",
                "requests_per_case": reps, **out}, (hx, hy)

    def latency_by_size(self, sizes=(1_000, 10_000, 100_000, 600_000, 1_000_000), reps=50):
        """One request at a time through spl_submit + spl_wait for n = M from 1e3 to 1e6 (the
        first n points of the benchmark curve, natural ends), FP64 and binary32 with one
        refinement step: the latency paths (the multi-CTA FP64 kernel up to SMs x 9,600 knots,
        the warp-cooperative binary32 kernel) and, past them, the tiled FP64 kernel.  Device time
        per request from the library's events, as distributions."""
        torch, spl = self.torch, self.spl
        out = {}
        for label, prec, refine in (("f64", spl.PREC_F64, 0), ("mixed_refine1", spl.PREC_F32_REFINE, 1)):
            for n in sizes:
                x, y = self.x[:n].contiguous(), self.y[:n].contiguous()
                ypp = torch.empty(n, dtype=torch.float64, device=self.dev)
                yq = torch.empty(n, dtype=torch.float64, device=self.dev)
                plan = self.ctx.plan(n, prec, refine_steps=refine)
                dev_ms = []
                for r in range(self.W + reps):
                    st, res = self.ctx.wait(self.ctx.submit(plan, x, y, spl.NATURAL, spl.NATURAL, n, ypp, yq), 60.0)
                    assert st == spl.OK, spl.status_str(st)
                    if r >= self.W:
                        dev_ms.append(float(res.device_ms))
                out["%s/n=%d" % (label, n)] = dist_summary(dev_ms)
        return {"workload": "one request at a time, n = M, the first n points of the n = 1e7 curve, natural ends",
                "unit": "ms (device, per request)", "requests_per_case": reps, **out}

    def noalloc(self, sizes=(100_000, 1_000_000), reps=20):
        """spl_fit_eval_noalloc (binary32 + one refinement step, fixed scratch inside the library,
        no allocation) beside spl_submit with the same precision, one instance of n = M at a
        time; device time from CUDA events around each call."""
        torch, spl = self.torch, self.spl
        out = {}
        for n in sizes:
            x, y = self.x[:n].contiguous(), self.y[:n].contiguous()
            ypp = torch.empty(n, dtype=torch.float64, device=self.dev)
            yq = torch.empty(n, dtype=torch.float64, device=self.dev)
            plan = self.ctx.plan(n, spl.PREC_F32_REFINE, refine_steps=1)
            t_na, t_sub = [], []
            for r in range(self.W + reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(self.stream)
                s, _ = spl.fit_eval_noalloc(x, y, spl.NATURAL, spl.NATURAL, n, ypp, yq, stream=self.stream,
                                            want_status=False)
                e1.record(self.stream)
                assert s == spl.OK
                e1.synchronize()
                ms = self._timed_submit(plan, n, yq, x=x, y=y, ypp_out=ypp)
                if r >= self.W:
                    t_na.append(e0.elapsed_time(e1))
                    t_sub.append(ms)
            out["n=%d" % n] = {"noalloc_ms": dist_summary(t_na), "submit_ms": dist_summary(t_sub)}
        return {"workload": "one instance of the n = 1e7 curve's first n points, M = n, binary32 + one refinement "
                            "step: spl_fit_eval_noalloc (warp-cooperative kernels, fixed scratch) and spl_submit", **out}

    def dfma_probe(self, warps_per_sm=8, trips=6000, reps=5, clock_mhz=None):
        """The FP64 pipe's rate on a pure DFMA stream (spl_selftest_dfma: one CTA of `warps_per_sm`
        warps per SM, four independent chains per thread), timed with CUDA events: the measured
        ceiling beside the unit-count peak of the FP64 roofline.  lanes/clk/SM uses the SM clock
        sampled during the main timed region (the maximum clock when none was sampled)."""
        torch, spl = self.torch, self.spl
        sms = torch.cuda.get_device_properties(self.dev).multi_processor_count
        sink = torch.empty(sms * warps_per_sm * 32, dtype=torch.float64, device=self.dev)
        times, ops = [], 0
        for r in range(self.W + reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(self.stream)
            ops = spl.selftest_dfma(trips, warps_per_sm, sink, stream=self.stream)
            e1.record(self.stream)
            e1.synchronize()
            if r >= self.W:
                times.append(e0.elapsed_time(e1))
        ms = float(np.median(times))
        rate = ops / (ms * 1e-3)
        mhz = clock_mhz or 2070.0
        return {"lane_ops_per_s_T": rate / 1e12, "lanes_per_clk_per_sm": rate / (sms * mhz * 1e6),
                "clock_mhz": mhz, "ms": ms, "lane_ops": ops, "warps_per_sm": warps_per_sm,
                "what": "DFMA lane operations per second, %d SMs x %d warps x 4 independent chains" % (sms, warps_per_sm)}

    def eval_variants(self, reps=None):
        """The three forms of section "Fast Interpolation" that the paper benchmarks (orig: one
        reciprocal then a multiply; noinv: a division at the end; vol: orig with the reciprocal
        pinned through a volatile local) on the separate evaluation kernel, from one stored FP64
        fit of the n = 1e7 curve: M = n sorted queries (the uniform grid) and M = n unsorted ones
        (seeded uniform positions).  The variants run in a shuffled order in every repetition, as
        in the paper's benchmark; each launch is timed with CUDA events."""
        torch, spl = self.torch, self.spl
        n = self.n
        K = reps or min(self.K, 30)
        ypp = torch.empty(n, dtype=torch.float64, device=self.dev)
        self._timed_submit(self.plan(spl.PREC_F64), 0, None, ypp_out=ypp)
        rng = np.random.default_rng(4)
        lo, hi = float(self.x[0]), float(self.x[-1])
        xq = torch.from_numpy(rng.uniform(lo, hi, n)).to(self.dev)
        yq = torch.empty(n, dtype=torch.float64, device=self.dev)
        jq = torch.empty(n, dtype=torch.int32, device=self.dev)
        names = ["orig", "noinv", "vol", "noop"]
        out, samples = {}, {}
        pick = np.sort(rng.choice(n, size=20000, replace=False))
        for mode, label in ((spl.QUERY_UNIFORM, "sorted"), (spl.QUERY_EXPLICIT, "unsorted")):
            plans = [self.ctx.plan(n, spl.PREC_F64, query_mode=mode, eval_variant=v) for v in range(4)]
            times = [[] for _ in range(4)]
            q = xq if mode == spl.QUERY_EXPLICIT else None
            for rep in range(self.W + K):
                for v in rng.permutation(4):
                    ms = self._timed_submit(plans[v], n, yq, jq, xq=q, ypp_in=ypp)
                    if rep >= self.W:
                        times[v].append(ms)
                    if rep == self.W + K - 1 and v < 3:
                        samples[(label, names[v])] = (yq.cpu().numpy()[pick], jq.cpu().numpy()[pick])
            out[label] = {names[v]: {"ms": dist_summary(times[v]), "queries_per_s": n / (np.median(times[v]) * 1e-3),
                                     "reps": K} for v in range(4)}
            out[label]["fastest"] = names[int(np.argmin([np.median(t) for t in times[:3]]))]
            # the paper's reading of its control loop: evaluation cost above query generation + bracketing
            out[label]["orig_minus_noop_ms"] = float(np.median(times[0]) - np.median(times[3]))
        res = {"workload": "evaluation only from a stored FP64 fit of the n = 1e7 curve (seed 1), M = 1e7 "
                           "queries: the uniform grid (sorted) and seeded uniform positions (unsorted), "
                           "galloping brackets on the grid, bisection on unsorted positions; noop = query "
                           "generation and bracketing only (the paper's control loop)", **out}
        return res, (pick, xq.cpu().numpy()[pick], samples)

    def n_schedule(self, draws=256, seed=5):
        """The paper's schedule of curve sizes: n = round((r (sqrt(1048576) - sqrt(4)) + sqrt(4))^2)
        for r on an even grid of 524,288 points in [0, 1], shuffled (section "Curve
        Interpolation", benchmark steps 2-4); here a seeded sample of `draws` entries of it.  Per
        draw: a new benchmark curve (device generator), then the fused FP64 fit + evaluation
        (M = n) and the three evaluation forms from the stored fit, in a shuffled order, each
        timed with CUDA events.  Reported as distributions of ns per point (the paper's point
        that no single central value describes such timings), overall and by size."""
        torch, spl = self.torch, self.spl
        rng = np.random.default_rng(seed)
        r = np.linspace(0.0, 1.0, 524288)
        sizes = np.rint((r * (np.sqrt(1048576.0) - np.sqrt(4.0)) + np.sqrt(4.0)) ** 2).astype(np.int64)
        rng.shuffle(sizes)
        sizes = sizes[:draws]
        nmax = int(sizes.max())
        fused = self.ctx.plan(nmax, spl.PREC_F64)
        evals = [self.ctx.plan(nmax, spl.PREC_F64, eval_variant=v) for v in range(3)]
        X = torch.empty(nmax, dtype=torch.float64, device=self.dev)
        Y = torch.empty(nmax, dtype=torch.float64, device=self.dev)
        ypp = torch.empty(nmax, dtype=torch.float64, device=self.dev)
        yq = torch.empty(nmax, dtype=torch.float64, device=self.dev)
        names = ["fit+eval (fused)", "eval orig", "eval noinv", "eval vol"]
        ns = {k: [] for k in names}
        wall = {k: [] for k in names}
        for i, n in enumerate(sizes):
            n = int(n)
            with torch.cuda.stream(self.stream):
                x, y = spl.generate_curve(seed, n, instance=i, device=self.local, stream=self.stream)
            X[:n].copy_(x)
            Y[:n].copy_(y)
            torch.cuda.synchronize(self.dev)
            xs, ys = X[:n], Y[:n]
            for k in rng.permutation(4):
                if k == 0:
                    _, ms, wl = self._timed_submit(fused, n, yq[:n], x=xs, y=ys, ypp_out=ypp[:n], detail=True)
                else:
                    _, ms, wl = self._timed_submit(evals[k - 1], n, yq[:n], ypp_in=ypp[:n], x=xs, y=ys,
                                                   detail=True)
                ns[names[k]].append(ms * 1e6 / n)
                wall[names[k]].append(wl * 1e6 / n)
        sizes_f = sizes.astype(np.float64)

        def dist(v, mask=None):
            a = np.asarray(v)
            if mask is not None:
                a = a[mask]
            if a.size == 0:
                return None
            return dist_summary(a)

        bins = {"n<1e3": sizes_f < 1e3, "1e3<=n<1e5": (sizes_f >= 1e3) & (sizes_f < 1e5), "n>=1e5": sizes_f >= 1e5}
        out = {k: {"all": dist(v), **{b: dist(v, msk) for b, msk in bins.items()}} for k, v in ns.items()}
        out_wall = {k: {b: dist(v, msk) for b, msk in bins.items()} for k, v in wall.items()}
        return {"workload": "the paper's size schedule n = round((r (1024 - 2) + 2)^2), r on 524,288 even "
                            "points, shuffled; %d seeded draws (n from %d to %d), one new curve per draw, "
                            "routines in shuffled order" % (draws, int(sizes.min()), nmax),
                "unit": "ns per point",
                "timing": "device: the library's CUDA events around one request (fit + evaluation: the "
                          "kernel alone, the descriptor a kernel parameter and the status written into pinned "
                          "host memory; evaluation from a stored fit: status reset, descriptor copy, kernel, "
                          "status copy back); wall: host clock around the Python submit and wait (includes "
                          "the binding's marshalling and the completion poll)",
                "routines": out, "wall": out_wall}


def serving(r, pool_count=512, seed=3, lo=1e2, hi=1e6, rate=20000.0, warm_s=1.0, run_s=8.0):
    """Poisson arrivals through the continuous-batching server (persistent device loop,
    mixed precision), admission under a 150 GB HBM budget; then the same pool at saturation,
    and the plain FP64 path on the same pool for comparison."""
    torch, spl = r.torch, r.spl
    from paper_2001_09253_gb300 import synth
    sizes = synth.sizes_loguniform(seed, pool_count, lo, hi)
    off = np.concatenate([[0], np.cumsum(sizes)])
    total = int(off[-1])
    X = torch.empty(total, dtype=torch.float64, device=r.dev)
    Y = torch.empty(total, dtype=torch.float64, device=r.dev)
    P = torch.empty(total, dtype=torch.float64, device=r.dev)
    Q = torch.empty(total, dtype=torch.float64, device=r.dev)
    nbytes = int(r.ctx.lib.spl_generate_scratch_bytes(int(sizes.max())))
    scratch = torch.empty(max(nbytes, 8), dtype=torch.uint8, device=r.dev)
    for i, nn in enumerate(sizes):
        assert r.ctx.lib.spl_generate_curve(seed, r.rank * pool_count + i, int(nn), X[off[i]:].data_ptr(),
                                            Y[off[i]:].data_ptr(), scratch.data_ptr(), nbytes,
                                            r.stream.cuda_stream) == 0
    r.stream.synchronize()
    reqs = []
    for i, nn in enumerate(sizes):
        o, nn = int(off[i]), int(nn)
        reqs.append(spl.make_request(X[o:o + nn], Y[o:o + nn], spl.NATURAL, spl.NATURAL, nn, P[o:o + nn], Q[o:o + nn]))
    srv = spl.Server(r.ctx, max_inflight=2048, tile_rows=0, budget_bytes=150 * 10 ** 9)
    st0 = srv.stats()
    # warm-up trace, then the measured trace (fresh Poisson draws, pool entries cycled)
    nw, nm = int(rate * warm_s), int(rate * run_s)
    s, _, _ = srv.replay(reqs, np.arange(nw) % pool_count, synth.poisson_arrivals(seed + 100, rate, nw))
    assert s == spl.OK
    arr = synth.poisson_arrivals(seed, rate, nm)
    pick = (np.arange(nm) * 7919) % pool_count
    s, lat, makespan = srv.replay(reqs, pick, arr)
    assert s == spl.OK
    pts = float(sizes[pick].sum())
    res = {"workload": "Poisson arrivals at %.0f requests/s for %.0f s, n log-uniform in [1e2, 1e6] (pool of %d "
                       "distinct seeded instances, seed 3), M = n, natural ends, mixed precision (binary32 solve and "
                       "cubic, exact binary64 differences and query positions), admission under a 150 GB HBM budget, "
                       "persistent device loop" % (rate, run_s, pool_count),
           "requests": nm, "offered_rate": rate, "value": nm / makespan, "unit": "instances/s",
           "points_per_s": pts / makespan, "latency_ms": {"p16": float(np.percentile(lat, 16)),
                                                          "p50": float(np.percentile(lat, 50)),
                                                          "p84": float(np.percentile(lat, 84)),
                                                          "p99": float(np.percentile(lat, 99)),
                                                          "max": float(lat.max()),
                                                          "what": "scheduled arrival to completion seen by the host"}}
    # saturation: every request of one pass over the pool arrives at once
    nsat = 4 * pool_count
    s, lat2, mk2 = srv.replay(reqs, np.arange(nsat) % pool_count, np.zeros(nsat))
    assert s == spl.OK
    pts2 = float(sizes.sum()) * 4
    res["saturation"] = {"requests": nsat, "value": nsat / mk2, "unit": "instances/s", "points_per_s": pts2 / mk2,
                         "gb_per_s": BYTES_PER_POINT * pts2 / mk2 / 1e9}
    st1 = srv.stats()
    res["loop_launches"] = st1["loop_launches"] - st0["loop_launches"]
    srv.close()
    torch.cuda.synchronize(r.dev)
    # the same stream with one refinement step per request (the precision the targets state)
    srvr = spl.Server(r.ctx, max_inflight=2048, tile_rows=0, budget_bytes=150 * 10 ** 9, refine_steps=1)
    s, _, _ = srvr.replay(reqs, np.arange(nw) % pool_count, synth.poisson_arrivals(seed + 101, rate, nw))
    assert s == spl.OK
    nr = int(rate * min(run_s, 4.0))
    s, latr, mkr = srvr.replay(reqs, pick[:nr], arr[:nr])
    assert s == spl.OK
    s, _, mkr2 = srvr.replay(reqs, np.arange(nsat) % pool_count, np.zeros(nsat))
    assert s == spl.OK
    srvr.close()
    torch.cuda.synchronize(r.dev)
    res["refined"] = {"workload": "the same arrivals (first %d) served with one refinement step of y'' per request"
                                  % nr, "requests": nr, "value": nr / mkr, "unit": "instances/s",
                      "latency_ms": {"p16": float(np.percentile(latr, 16)), "p50": float(np.percentile(latr, 50)),
                                     "p84": float(np.percentile(latr, 84)), "p99": float(np.percentile(latr, 99)),
                                     "max": float(latr.max())},
                      "saturation": {"requests": nsat, "value": nsat / mkr2, "unit": "instances/s",
                                     "gb_per_s": BYTES_PER_POINT * pts2 / mkr2 / 1e9}}
    rng = np.random.default_rng(1)
    sample = {}
    for i in rng.choice(pool_count, size=24, replace=False):
        o, nn = int(off[i]), int(sizes[i])
        sample[int(i)] = (P[o:o + nn].cpu().numpy(), Q[o:o + nn].cpu().numpy())
    # the plain FP64 path on the same pool (one graph-captured launch over all of it)
    plan = r.plan(spl.PREC_F64, 0, max_n=int(sizes.max()))
    b = r.ctx.batch(plan, reqs, keep=(X, Y, P, Q))
    for _ in range(2):
        b.launch()
        assert (b.wait() == 0).all()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(r.stream)
    K = 5
    for _ in range(K):
        b.launch()
    e1.record(r.stream)
    assert (b.wait() == 0).all()
    t_ms = e0.elapsed_time(e1) / K
    res["plain_f64_same_pool"] = {"value": pool_count / (t_ms * 1e-3), "unit": "instances/s",
                                  "points_per_s": total / (t_ms * 1e-3), "ms_per_pool": t_ms}
    b.close()
    res["served_over_plain_instances_per_s"] = res["saturation"]["value"] / res["plain_f64_same_pool"]["value"]
    # the same pool as one non-served binary32 batch (graph-captured launch over all of it), without
    # and with refinement: what continuous batching buys beyond the drop to binary32
    for refine in (0, 1):
        planm = r.plan(spl.PREC_F32_REFINE, refine, max_n=int(sizes.max()))
        bm = r.ctx.batch(planm, reqs, keep=(X, Y, P, Q))
        for _ in range(2):
            bm.launch()
            assert (bm.wait() == 0).all()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(r.stream)
        for _ in range(K):
            bm.launch()
        e1.record(r.stream)
        assert (bm.wait() == 0).all()
        tm = e0.elapsed_time(e1) / K
        res["plain_mixed_refine%d_same_pool" % refine] = {"value": pool_count / (tm * 1e-3), "unit": "instances/s",
                                                          "points_per_s": total / (tm * 1e-3), "ms_per_pool": tm}
        bm.close()
    res["served_over_plain_same_precision"] = (res["saturation"]["value"] /
                                               res["plain_mixed_refine0_same_pool"]["value"])
    return res, (sizes, seed, r.rank * pool_count, sample)


def short_line(r, which, res):
    print(json.dumps({"profile_run": True, "path": which, "n": r.n, "steps": r.K,
                      "ms_per_step": res["ms_per_step"], "gpu_launches": res.get("launches", res.get("gpu_launches")),
                      "e2e": res.get("e2e")}))


def run_ours(args, world, rank, local):
    r = Runner(args, world, rank, local)
    spl = r.spl
    if args.only:
        if args.only in ("variants", "schedule", "n1000", "noalloc", "dfma", "serving", "latency"):
            res = (r.eval_variants()[0] if args.only == "variants" else r.n_schedule() if args.only == "schedule"
                   else r.config1()[0] if args.only == "n1000" else r.dfma_probe() if args.only == "dfma"
                   else serving(r)[0] if args.only == "serving" else r.latency_by_size() if args.only == "latency"
                   else r.noalloc())
            if rank == 0:
                print(json.dumps({"profile_run": True, "path": args.only, "result": res}))
            r.ctx.close()
            return
        if args.only == "batched":
            res, _ = r.batched(steps=max(args.steps, 1))
        else:
            prec = spl.PREC_F64 if args.only == "f64" else spl.PREC_F32_REFINE
            plan = r.plan(prec, 1 if args.only == "mixed-refine" else 0)
            res = r.time_single(plan)
            if args.only == "f64" and not args.no_e2e:
                res["e2e"] = r.time_e2e(plan)
        if rank == 0:
            short_line(r, args.only, res)
        r.ctx.close()
        return
    n = r.n
    plan64 = r.plan(spl.PREC_F64)
    main = r.time_single(plan64, with_clocks=True)
    e2e = None if args.no_e2e else r.time_e2e(plan64)
    mixed0 = r.time_single(r.plan(spl.PREC_F32_REFINE, 0))
    mixed1 = r.time_single(r.plan(spl.PREC_F32_REFINE, 1))
    batched, bdata = r.batched()
    served, sdata = (None, None) if args.no_serving else serving(r)
    variants, vdata = r.eval_variants()
    schedule = r.n_schedule()
    small, c1data = r.config1()
    noalloc = r.noalloc()
    lat_sizes = r.latency_by_size()
    dfma = r.dfma_probe(clock_mhz=(main.get("clocks") or {}).get("sm_mhz"))
    if rank != 0:
        r.ctx.close()
        return

    ms = main["ms_per_step"]
    achieved = FLOPS_PER_POINT * n / (ms * 1e-3) / 1e12
    gbs = BYTES_PER_POINT * n / (ms * 1e-3) / 1e9
    pk = measured_peaks()
    hbm = pk.get("hbm_gbs")

    def path_entry(res, name, tol, dtype):
        msx = res["ms_per_step"]
        g = BYTES_PER_POINT * n / (msx * 1e-3) / 1e9
        return {"workload": name, "value": res["value"], "unit": "instances/s", "ms_per_step": msx,
                "points_per_s": res["value"] * n, "gb_per_s": g, "hbm_frac_of_measured": g / hbm if hbm else None,
                "latency_ms": {"p50": res["p50_ms"], "p99": res["p99_ms"]}, "gpu_launches": res["launches"],
                "dtype": dtype, "tolerance": tol}

    # the large distributions first, the compact per-configuration entries last (a reader of the
    # line's tail sees those)
    others = {
        "n_schedule": schedule,
        "newint_variants": variants,
        "n1000": small,
        "latency_by_size": lat_sizes,
        "noalloc": noalloc,
        "mixed_f32": path_entry(mixed0, "n=M=1e7 seed 1, binary32 solve + cubic, exact binary64 differences "
                                        "and query positions, no refinement", TOL["mixed"], "f32"),
        "mixed_f32_refine1": path_entry(mixed1, "same, plus one refinement step of y'' against a double-float "
                                                "residual (two launches)", TOL["mixed"], "f32+df"),
        "batched": batched,
        "serving": served,
    }
    others["mixed_f32"]["roofline"] = {"bound": "hbm", "traffic": profiled_traffic("mixed"),
                                       "achieved": others["mixed_f32"]["gb_per_s"], "peak": hbm, "unit": "GB/s",
                                       "frac": others["mixed_f32"]["hbm_frac_of_measured"],
                                       "issue_active_ncu": profiled_fraction("mixed", "issue_active_pct")}

    cpu = None
    if not args.no_cpu_baseline and world == 1:
        cpu, errs = cpu_baseline_and_errors(r, main, mixed0, mixed1, bdata, sdata, vdata)
        others_cpu = cpu_baselines_other(bdata, sdata, c1data)
        others["n1000"]["cpu_baseline"] = others_cpu.get("n1000")
        others["batched"]["cpu_baseline"] = others_cpu.get("batched")
        if served is not None:
            others["serving"]["cpu_baseline"] = others_cpu.get("serving_pool")
        if served is not None:
            others["serving"]["error_vs_oracle"] = errs["serving"]
        others["mixed_f32"]["error_vs_oracle"] = errs["mixed0"]
        others["mixed_f32_refine1"]["error_vs_oracle"] = errs["mixed1"]
        others["batched"]["error_vs_oracle"] = errs["batched"]
        others["newint_variants"]["error_vs_oracle"] = errs["variants"]
        main_err = errs["f64"]
    else:
        main_err = None

    line = {
        "metric": METRIC, "value": main["value"], "unit": "instances/s", "n_gpus": world, "steps": r.K,
        "warmup": r.W, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "m": n,
                   "instances_per_step": 1, "l2": "inputs+outputs 320 MB > 129 MB L2, no flush",
                   "parallelism": "one instance per GPU"},
        "points_per_s": main["value"] * n, "gb_per_s": gbs,
        "latency_ms": {"p50": main["p50_ms"], "p99": main["p99_ms"],
                       "what": "device time per step (events around each launch, %d in flight)" % r.window},
        "error_vs_oracle": main_err,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": PEAK_FP64_OPS_T, "unit": "TFLOP/s",
                     "frac": achieved / PEAK_FP64_OPS_T, "traffic": profiled_traffic("f64"),
                     "what": ("FP64 pipe: %d algorithmic FP64 ops/point (paper's counts, a division = 1) per second; "
                              "peak = 2 FP64 ops/clk/SM x 152 SMs x 2.07 GHz (one op per lane per clock)"
                              % FLOPS_PER_POINT),
                     "frac_of_fma_counted_peak": achieved / PEAK_FP64_TFLOPS,
                     "dfma_stream_measured": dfma,
                     "frac_of_dfma_stream": achieved / dfma["lane_ops_per_s_T"],
                     "fp64_pipe_active_ncu": profiled_fraction("f64", "fp64_pipe_active_pct"),
                     "hbm_gbs": gbs, "hbm_frac_of_measured": gbs / hbm if hbm else None},
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(main["launches"]),
        "clocks": main["clocks"],
        "other_configs": others,
    }
    line["summary"] = summary(line)
    print(json.dumps(line), flush=True)
    r.ctx.close()


def oracle_rate(curves, threads: int):
    """The FP64 oracle, as it stands, over a list of (x, y) instances (natural ends, M = n) on
    `threads` host threads (ctypes releases the interpreter lock while the C code runs).  Returns
    (instances per second, seconds)."""
    import concurrent.futures as cf
    import oracle

    def one(xy):
        r = oracle.fit_eval(xy[0], xy[1], oracle.NATURAL, oracle.NATURAL, len(xy[0]))
        assert r["status"] == oracle.OK
        return 0

    t0 = time.perf_counter()
    if threads <= 1:
        for xy in curves:
            one(xy)
    else:
        with cf.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(one, curves))
    el = time.perf_counter() - t0
    return len(curves) / el, el


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        return os.cpu_count() or 1


def cpu_baselines_other(bdata, sdata, c1data):
    """Host baselines of the other workloads, the oracle as it stands: the smallest configuration
    single-threaded (the paper's methodology), the batched workload single-threaded and on all
    host cores (parallel over instances), the served pool on all host cores."""
    import oracle
    from paper_2001_09253_gb300 import synth
    cores = host_cores()
    out = {}
    if c1data is not None:
        hx, hy = c1data
        oracle.fit_eval(hx, hy)
        reps, t0 = 0, time.perf_counter()
        while time.perf_counter() - t0 < 1.0:
            oracle.fit_eval(hx, hy, oracle.NATURAL, oracle.NATURAL, len(hx))
            reps += 1
        el = time.perf_counter() - t0
        out["n1000"] = {"value": reps / el, "unit": "instances/s", "us_per_instance": 1e6 * el / reps, "cores": 1,
                        "kind": "oracle", "sample": "%d repetitions of the n = 1000 instance (seed 0), single "
                                                    "thread, Python call overhead included" % reps}
    if bdata is not None:
        sizes = bdata[0]
        curves = [synth.curve(2, int(nn), instance=i) for i, nn in enumerate(sizes)]
        v1, el1 = oracle_rate(curves[:1024], 1)
        vn, eln = oracle_rate(curves, cores)
        out["batched"] = {"single_thread": {"value": v1, "unit": "instances/s", "cores": 1, "kind": "oracle",
                                            "sample": "first 1024 of the 4096 instances (%.1f s)" % el1},
                          "all_cores": {"value": vn, "unit": "instances/s", "cores": cores, "kind": "oracle",
                                        "sample": "all 4096 instances, one per task (%.1f s)" % eln}}
    if sdata is not None:
        sizes_s, seed_s, base_s = sdata[0], sdata[1], sdata[2]
        curves = [synth.curve(seed_s, int(nn), instance=base_s + i) for i, nn in enumerate(sizes_s)]
        vn, eln = oracle_rate(curves, cores)
        out["serving_pool"] = {"value": vn, "unit": "instances/s", "cores": cores, "kind": "oracle",
                               "sample": "the %d pool instances once, one per task (%.1f s); the served stream "
                                         "cycles the same pool" % (len(curves), eln)}
    return out


def summary(line):
    """The headline numbers of every configuration, compact, at the end of the JSON line."""
    def g(d, *ks):
        for k in ks:
            if not isinstance(d, dict) or k not in d or d[k] is None:
                return None
            d = d[k]
        return float("%.4g" % d) if isinstance(d, float) else d

    oc = line.get("other_configs", {})
    out = {"f64_1e7": {"ms": g(line, "ms_per_step"), "inst_s": g(line, "value"),
                       "alu_frac": g(line, "roofline", "frac"),
                       "frac_of_dfma_stream": g(line, "roofline", "frac_of_dfma_stream"),
                       "e2e_inst_s": g(line, "e2e", "value"),
                       "err_ypp": g(line, "error_vs_oracle", "ypp"), "err_yq": g(line, "error_vs_oracle", "yq"),
                       "oracle_inst_s_1core": g(line, "cpu_baseline", "value")}}
    for key, name in (("mixed_f32", "mixed_1e7"), ("mixed_f32_refine1", "mixed_refine1_1e7")):
        e = oc.get(key) or {}
        out[name] = {"ms": g(e, "ms_per_step"), "gb_s": g(e, "gb_per_s"), "hbm_frac": g(e, "hbm_frac_of_measured"),
                     "err_ypp": g(e, "error_vs_oracle", "ypp"), "err_yq": g(e, "error_vs_oracle", "yq")}
    b = oc.get("batched") or {}
    out["batched_4096"] = {"ms": g(b, "ms_per_step"), "inst_s": g(b, "value"), "gb_s": g(b, "gb_per_s"),
                           "err_ypp": g(b, "error_vs_oracle", "ypp"),
                           "oracle_inst_s_1core": g(b, "cpu_baseline", "single_thread", "value"),
                           "oracle_inst_s_all": g(b, "cpu_baseline", "all_cores", "value"),
                           "cores": g(b, "cpu_baseline", "all_cores", "cores")}
    sv = oc.get("serving") or {}
    out["serving_20k"] = {"inst_s": g(sv, "value"), "p50_ms": g(sv, "latency_ms", "p50"),
                          "p99_ms": g(sv, "latency_ms", "p99"), "sat_inst_s": g(sv, "saturation", "value"),
                          "plain_f64_inst_s": g(sv, "plain_f64_same_pool", "value"),
                          "plain_mixed_inst_s": g(sv, "plain_mixed_refine0_same_pool", "value"),
                          "served_over_plain_f64": g(sv, "served_over_plain_instances_per_s"),
                          "served_over_plain_same_precision": g(sv, "served_over_plain_same_precision"),
                          "oracle_inst_s_all": g(sv, "cpu_baseline", "value"), "err_yq": g(sv, "error_vs_oracle", "yq"),
                          "refined_p50_ms": g(sv, "refined", "latency_ms", "p50"),
                          "refined_p99_ms": g(sv, "refined", "latency_ms", "p99"),
                          "refined_sat_inst_s": g(sv, "refined", "saturation", "value")}
    c1 = oc.get("n1000") or {}
    out["n1000"] = {k: {"dev_p50_ms": g(c1, k, "device_ms", "median"), "dev_p99_ms": g(c1, k, "device_ms", "p99"),
                        "wall_p50_ms": g(c1, k, "wall_ms", "median"), "wall_p99_ms": g(c1, k, "wall_ms", "p99")}
                    for k in ("f64/natural", "mixed_refine1/natural")}
    out["n1000"]["oracle_us_1core"] = g(c1, "cpu_baseline", "us_per_instance")
    na = oc.get("noalloc") or {}
    out["noalloc_p50_ms"] = {k: {"noalloc": g(na, k, "noalloc_ms", "median"), "submit": g(na, k, "submit_ms", "median")}
                             for k in ("n=100000", "n=1000000")}
    ls = oc.get("latency_by_size") or {}
    out["latency_p50_ms"] = {k: g(ls, k, "median") for k in ls if "/n=" in k}
    v = oc.get("newint_variants") or {}
    out["eval_1e7_ms"] = {lab: {nm: g(v, lab, nm, "ms", "median") for nm in ("orig", "noinv", "vol", "noop")}
                          for lab in ("sorted", "unsorted")}
    return out


def cpu_baseline_and_errors(r, main, mixed0, mixed1, bdata, sdata, vdata=None):
    """The FP64 oracle, as it stands, single-threaded on the host cores: its rate on the main
    workload (repeated for ~10 s) and the error of every GPU result against its outputs."""
    import oracle
    from paper_2001_09253_gb300 import synth
    n = r.n
    x, y = synth.curve(SEED, n)
    oracle.fit_eval(x[:1000], y[:1000])
    reps, t0 = 0, time.perf_counter()
    ref = None
    while True:
        ref = oracle.fit_eval(x, y, oracle.NATURAL, oracle.NATURAL, n)
        assert ref["status"] == oracle.OK
        reps += 1
        el = time.perf_counter() - t0
        if el >= 10.0 or reps >= 30:
            break
    cpu = {"value": reps / el, "unit": "instances/s", "cores": 1, "kind": "oracle",
           "sample": "%d full n=1e7 instances (%.1f s), single thread" % (reps, el)}

    def errs(res):
        ypp = res["ypp"].cpu().numpy()
        yq = res["yq"].cpu().numpy()
        return error_pair(x, y, ref, ypp, yq)

    out = {"f64": errs(main), "mixed0": errs(mixed0), "mixed1": errs(mixed1)}
    sizes, off, X, Y, P, Q = bdata
    rng = np.random.default_rng(0)
    pick = rng.choice(len(sizes), size=64, replace=False)
    worst = [0.0, 0.0]
    Pc, Qc = P.cpu().numpy(), Q.cpu().numpy()
    for i in pick:
        nn, o = int(sizes[i]), int(off[i])
        xi, yi = synth.curve(2, nn, instance=i)
        rf = oracle.fit_eval(xi, yi, oracle.NATURAL, oracle.NATURAL, nn)
        e = error_pair(xi, yi, rf, Pc[o:o + nn], Qc[o:o + nn])
        worst = [max(worst[0], e["ypp"]), max(worst[1], e["yq"])]
    out["batched"] = {"ypp": worst[0], "yq": worst[1], "sample": "64 of 4096 instances"}
    if vdata is not None:
        # evaluation forms: brackets bit-exact and values within the FP64 tolerance on a sample,
        # against the oracle's bisection and its interpolation form with the oracle's y''
        pick, xq_pick, samples = vdata
        grid_q = oracle.grid(x, n)[pick]
        ve = {}
        for (label, name), (yq_s, jq_s) in samples.items():
            q = grid_q if label == "sorted" else xq_pick
            jref = oracle.bracket_any(x, q)
            yref = oracle.evaluate(x, y, ref["ypp"], q, jref)
            j64 = jq_s.astype(np.int64)
            same = bool(np.array_equal(j64, jref))
            h = x[jref + 1] - x[jref]
            curv = h * h * np.maximum(np.abs(ref["ypp"][jref]), np.abs(ref["ypp"][jref + 1])) / 6.0
            scale = np.maximum.reduce([np.abs(y[jref]), np.abs(y[jref + 1]), np.abs(yref), curv])
            ve["%s/%s" % (label, name)] = {"brackets_bit_exact": same,
                                            "yq": float(np.max(np.abs(yq_s - yref) / scale))}
        ve["sample"] = "%d of the 1e7 queries per variant and ordering" % len(pick)
        out["variants"] = ve
    if sdata is None:
        return cpu, out
    sizes_s, seed_s, base_s, sample = sdata
    worst = [0.0, 0.0]
    for i, (ypp_i, yq_i) in sample.items():
        nn = int(sizes_s[i])
        xi, yi = synth.curve(seed_s, nn, instance=base_s + i)
        rf = oracle.fit_eval(xi, yi, oracle.NATURAL, oracle.NATURAL, nn)
        e = error_pair(xi, yi, rf, ypp_i, yq_i)
        worst = [max(worst[0], e["ypp"]), max(worst[1], e["yq"])]
    out["serving"] = {"ypp": worst[0], "yq": worst[1], "sample": "%d of the pool's instances" % len(sample)}
    return cpu, out


def error_pair(x, y, ref, ypp, yq):
    e1 = float(np.max(np.abs(ypp - ref["ypp"])) / max(np.max(np.abs(ref["ypp"])), 1e-300))
    j = ref["jq"]
    h = x[j + 1] - x[j]
    curv = h * h * np.maximum(np.abs(ref["ypp"][j]), np.abs(ref["ypp"][j + 1])) / 6.0
    scale = np.maximum.reduce([np.abs(y[j]), np.abs(y[j + 1]), np.abs(ref["yq"]), curv])
    e2 = float(np.max(np.abs(yq - ref["yq"]) / np.maximum(scale, 1e-300)))
    return {"ypp": e1, "yq": e2}


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
