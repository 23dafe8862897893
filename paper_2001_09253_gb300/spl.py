"""Thin ctypes binding of libspl.so (include/spl.h): argument marshalling only.

Every step of the spline path runs in the CUDA library; this module converts
torch tensors / numpy arrays to pointers and back.  PyTorch supplies the device
memory (the arena handed to the library, the output tensors) and the stream.
There is no CPU fallback: if the library is missing or cannot load, every call
raises.
"""
from __future__ import annotations

import ctypes
import os
import threading
import weakref

import numpy as np

from . import build as _build

# spl_status
OK, PENDING = 0, 1
ERR_INVALID_ARG, ERR_NOT_INCREASING, ERR_NONFINITE, ERR_BUDGET = -1, -2, -3, -4
ERR_QUEUE_FULL, ERR_TIMEOUT, ERR_CUDA, ERR_UNKNOWN_TICKET, ERR_STATE = -5, -6, -7, -8, -9
PREC_F64, PREC_F32_REFINE = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
QUERY_UNIFORM, QUERY_EXPLICIT = 0, 1
EVAL_ORIG, EVAL_NOINV, EVAL_VOL, EVAL_NOOP = 0, 1, 2, 3
KERNEL_NONE, KERNEL_FUSED_F64, KERNEL_SMALL_F64, KERNEL_MID_F64, KERNEL_SCAN_MIXED = 0, 1, 2, 3, 4
NATURAL = 1e32

EXPORTS = [
    "spl_status_str", "spl_create", "spl_destroy", "spl_plan_create", "spl_plan_destroy", "spl_submit",
    "spl_submit_batch", "spl_poll", "spl_wait", "spl_get_stats", "spl_batch_create", "spl_batch_launch",
    "spl_batch_wait", "spl_batch_destroy", "spl_generate_scratch_bytes", "spl_generate_curve",
    "spl_fit_eval_noalloc", "spl_serve_create", "spl_serve_submit", "spl_serve_poll", "spl_serve_wait",
    "spl_serve_replay", "spl_serve_stats", "spl_serve_destroy", "spl_selftest_div64", "spl_selftest_dfma",
    "spl_launch_geometry",
]
NOALLOC_MAX_N = 1048576


class CtxDesc(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int32), ("max_slots", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("arena", ctypes.c_void_p), ("arena_bytes", ctypes.c_uint64)]


class PlanDesc(ctypes.Structure):
    _fields_ = [("max_n", ctypes.c_uint64), ("precision", ctypes.c_int32), ("refine_steps", ctypes.c_int32),
                ("tile_rows", ctypes.c_int32), ("query_mode", ctypes.c_int32), ("eval_variant", ctypes.c_int32),
                ("fault_flags", ctypes.c_uint32)]


class Geometry(ctypes.Structure):
    _fields_ = [("fit_kernel", ctypes.c_int32), ("separate_eval", ctypes.c_int32), ("tile_rows", ctypes.c_int32),
                ("direct", ctypes.c_int32), ("cta_rows", ctypes.c_int64), ("ctas", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("yp1", ctypes.c_double), ("ypn", ctypes.c_double), ("m", ctypes.c_uint64),
                ("ypp_out", ctypes.c_void_p), ("yq_out", ctypes.c_void_p), ("jq_out", ctypes.c_void_p),
                ("mem", ctypes.c_int32), ("reserved", ctypes.c_int32), ("xq", ctypes.c_void_p),
                ("ypp_in", ctypes.c_void_p)]


class ServeDesc(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_uint32), ("tile_rows", ctypes.c_uint32), ("budget_bytes", ctypes.c_uint64),
                ("max_tiles", ctypes.c_uint64), ("idle_timeout_ms", ctypes.c_uint32), ("deadline_ms", ctypes.c_uint32),
                ("fault_flags", ctypes.c_uint32), ("refine_steps", ctypes.c_uint32)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("device_ms", ctypes.c_float), ("latency_ms", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("requests_done", ctypes.c_uint64), ("arena_high_water", ctypes.c_uint64)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libspl.so (building it first if it is absent).  Raises on failure."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = path or _build.LIB
        if not os.path.exists(path):
            _build.build()
        L = ctypes.CDLL(path)
        vp, u64, i32, u32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int32, ctypes.c_uint32
        L.spl_status_str.argtypes = [i32]
        L.spl_status_str.restype = ctypes.c_char_p
        L.spl_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(CtxDesc)]
        L.spl_destroy.argtypes = [vp]
        L.spl_destroy.restype = None
        L.spl_plan_create.argtypes = [vp, ctypes.POINTER(PlanDesc), ctypes.POINTER(vp)]
        L.spl_plan_destroy.argtypes = [vp]
        L.spl_plan_destroy.restype = None
        L.spl_submit.argtypes = [vp, vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]
        L.spl_submit_batch.argtypes = [vp, vp, ctypes.POINTER(Request), u32, ctypes.POINTER(u64)]
        L.spl_poll.argtypes = [vp, u64, ctypes.POINTER(Result)]
        L.spl_wait.argtypes = [vp, u64, u64, ctypes.POINTER(Result)]
        L.spl_get_stats.argtypes = [vp, ctypes.POINTER(Stats)]
        L.spl_launch_geometry.argtypes = [ctypes.POINTER(PlanDesc), ctypes.POINTER(u64), u32, i32, i32, i32,
                                          ctypes.POINTER(Geometry)]
        L.spl_batch_create.argtypes = [vp, vp, ctypes.POINTER(Request), u32, ctypes.POINTER(vp)]
        L.spl_batch_launch.argtypes = [vp]
        L.spl_batch_wait.argtypes = [vp, u64, ctypes.POINTER(i32)]
        L.spl_batch_destroy.argtypes = [vp]
        L.spl_batch_destroy.restype = None
        L.spl_generate_scratch_bytes.argtypes = [u64]
        L.spl_generate_scratch_bytes.restype = u64
        L.spl_generate_curve.argtypes = [u64, u64, u64, vp, vp, vp, u64, vp]
        L.spl_fit_eval_noalloc.argtypes = [vp, vp, u64, ctypes.c_double, ctypes.c_double, u64, vp, vp, vp,
                                           ctypes.POINTER(i32)]
        L.spl_serve_create.argtypes = [vp, ctypes.POINTER(ServeDesc), ctypes.POINTER(vp)]
        L.spl_serve_submit.argtypes = [vp, ctypes.POINTER(Request), ctypes.POINTER(u64)]
        L.spl_serve_poll.argtypes = [vp, u64, ctypes.POINTER(Result)]
        L.spl_serve_wait.argtypes = [vp, u64, u64, ctypes.POINTER(Result)]
        dp = ctypes.POINTER(ctypes.c_double)
        L.spl_serve_replay.argtypes = [vp, ctypes.POINTER(Request), u32, ctypes.POINTER(u32), dp, u64, dp, dp]
        L.spl_serve_stats.argtypes = [vp, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)]
        L.spl_serve_destroy.argtypes = [vp]
        L.spl_serve_destroy.restype = None
        L.spl_selftest_div64.argtypes = [vp, vp, u64, vp, vp, vp, vp, vp]
        L.spl_selftest_dfma.argtypes = [u64, i32, ctypes.c_double, ctypes.c_double, vp, u64, ctypes.POINTER(u64), vp]
        for name in ["spl_create", "spl_plan_create", "spl_submit", "spl_submit_batch", "spl_poll", "spl_wait",
                     "spl_get_stats", "spl_batch_create", "spl_batch_launch", "spl_batch_wait",
                     "spl_generate_curve", "spl_fit_eval_noalloc", "spl_serve_create", "spl_serve_submit",
                     "spl_serve_poll", "spl_serve_wait", "spl_serve_replay", "spl_serve_stats",
                     "spl_selftest_div64", "spl_selftest_dfma"]:
            getattr(L, name).restype = i32
        _lib = L
        return L


def status_str(s: int) -> str:
    return load().spl_status_str(int(s)).decode()


class SplError(RuntimeError):
    def __init__(self, status: int, what: str = ""):
        self.status = int(status)
        super().__init__("%s: %s (%d)" % (what, status_str(status), status))


def _check(s: int, what: str):
    if s < 0:
        raise SplError(s, what)
    return s


def _ptr(a):
    """Address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data
    return a.data_ptr()


def _is_host(a) -> bool:
    if isinstance(a, np.ndarray):
        return True
    return a.device.type == "cpu"


def make_request(x, y, yp1=NATURAL, ypn=NATURAL, m=None, ypp_out=None, yq_out=None, jq_out=None,
                 xq=None, ypp_in=None) -> Request:
    n = int(x.shape[0])
    if m is None:
        m = int(xq.shape[0]) if xq is not None else n
    r = Request()
    r.n, r.x, r.y = n, _ptr(x), _ptr(y)
    r.yp1, r.ypn, r.m = float(yp1), float(ypn), int(m)
    r.ypp_out, r.yq_out, r.jq_out = _ptr(ypp_out), _ptr(yq_out), _ptr(jq_out)
    r.xq, r.ypp_in = _ptr(xq), _ptr(ypp_in)
    r.mem = MEM_HOST if _is_host(x) else MEM_DEVICE
    return r


class Plan:
    """spl_plan_create: options shared by the requests submitted with the plan (spl_plan_desc in
    include/spl.h).  fault_flags is for failure-detection tests only: bit 0 makes the last CTA of
    the multi-CTA FP64 kernel withhold its partial solutions, so that the request completes with
    ERR_TIMEOUT."""

    def __init__(self, ctx: "Context", max_n: int, precision: int = PREC_F64, refine_steps: int = 0,
                 tile_rows: int = 0, query_mode: int = 0, eval_variant: int = 0, fault_flags: int = 0):
        self.ctx = ctx
        d = PlanDesc(max_n=int(max_n), precision=int(precision), refine_steps=int(refine_steps),
                     tile_rows=int(tile_rows), query_mode=int(query_mode), eval_variant=int(eval_variant),
                     fault_flags=int(fault_flags))
        h = ctypes.c_void_p()
        _check(ctx.lib.spl_plan_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)), "spl_plan_create")
        self.handle = h

    def close(self):
        if self.handle:
            self.ctx.lib.spl_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    def __init__(self, ctx: "Context", plan: Plan, requests, keep=()):
        self.ctx, self.plan, self.count = ctx, plan, len(requests)
        self._keep = keep
        arr = (Request * len(requests))(*requests)
        h = ctypes.c_void_p()
        _check(ctx.lib.spl_batch_create(ctx.handle, plan.handle, arr, len(requests), ctypes.byref(h)),
               "spl_batch_create")
        self.handle = h

    def launch(self):
        _check(self.ctx.lib.spl_batch_launch(self.handle), "spl_batch_launch")

    def wait(self, timeout_s: float = 60.0):
        st = (ctypes.c_int32 * self.count)()
        s = self.ctx.lib.spl_batch_wait(self.handle, int(timeout_s * 1e9), st)
        if s == ERR_TIMEOUT or s == ERR_CUDA or s == ERR_STATE:
            raise SplError(s, "spl_batch_wait")
        return np.frombuffer(st, dtype=np.int32).copy()

    def close(self):
        if self.handle:
            self.ctx.lib.spl_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Context:
    """One library context on one device and one stream, with a torch-allocated arena."""

    def __init__(self, device: int = 0, stream=None, arena_bytes: int = 1 << 30, max_slots: int = 1024,
                 arena=None):
        import torch
        self.lib = load()
        self.torch = torch
        self.device = int(device)
        dev = torch.device("cuda", self.device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(dev)
        self._servers = weakref.WeakSet()  # closed before the context (they use its arena)
        if arena is None:
            arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        self.arena = arena
        d = CtxDesc(device=self.device, max_slots=int(max_slots), stream=self.stream.cuda_stream,
                    arena=arena.data_ptr(), arena_bytes=arena.numel() * arena.element_size())
        h = ctypes.c_void_p()
        _check(self.lib.spl_create(ctypes.byref(h), ctypes.byref(d)), "spl_create")
        self.handle = h
        self._keep = {}

    def plan(self, max_n: int, precision: int = PREC_F64, refine_steps: int = 0, tile_rows: int = 0,
             query_mode: int = 0, eval_variant: int = 0, fault_flags: int = 0) -> Plan:
        return Plan(self, max_n, precision, refine_steps, tile_rows, query_mode, eval_variant, fault_flags)

    def submit(self, plan: Plan, x, y, yp1=NATURAL, ypn=NATURAL, m=None, ypp_out=None, yq_out=None,
               jq_out=None, xq=None, ypp_in=None) -> int:
        r = make_request(x, y, yp1, ypn, m, ypp_out, yq_out, jq_out, xq, ypp_in)
        t = ctypes.c_uint64()
        _check(self.lib.spl_submit(self.handle, plan.handle, ctypes.byref(r), ctypes.byref(t)), "spl_submit")
        self._keep[t.value] = (x, y, ypp_out, yq_out, jq_out)
        return t.value

    def submit_batch(self, plan: Plan, requests, keep=()):
        arr = (Request * len(requests))(*requests)
        ts = (ctypes.c_uint64 * len(requests))()
        _check(self.lib.spl_submit_batch(self.handle, plan.handle, arr, len(requests), ts), "spl_submit_batch")
        out = list(ts)
        for t in out:
            self._keep[t] = keep
        return out

    def poll(self, ticket: int):
        res = Result()
        s = self.lib.spl_poll(self.handle, int(ticket), ctypes.byref(res))
        if s != PENDING:
            self._keep.pop(int(ticket), None)
        return s, res

    def wait(self, ticket: int, timeout_s: float = 60.0):
        res = Result()
        s = self.lib.spl_wait(self.handle, int(ticket), int(timeout_s * 1e9), ctypes.byref(res))
        if s != PENDING and not (s == ERR_TIMEOUT and res.status == PENDING):  # completed
            self._keep.pop(int(ticket), None)
        return s, res

    def batch(self, plan: Plan, requests, keep=()) -> Batch:
        return Batch(self, plan, requests, keep)

    def stats(self) -> dict:
        st = Stats()
        _check(self.lib.spl_get_stats(self.handle, ctypes.byref(st)), "spl_get_stats")
        return {k: getattr(st, k) for k, _ in Stats._fields_}

    def close(self):
        if getattr(self, "handle", None):
            for srv in list(getattr(self, "_servers", ())):
                srv.close()
            self.lib.spl_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching server on a persistent device loop (spl_serve_*)."""

    def __init__(self, ctx: Context, max_inflight: int = 1024, tile_rows: int = 0, budget_bytes: int = 1 << 34,
                 max_tiles: int = 0, idle_timeout_ms: int = 0, deadline_ms: int = 0, fault_flags: int = 0,
                 refine_steps: int = 0):
        self.ctx, self.lib = ctx, ctx.lib
        d = ServeDesc(max_inflight=int(max_inflight), tile_rows=int(tile_rows), budget_bytes=int(budget_bytes),
                      max_tiles=int(max_tiles), idle_timeout_ms=int(idle_timeout_ms), deadline_ms=int(deadline_ms),
                      fault_flags=int(fault_flags), refine_steps=int(refine_steps))
        h = ctypes.c_void_p()
        _check(self.lib.spl_serve_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)), "spl_serve_create")
        self.handle = h
        ctx._servers.add(self)
        self._keep = {}

    def submit(self, x, y, yp1=NATURAL, ypn=NATURAL, m=None, ypp_out=None, yq_out=None, jq_out=None,
               sync=True) -> int:
        """sync: first wait for the caller's current stream, since the running device loop may
        pick the request up at once and pending writes to its arrays (their creation, a fill) must
        land first; False when the caller has made the arrays ready itself."""
        import torch
        r = make_request(x, y, yp1, ypn, m, ypp_out, yq_out, jq_out)
        if sync and x.is_cuda:  # host arrays are refused below (the loop reads device memory only)
            torch.cuda.current_stream(x.device).synchronize()
        t = ctypes.c_uint64()
        _check(self.lib.spl_serve_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "spl_serve_submit")
        self._keep[t.value] = (x, y, ypp_out, yq_out, jq_out)
        return t.value

    def poll(self, ticket: int):
        res = Result()
        s = self.lib.spl_serve_poll(self.handle, int(ticket), ctypes.byref(res))
        if s != PENDING:
            self._keep.pop(int(ticket), None)
        return s, res

    def wait(self, ticket: int, timeout_s: float = 60.0):
        res = Result()
        s = self.lib.spl_serve_wait(self.handle, int(ticket), int(timeout_s * 1e9), ctypes.byref(res))
        if s not in (PENDING, ERR_TIMEOUT):
            self._keep.pop(int(ticket), None)
        return s, res

    def replay(self, pool, pick, arrival_s):
        """Replay an arrival trace (pool: list of Request; pick, arrival_s: numpy arrays)."""
        n = len(pick)
        arr = (Request * len(pool))(*pool)
        pk = np.ascontiguousarray(pick, dtype=np.uint32)
        at = np.ascontiguousarray(arrival_s, dtype=np.float64)
        lat = np.zeros(max(n, 1))
        mk = ctypes.c_double()
        dp = ctypes.POINTER(ctypes.c_double)
        s = self.lib.spl_serve_replay(self.handle, arr, len(pool), pk.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                      at.ctypes.data_as(dp), n, lat.ctypes.data_as(dp), ctypes.byref(mk))
        return s, lat[:n], mk.value

    def stats(self) -> dict:
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(self.lib.spl_serve_stats(self.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)),
               "spl_serve_stats")
        return {"loop_launches": a.value, "waiting": b.value, "resident": c.value}

    def close(self):
        if getattr(self, "handle", None):
            self.lib.spl_serve_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def launch_geometry(sizes, sm_count: int, precision: int = PREC_F64, refine_steps: int = 0, tile_rows: int = 0,
                    query_mode: int = QUERY_UNIFORM, max_n: int | None = None, mem: int = MEM_DEVICE,
                    stored_fit: bool = False):
    """spl_launch_geometry: the kernel and tiling a submission of instances of `sizes` knots would
    take on a device of sm_count SMs (a pure function; no GPU needed).  Returns a dict, or raises
    SplError for arguments the library rejects."""
    L = load()
    ns = [int(v) for v in sizes]
    arr = (ctypes.c_uint64 * len(ns))(*ns)
    d = PlanDesc(max_n=int(max_n if max_n is not None else max(ns + [3])), precision=precision,
                 refine_steps=refine_steps, tile_rows=tile_rows, query_mode=query_mode, eval_variant=EVAL_ORIG,
                 fault_flags=0)
    g = Geometry()
    s = L.spl_launch_geometry(ctypes.byref(d), arr, len(ns), mem, 1 if stored_fit else 0, sm_count, ctypes.byref(g))
    if s != OK:
        raise SplError(s)
    return {"fit_kernel": g.fit_kernel, "separate_eval": bool(g.separate_eval), "tile_rows": g.tile_rows,
            "direct": bool(g.direct), "cta_rows": g.cta_rows, "ctas": g.ctas}


def fit_eval_noalloc(x, y, yp1=NATURAL, ypn=NATURAL, m=None, ypp_out=None, yq_out=None, stream=None,
                     want_status=True):
    """spl_fit_eval_noalloc: one instance, no allocation inside the library (device tensors
    in and out, n <= NOALLOC_MAX_N).  m defaults to n when yq_out is given, else to 0 (fit only).
    Returns (call status, device status or None)."""
    L = load()
    n = int(x.shape[0])
    if m is None:
        m = n if yq_out is not None else 0
    m = int(m)
    st = ctypes.c_int32(PENDING)
    s = L.spl_fit_eval_noalloc(_ptr(x), _ptr(y), n, float(yp1), float(ypn), m, _ptr(ypp_out), _ptr(yq_out),
                               stream.cuda_stream if stream is not None else None,
                               ctypes.byref(st) if want_status else None)
    return s, (st.value if want_status else None)


def selftest_div64(num, den, stream=None):
    """spl_selftest_div64 on device tensors: returns (q_fast, r_fast, q_ieee, r_ieee) tensors."""
    import torch
    L = load()
    n = int(num.shape[0])
    outs = [torch.empty(max(n, 1), dtype=torch.float64, device=num.device) for _ in range(4)]
    st = stream if stream is not None else torch.cuda.current_stream(num.device)
    _check(L.spl_selftest_div64(_ptr(num), _ptr(den), n, *[_ptr(o) for o in outs], st.cuda_stream),
           "spl_selftest_div64")
    return tuple(o[:n] for o in outs)


def selftest_dfma(trips: int, warps_per_sm: int, sink, mul: float = 0.999999, add: float = 1e-6, stream=None):
    """spl_selftest_dfma: enqueues the DFMA-stream probe on `stream` (sink: a float64 device tensor of
    at least SMs x warps_per_sm x 32 elements) and returns the DFMA lane operations it performs."""
    import torch
    L = load()
    ops = ctypes.c_uint64(0)
    st = stream if stream is not None else torch.cuda.current_stream(sink.device)
    _check(L.spl_selftest_dfma(int(trips), int(warps_per_sm), float(mul), float(add), _ptr(sink), int(sink.numel()),
                               ctypes.byref(ops), st.cuda_stream), "spl_selftest_dfma")
    return ops.value


def generate_curve(seed: int, n: int, instance: int = 0, device: int = 0, stream=None):
    """Benchmark curve generated on the device (bit-identical to synth.curve)."""
    import torch
    L = load()
    dev = torch.device("cuda", device)
    x = torch.empty(n, dtype=torch.float64, device=dev)
    y = torch.empty(n, dtype=torch.float64, device=dev)
    nbytes = int(L.spl_generate_scratch_bytes(n))
    scratch = torch.empty(max(nbytes, 8), dtype=torch.uint8, device=dev)
    st = stream if stream is not None else torch.cuda.current_stream(dev)
    _check(L.spl_generate_curve(seed, instance, n, x.data_ptr(), y.data_ptr(), scratch.data_ptr(), nbytes,
                                st.cuda_stream), "spl_generate_curve")
    return x, y
