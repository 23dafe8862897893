"""FP64 CPU oracle for the spline fit + evaluation path (arXiv 2001.09253).

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or runs anything in this directory.

The arithmetic lives in ``spline_oracle.c`` (plain single-threaded C, built
with ``-ffp-contract=off``); this module only compiles it and marshals numpy
arrays through ctypes.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spline_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, INVALID_ARG, NOT_INCREASING, NONFINITE = 0, 1, 2, 3
NATURAL = 1e32  # any end slope above 0.99e30 selects the natural end condition


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/_build/liboracle.so`` (gcc, -O2, no FMA contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _bind(path):
    L = ctypes.CDLL(path)
    i64, dp, lp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int64)
    d = ctypes.c_double
    L.orc_validate.argtypes = [i64, dp, dp, d, d]
    L.orc_validate.restype = ctypes.c_int
    L.orc_fit.argtypes = [i64, dp, dp, d, d, dp, dp]
    L.orc_fit.restype = ctypes.c_int
    L.orc_grid.argtypes = [i64, dp, i64, dp]
    L.orc_grid.restype = None
    L.orc_bracket_sweep.argtypes = [i64, dp, i64, dp, lp]
    L.orc_bracket_sweep.restype = None
    L.orc_bracket_any.argtypes = [i64, dp, i64, dp, lp]
    L.orc_bracket_any.restype = None
    L.orc_interp.argtypes = [d, d, d, d, d, d, d]
    L.orc_interp.restype = d
    L.orc_eval.argtypes = [i64, dp, dp, dp, i64, dp, lp, dp]
    L.orc_eval.restype = None
    L.orc_fit_eval.argtypes = [i64, dp, dp, d, d, i64, dp, dp, lp, dp]
    L.orc_fit_eval.restype = ctypes.c_int
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _bind(build())
    return _lib


@contextlib.contextmanager
def swapped(path: str):
    """Temporarily route every call in this module to another build of the
    oracle source (used by the tests that plant a mistake in a copy of it)."""
    global _lib
    with _lock:
        old = _lib
        _lib = _bind(path)
    try:
        yield
    finally:
        with _lock:
            _lib = old


def compile_source(src_path: str, out_path: str) -> str:
    """Compile a (possibly modified) copy of the oracle source with the oracle's own flags."""
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-o", out_path, src_path, "-lm"], check=True)
    return out_path


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _lp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def validate(x, y, yp1=NATURAL, ypn=NATURAL) -> int:
    x, y = _f64(x), _f64(y)
    return lib().orc_validate(len(x), _dp(x), _dp(y), float(yp1), float(ypn))


def fit(x, y, yp1=NATURAL, ypn=NATURAL):
    """Second derivatives y'' (natural end when the slope is above 0.99e30).

    Returns ``(status, ypp)``; ``ypp`` is None unless status == OK."""
    x, y = _f64(x), _f64(y)
    n = len(x)
    if len(y) != n:
        return INVALID_ARG, None
    ypp = np.zeros(max(n, 1))
    cp = np.zeros(max(n, 1))
    st = lib().orc_fit(n, _dp(x), _dp(y), float(yp1), float(ypn), _dp(ypp), _dp(cp))
    return st, (ypp[:n] if st == OK else None)


def grid(x, m: int) -> np.ndarray:
    x = _f64(x)
    xq = np.zeros(max(m, 1))
    lib().orc_grid(len(x), _dp(x), m, _dp(xq))
    return xq[:m]


def bracket_sweep(x, xq) -> np.ndarray:
    x, xq = _f64(x), _f64(xq)
    jq = np.zeros(max(len(xq), 1), dtype=np.int64)
    lib().orc_bracket_sweep(len(x), _dp(x), len(xq), _dp(xq), _lp(jq))
    return jq[:len(xq)]


def bracket_any(x, xq) -> np.ndarray:
    x, xq = _f64(x), _f64(xq)
    jq = np.zeros(max(len(xq), 1), dtype=np.int64)
    lib().orc_bracket_any(len(x), _dp(x), len(xq), _dp(xq), _lp(jq))
    return jq[:len(xq)]


def interp(q, xj, xj1, yj, yj1, ppj, ppj1) -> float:
    return lib().orc_interp(float(q), float(xj), float(xj1), float(yj), float(yj1), float(ppj), float(ppj1))


def evaluate(x, y, ypp, xq, jq=None) -> np.ndarray:
    """Interpolated values at arbitrary queries (bracketing by definition unless jq is given)."""
    x, y, ypp, xq = _f64(x), _f64(y), _f64(ypp), _f64(xq)
    if jq is None:
        jq = bracket_any(x, xq)
    jq = np.ascontiguousarray(jq, dtype=np.int64)
    yq = np.zeros(max(len(xq), 1))
    lib().orc_eval(len(x), _dp(x), _dp(y), _dp(ypp), len(xq), _dp(xq), _lp(jq), _dp(yq))
    return yq[:len(xq)]


def fit_eval(x, y, yp1=NATURAL, ypn=NATURAL, m: int | None = None):
    """The whole path for one instance with m uniform queries (m = n by default).

    Returns a dict with status, ypp, xq, jq, yq (arrays None unless OK)."""
    x, y = _f64(x), _f64(y)
    n = len(x)
    if m is None:
        m = n
    ypp = np.zeros(max(n, 1))
    xq = np.zeros(max(m, 1))
    jq = np.zeros(max(m, 1), dtype=np.int64)
    yq = np.zeros(max(m, 1))
    st = lib().orc_fit_eval(n, _dp(x), _dp(y), float(yp1), float(ypn), m, _dp(ypp), _dp(xq), _lp(jq), _dp(yq))
    if st != OK:
        return {"status": st, "ypp": None, "xq": None, "jq": None, "yq": None}
    return {"status": st, "ypp": ypp[:n], "xq": xq[:m], "jq": jq[:m], "yq": yq[:m]}
