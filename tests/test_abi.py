"""The C-ABI library builds for sm_103a, loads, and exports every entry point that
include/spl.h declares (no GPU needed: nothing here launches work)."""
import ctypes
import os
import re

import pytest

from paper_2001_09253_gb300 import build, spl

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "spl.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(spl_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert sorted(spl.EXPORTS) == sorted(set(spl.EXPORTS))
    assert set(spl.EXPORTS) <= set(names)


def test_status_strings_without_gpu():
    lib = spl.load()
    assert lib.spl_status_str(0) == b"ok"
    assert lib.spl_status_str(-2) == b"knots not strictly increasing"
    assert lib.spl_status_str(12345) == b"unknown status"


def test_create_rejects_bad_descriptors_without_touching_a_gpu():
    lib = spl.load()
    h = ctypes.c_void_p()
    d = spl.CtxDesc(device=0, max_slots=0, stream=None, arena=None, arena_bytes=1 << 30)
    assert lib.spl_create(ctypes.byref(h), ctypes.byref(d)) == spl.ERR_INVALID_ARG
    d = spl.CtxDesc(device=0, max_slots=4, stream=None, arena=None, arena_bytes=1024)
    assert lib.spl_create(ctypes.byref(h), ctypes.byref(d)) == spl.ERR_INVALID_ARG
    assert lib.spl_create(None, ctypes.byref(d)) == spl.ERR_INVALID_ARG


def test_sm103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_cpu_fallback_without_a_gpu():
    """Without a CUDA device the entry points that compute fail with SPL_ERR_CUDA: nothing
    falls back to the CPU (only meaningful on a machine without a GPU)."""
    import numpy as np
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib = spl.load()
    h = ctypes.c_void_p()
    d = spl.CtxDesc(device=0, max_slots=4, stream=None, arena=None, arena_bytes=64 << 20)
    assert lib.spl_create(ctypes.byref(h), ctypes.byref(d)) == spl.ERR_CUDA
    assert not h.value
    x = np.arange(10, dtype=np.float64)
    y = np.sin(x)
    yq = np.full(10, np.nan)
    st = ctypes.c_int32(spl.PENDING)
    r = lib.spl_fit_eval_noalloc(x.ctypes.data, y.ctypes.data, 10, 1e32, 1e32, 10, None, yq.ctypes.data, None,
                                 ctypes.byref(st))
    assert r == spl.ERR_CUDA
    assert np.isnan(yq).all()  # no output written by any other route
