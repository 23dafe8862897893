"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI and the
oracle on the same seeded inputs, and compare with the stated tolerances.

Error measures (the same in every parity test):
  * bracket indices: bit-exact;
  * y'': normwise, max|d| / max|y''_oracle|;
  * S(x_k): per query, |d_k| / scale_k with
        scale_k = max(|y_j|, |y_{j+1}|, |S_k|, h_j^2 max(|y''_j|, |y''_{j+1}|) / 6)
    (the magnitudes of the terms of the interpolation form on interval j).
"""
from __future__ import annotations

import numpy as np

import oracle

TOL_F64 = 1e-12
TOL_MIXED = 1e-5


def ypp_error(got, ref) -> float:
    got, ref = np.asarray(got, float), np.asarray(ref, float)
    if ref.size == 0:
        return 0.0
    return float(np.max(np.abs(got - ref)) / max(float(np.max(np.abs(ref))), 1e-300))


def yq_error(x, y, ypp_ref, jq, yq_got, yq_ref) -> float:
    if len(yq_ref) == 0:
        return 0.0
    j = np.asarray(jq, dtype=np.int64)
    h = x[j + 1] - x[j]
    curv = h * h * np.maximum(np.abs(ypp_ref[j]), np.abs(ypp_ref[j + 1])) / 6.0
    scale = np.maximum.reduce([np.abs(y[j]), np.abs(y[j + 1]), np.abs(yq_ref), curv, np.full(len(j), 1e-300)])
    return float(np.max(np.abs(np.asarray(yq_got) - yq_ref) / scale))


def run_gpu(ctx, plan, x, y, yp1, ypn, m, want_ypp=True, want_jq=True, device_inputs=True):
    """One instance through spl_submit + spl_wait.  Returns (status, ypp, yq, jq) as numpy."""
    import torch
    n = len(x)
    dev = torch.device("cuda", ctx.device)
    if device_inputs:
        xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
        yt = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
        ypp = torch.full((n,), np.nan, dtype=torch.float64, device=dev) if want_ypp else None
        yq = torch.full((max(m, 1),), np.nan, dtype=torch.float64, device=dev)
        jq = torch.full((max(m, 1),), -7, dtype=torch.int32, device=dev) if want_jq else None
    else:
        xt = torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
        yt = torch.from_numpy(np.ascontiguousarray(y)).pin_memory()
        ypp = torch.full((n,), np.nan, dtype=torch.float64).pin_memory() if want_ypp else None
        yq = torch.full((max(m, 1),), np.nan, dtype=torch.float64).pin_memory()
        jq = torch.full((max(m, 1),), -7, dtype=torch.int32).pin_memory() if want_jq else None
    t = ctx.submit(plan, xt, yt, yp1, ypn, m, ypp, yq if m > 0 else None, jq if m > 0 else None)
    st, _ = ctx.wait(t, 120.0)
    torch.cuda.synchronize(dev)
    out_ypp = ypp.cpu().numpy() if ypp is not None else None
    return st, out_ypp, yq.cpu().numpy()[:m], (jq.cpu().numpy()[:m] if jq is not None else None)


def check_instance(ctx, plan, x, y, yp1, ypn, m, tol=TOL_F64, device_inputs=True):
    """Run both sides and assert parity; returns (ypp_err, yq_err)."""
    ref = oracle.fit_eval(x, y, yp1, ypn, m)
    assert ref["status"] == oracle.OK
    st, ypp, yq, jq = run_gpu(ctx, plan, x, y, yp1, ypn, m, device_inputs=device_inputs)
    assert st == 0, "GPU status %d" % st
    e1 = ypp_error(ypp, ref["ypp"])
    assert e1 <= tol, "y'' error %.3e" % e1
    if m > 0:
        assert np.array_equal(jq.astype(np.int64), ref["jq"]), "bracket indices differ at %s" % (
            np.nonzero(jq.astype(np.int64) != ref["jq"])[0][:10],)
        e2 = yq_error(x, y, ref["ypp"], ref["jq"], yq, ref["yq"])
        assert e2 <= tol, "S(x_k) error %.3e" % e2
    else:
        e2 = 0.0
    return e1, e2
