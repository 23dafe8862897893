"""spl_fit_eval_noalloc, the entry point for callers that cannot allocate device memory
(applications that own all device memory themselves, or run under a hard memory budget),
checked through the C ABI against spl_submit with the same precision and refinement.

This file is collected last on purpose, so that a failure here leaves every other test
already run; it passes alone in a fresh process as well."""
import numpy as np
import pytest

from paper_2001_09253_gb300 import spl, synth

pytestmark = pytest.mark.gpu

NAT = spl.NATURAL
TOL = 1e-5  # the mixed-precision tolerance of the parity tests


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def test_noalloc_matches_submit_on_two_calls_in_a_row():
    import torch
    ctx = spl.Context(device=0, arena_bytes=1 << 30, max_slots=16)
    plan = ctx.plan(max_n=spl.NOALLOC_MAX_N, precision=spl.PREC_F32_REFINE, refine_steps=1)
    cases = [(200_003, 40, NAT, NAT, 250_000), (spl.NOALLOC_MAX_N, 41, -1.0, 0.5, 777_777)]
    for n, seed, yp1, ypn, m in cases:  # two calls in a row; the second reuses the scratch
        x, y = synth.curve(seed, n)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ref_ypp = torch.empty(n, dtype=torch.float64, device="cuda")
        ref_yq = torch.empty(m, dtype=torch.float64, device="cuda")
        t = ctx.submit(plan, xt, yt, yp1, ypn, m, ref_ypp, ref_yq)
        s, _ = ctx.wait(t)
        assert s == spl.OK
        ypp = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        yq = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
        s, dev_status = spl.fit_eval_noalloc(xt, yt, yp1, ypn, m, ypp, yq, stream=torch.cuda.current_stream())
        assert s == spl.OK and dev_status == spl.OK
        torch.cuda.synchronize()
        assert _rel(ypp.cpu().numpy(), ref_ypp.cpu().numpy()) <= TOL
        assert _rel(yq.cpu().numpy(), ref_yq.cpu().numpy()) <= TOL
    ctx.close()


def test_noalloc_limits_and_errors():
    import torch
    n = spl.NOALLOC_MAX_N + 1
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    s, _ = spl.fit_eval_noalloc(x, x, NAT, NAT, 0)
    assert s == spl.ERR_BUDGET
    s, _ = spl.fit_eval_noalloc(x[:2], x[:2], NAT, NAT, 0)
    assert s == spl.ERR_INVALID_ARG
    xs, ys = synth.curve(42, 5000)
    xt, yt = torch.from_numpy(xs).cuda(), torch.from_numpy(ys).cuda()
    out = torch.empty(5000, dtype=torch.float64, device="cuda")
    s, _ = spl.fit_eval_noalloc(xt, yt, float("nan"), NAT, 5000, None, out)
    assert s == spl.ERR_INVALID_ARG
    bad = ys.copy()
    bad[77] = np.inf
    s, st = spl.fit_eval_noalloc(xt, torch.from_numpy(bad).cuda(), NAT, NAT, 5000, None, out)
    assert s == spl.OK and st == spl.ERR_NONFINITE
    # the status word starts from zero again on the next call
    s, st = spl.fit_eval_noalloc(xt, yt, NAT, NAT, 5000, None, out)
    assert s == spl.OK and st == spl.OK
