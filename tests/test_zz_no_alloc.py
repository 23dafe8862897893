"""spl_fit_eval_noalloc, the entry point for callers that cannot allocate device memory
(applications that own all device memory themselves, or run under a hard memory budget),
checked through the C ABI against the oracle and against spl_submit with the same precision and
refinement.

This file is collected last on purpose, so that a failure here leaves every other test
already run; it passes alone in a fresh process as well."""
import numpy as np
import pytest

import oracle
from paper_2001_09253_gb300 import spl, synth
from parity_util import TOL_MIXED, ypp_error, yq_error

pytestmark = pytest.mark.gpu

NAT = spl.NATURAL
TOL_REFINED_YPP = 1e-8   # y'' after the refinement step (double-float residual)
TOL_SAME_YPP = 1e-9      # y'' of this path against spl_submit's refined y''
TOL_SAME_YQ = 1e-6       # S(x_k): both evaluate the cubic in binary32


def _rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def _noalloc(x, y, yp1, ypn, m, want_ypp=True):
    import torch
    n = len(x)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ypp = torch.full((n,), np.nan, dtype=torch.float64, device="cuda") if want_ypp else None
    yq = torch.full((max(m, 1),), np.nan, dtype=torch.float64, device="cuda") if m > 0 else None
    s, dev_status = spl.fit_eval_noalloc(xt, yt, yp1, ypn, m, ypp, yq, stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return s, dev_status, (ypp.cpu().numpy() if want_ypp else None), (yq.cpu().numpy()[:m] if m > 0 else None)


def _check_oracle(x, y, yp1, ypn, m, ypp, yq):
    ref = oracle.fit_eval(x, y, yp1, ypn, m)
    assert ref["status"] == oracle.OK
    if ypp is not None:
        e1 = ypp_error(ypp, ref["ypp"])
        assert e1 <= TOL_REFINED_YPP, "y'' error %.3e" % e1
    if m > 0:
        e2 = yq_error(x, y, ref["ypp"], ref["jq"], yq, ref["yq"])
        assert e2 <= TOL_MIXED, "S(x_k) error %.3e" % e2


def test_noalloc_matches_submit_and_oracle_on_two_calls_in_a_row():
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
        s, dev_status, ypp, yq = _noalloc(x, y, yp1, ypn, m)
        assert s == spl.OK and dev_status == spl.OK
        assert _rel(ypp, ref_ypp.cpu().numpy()) <= TOL_SAME_YPP
        assert _rel(yq, ref_yq.cpu().numpy()) <= TOL_SAME_YQ
        _check_oracle(x, y, yp1, ypn, m, ypp, yq)
    ctx.close()


@pytest.mark.parametrize("n", [3, 4, 127, 128, 129, 5000])
@pytest.mark.parametrize("bc", [(NAT, NAT), (-1.0, 1.0), (NAT, 0.5), (0.25, NAT)])
def test_noalloc_small_and_ragged_sizes_against_the_oracle(n, bc):
    x, y = synth.curve(3000 + n, n)
    for m in sorted({1, 2, n, 2 * n + 1}):
        s, dev_status, ypp, yq = _noalloc(x, y, bc[0], bc[1], m)
        assert s == spl.OK and dev_status == spl.OK
        _check_oracle(x, y, bc[0], bc[1], m, ypp, yq)


def test_noalloc_without_ypp_output_and_fit_only():
    x, y = synth.curve(77, 4099)
    s, st, ypp, yq = _noalloc(x, y, -0.5, NAT, 6000, want_ypp=False)
    assert s == spl.OK and st == spl.OK and ypp is None
    _check_oracle(x, y, -0.5, NAT, 6000, None, yq)
    s, st, ypp, yq = _noalloc(x, y, -0.5, NAT, 0)
    assert s == spl.OK and st == spl.OK and yq is None
    _check_oracle(x, y, -0.5, NAT, 0, ypp, None)


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
    s, _ = spl.fit_eval_noalloc(xt, yt, NAT, NAT, 5000, None, None)  # queries without an output
    assert s == spl.ERR_INVALID_ARG
    bad = ys.copy()
    bad[77] = np.inf
    s, st = spl.fit_eval_noalloc(xt, torch.from_numpy(bad).cuda(), NAT, NAT, 5000, None, out)
    assert s == spl.OK and st == spl.ERR_NONFINITE
    # the status word starts from zero again on the next call
    s, st = spl.fit_eval_noalloc(xt, yt, NAT, NAT, 5000, None, out)
    assert s == spl.OK and st == spl.OK
