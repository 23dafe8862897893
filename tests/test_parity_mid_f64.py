"""GPU parity of the multi-CTA FP64 latency kernel (one instance of up to SMs x 9,600 knots on a
cooperative grid of CTAs that exchange the affine maps of their partial d' and y'' solutions)
against the oracle, through the C ABI; and its bounded device-side waits."""
import time

import numpy as np
import pytest

import oracle
from paper_2001_09253_gb300 import spl, synth
from parity_util import TOL_F64, check_instance, run_gpu, ypp_error, yq_error

pytestmark = pytest.mark.gpu

NAT = oracle.NATURAL


@pytest.fixture(scope="module")
def ctx():
    c = spl.Context(device=0, arena_bytes=2 << 30, max_slots=64)
    yield c
    c.close()


def _plan(ctx, max_n=1 << 24, fault_flags=0):
    return ctx.plan(max_n=max_n, precision=spl.PREC_F64, fault_flags=fault_flags)


def _sm_count():
    import torch
    return torch.cuda.get_device_properties(0).multi_processor_count


@pytest.mark.parametrize("n", [511, 512, 513, 1000, 2048, 2049, 4096, 4097, 5000, 6143, 20000, 65537])
def test_mid_sizes_ends_and_query_counts(ctx, n):
    """One CTA up to 512 knots (pieces of up to 4 rows), several from 513 up (1-row pieces, 128
    rows per CTA, up to SMs x 128 knots; longer pieces beyond): ragged last CTAs and pieces,
    every end-condition pair, query counts below, at and above n."""
    x, y = synth.curve(6000 + n, n)
    plan = _plan(ctx)
    for bc in ((NAT, NAT), (-1.0, 1.0), (NAT, 2.0), (-3.0, NAT)):
        for m in sorted({1, 2, n, 2 * n + 1}):
            check_instance(ctx, plan, x, y, bc[0], bc[1], m)
    check_instance(ctx, plan, x, y, NAT, NAT, 0)


@pytest.mark.parametrize("which", ["staged_max", "unstaged_min", "max", "beyond", "mid"])
def test_mid_largest_instances(ctx, which):
    """The largest instance with x and y staged in shared memory (SMs x 4,096 knots, 32-row
    pieces), one knot more (33-row pieces, x and y read from global memory), the largest the path
    takes (SMs x 9,600 knots, 75-row pieces), one knot more (the tiled kernel), and 2e5 knots
    (11-row pieces)."""
    sms = _sm_count()
    n = {"staged_max": sms * 4096, "unstaged_min": sms * 4096 + 1, "max": sms * 9600, "beyond": sms * 9600 + 1,
         "mid": 200_000}[which]
    x, y = synth.curve(77, n)
    check_instance(ctx, _plan(ctx), x, y, NAT, NAT, n)
    check_instance(ctx, _plan(ctx), x, y, -1.0, 0.5, n // 3)


def test_mid_adversarial_gaps_and_far_knots(ctx):
    """8-decade gaps (y'' spanning many orders across CTA boundaries), geometric gap runs, and
    knots near 5e6 with small gaps."""
    x, y = synth.curve_adversarial(11, 100_000, decades=8)
    check_instance(ctx, _plan(ctx), x, y, NAT, NAT, 150_001)
    check_instance(ctx, _plan(ctx), x, y, 0.5, -2.0, 99_999)
    g = np.concatenate([0.7 ** np.arange(60), 0.7 ** np.arange(60)[::-1]] * 100)
    xg = np.concatenate([[0.0], np.cumsum(g)])
    for yg in (np.sin(7 * xg), np.random.default_rng(3).random(len(xg))):
        check_instance(ctx, _plan(ctx), xg, yg, NAT, NAT, 2 * len(xg))
        check_instance(ctx, _plan(ctx), xg, yg, 1.0, -1.0, len(xg))
    x, y = synth.curve(12, 30_000)
    check_instance(ctx, _plan(ctx), x + 5.0e6, y, -1.0, 1.0, 30_000)


def test_mid_consecutive_requests_reuse_the_exchange_area(ctx):
    """A single request in device memory launches the multi-CTA kernel without clearing its exchange
    area: each launch waits for flags that hold its own launch number.  Grids that shrink and grow
    between consecutive requests (the area still holding flags of earlier, larger grids) all equal
    the oracle."""
    plan = _plan(ctx)
    for i, n in enumerate([20_000, 1_000, 65_537, 600, 5_000, 20_000, 130, 65_537, 2_049]):
        x, y = synth.curve(900 + i, n)
        check_instance(ctx, plan, x, y, NAT, NAT, n)
        check_instance(ctx, plan, x, y, -1.0, 0.5, n // 2 + 1)


def test_mid_validation_errors_reported(ctx):
    """Input errors found on the device reach the request's status (the kernel ORs its status bits
    into the job's pinned status word); the context keeps working."""
    x, y = synth.curve(16, 5000)
    plan = _plan(ctx)
    bad = x.copy()
    bad[2500] = bad[2499]
    st, *_ = run_gpu(ctx, plan, bad, y, NAT, NAT, 100)
    assert st == spl.ERR_NOT_INCREASING
    bad = y.copy()
    bad[4999] = np.nan
    st, *_ = run_gpu(ctx, plan, x, bad, NAT, NAT, 100)
    assert st == spl.ERR_NONFINITE
    bad = x.copy()
    bad[0] = -np.inf
    st, *_ = run_gpu(ctx, plan, bad, y, -1.0, 1.0, 100)
    assert st == spl.ERR_NONFINITE
    check_instance(ctx, plan, x, y, NAT, NAT, 5000)


def test_mid_in_a_graph_batch(ctx):
    """One instance as a reusable batch: the cooperative launch captured in a CUDA graph and
    replayed; every replay equals the oracle."""
    import torch
    n = 30_000
    x, y = synth.curve(13, n)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ypp = torch.empty(n, dtype=torch.float64, device="cuda")
    yq = torch.empty(n, dtype=torch.float64, device="cuda")
    jq = torch.empty(n, dtype=torch.int32, device="cuda")
    b = ctx.batch(_plan(ctx), [spl.make_request(xt, yt, -1.0, 1.0, n, ypp, yq, jq)], keep=(xt, yt, ypp, yq, jq))
    ref = oracle.fit_eval(x, y, -1.0, 1.0, n)
    for _ in range(3):
        ypp.fill_(float("nan"))
        b.launch()
        assert (b.wait() == 0).all()
        assert np.array_equal(jq.cpu().numpy().astype(np.int64), ref["jq"])
        assert ypp_error(ypp.cpu().numpy(), ref["ypp"]) <= TOL_F64
        assert yq_error(x, y, ref["ypp"], ref["jq"], yq.cpu().numpy(), ref["yq"]) <= TOL_F64
    b.close()


def test_mid_wait_timeout_reported_and_context_usable(ctx):
    """Failure detection without a GPU fault: the last CTA withholds its maps (plan fault bit 0),
    the other CTAs' bounded waits run out, the request completes with SPL_ERR_TIMEOUT within a
    second, and the context serves the next request normally."""
    import torch
    n = 20_000
    x, y = synth.curve(14, n)
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    ypp = torch.empty(n, dtype=torch.float64, device="cuda")
    yq = torch.empty(n, dtype=torch.float64, device="cuda")
    t0 = time.perf_counter()
    st, res = ctx.wait(ctx.submit(_plan(ctx, fault_flags=1), xt, yt, NAT, NAT, n, ypp, yq), 10.0)
    assert st == spl.ERR_TIMEOUT and res.status == spl.ERR_TIMEOUT  # completed, not still pending
    assert time.perf_counter() - t0 < 5.0
    check_instance(ctx, _plan(ctx), x, y, NAT, NAT, n)


def test_fault_flags_validated(ctx):
    with pytest.raises(spl.SplError):
        _plan(ctx, fault_flags=2)


def test_direct_requests_in_flight_together(ctx):
    """Single requests in device memory queued back to back without waiting (each launched as its
    kernel alone, on the context's one stream): multi-CTA FP64 requests of changing grids and
    binary32 requests with and without the refinement step share the context's exchange area and
    tile counter in stream order.  Every result equals the oracle."""
    import torch
    f64 = _plan(ctx)
    f32 = ctx.plan(max_n=1 << 22, precision=spl.PREC_F32_REFINE, refine_steps=0)
    f32r = ctx.plan(max_n=1 << 22, precision=spl.PREC_F32_REFINE, refine_steps=1)
    # (plan, n, S tolerance, y'' tolerance): the refined y'' to 1e-8, as for refined batches
    F64, F32, F32R = (f64, TOL_F64, TOL_F64), (f32, 1e-5, 1e-5), (f32r, 1e-5, 1e-8)
    cases = [(F64, 20_000), (F32R, 5_000), (F64, 1_000), (F32, 300_000), (F64, 65_537), (F32R, 129),
             (F64, 600), (F32, 97_280), (F64, 3_001), (F32R, 200_000)]
    runs = []
    for i, ((plan, tol, tol_ypp), n) in enumerate(cases):
        x, y = synth.curve(970 + i, n)
        bc = (NAT, NAT) if i % 2 == 0 else (-1.0, 0.5)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ypp = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        yq = torch.full((n,), float("nan"), dtype=torch.float64, device="cuda")
        jq = torch.full((n,), -7, dtype=torch.int32, device="cuda")
        t = ctx.submit(plan, xt, yt, bc[0], bc[1], n, ypp, yq, jq)
        runs.append((t, x, y, bc, n, tol, tol_ypp, (xt, yt, ypp, yq, jq)))
    for t, x, y, bc, n, tol, tol_ypp, (xt, yt, ypp, yq, jq) in runs:
        st, _ = ctx.wait(t, 60.0)
        assert st == spl.OK
        ref = oracle.fit_eval(x, y, bc[0], bc[1], n)
        assert np.array_equal(jq.cpu().numpy().astype(np.int64), ref["jq"])
        assert ypp_error(ypp.cpu().numpy(), ref["ypp"]) <= tol_ypp
        assert yq_error(x, y, ref["ypp"], ref["jq"], yq.cpu().numpy(), ref["yq"]) <= tol
