"""GPU parity of the plain FP64 path against the oracle, through the C ABI."""
import numpy as np
import pytest

import oracle
from paper_2001_09253_gb300 import spl, synth
from parity_util import TOL_F64, check_instance, run_gpu, ypp_error, yq_error

pytestmark = pytest.mark.gpu

NAT = oracle.NATURAL


@pytest.fixture(scope="module")
def ctx():
    c = spl.Context(device=0, arena_bytes=2 << 30, max_slots=8192)
    yield c
    c.close()


def _plan(ctx, tile_rows=0, max_n=1 << 26):
    return ctx.plan(max_n=max_n, precision=spl.PREC_F64, tile_rows=tile_rows)


@pytest.mark.parametrize("bc", [(NAT, NAT), (-1.0, 1.0), (0.0, 0.0), (NAT, 2.0), (-3.0, NAT)])
def test_smallest_config_n1000(ctx, bc):
    """n = M = 1000, seed 0: auto tiling and forced small tiles (many halos, ragged tail)."""
    x, y = synth.curve(0, 1000)
    for L in (0, 16, 37, 150):
        check_instance(ctx, _plan(ctx, L), x, y, bc[0], bc[1], 1000)


@pytest.mark.parametrize("n", [3, 4, 5, 16, 17, 31, 32, 33, 63, 64, 65, 127, 128, 129, 200, 257])
@pytest.mark.parametrize("L", [16, 64, 100])
def test_sizes_and_tiles(ctx, n, L):
    x, y = synth.curve(1000 + n, n)
    for m in sorted({0, 1, 2, 3, n, 2 * n + 1, max(2, n // 3)}):
        check_instance(ctx, _plan(ctx, L), x, y, -1.0, 1.0, m)
        check_instance(ctx, _plan(ctx, L), x, y, NAT, NAT, m)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_adversarial_gap_ratios(ctx, seed):
    """Gaps spread over 8 decades: the halo truncation must stay invisible."""
    x, y = synth.curve_adversarial(seed, 5000, decades=8)
    for L in (16, 300, 0):
        check_instance(ctx, _plan(ctx, L), x, y, NAT, NAT, 7001)
        check_instance(ctx, _plan(ctx, L), x, y, 0.5, -2.0, 3000)


def test_geometric_gaps_worst_case_decay(ctx):
    """Gaps shrinking and growing geometrically push c' and a/(b - a c') toward their bounds."""
    g = np.concatenate([0.7 ** np.arange(60), 0.7 ** np.arange(60)[::-1]] * 20)
    x = np.concatenate([[0.0], np.cumsum(g)])
    rough = np.random.default_rng(0).random(len(x))
    # smooth data makes d_j = 6(s_j - s_{j-1}) cancel at the tiny gaps: slopes must be
    # correctly rounded quotients on both sides for the results to agree
    for y in (np.sin(7 * x), rough):
        for L in (16, 40, 0):
            check_instance(ctx, _plan(ctx, L), x, y, NAT, NAT, 4 * len(x))
            check_instance(ctx, _plan(ctx, L), x, y, 1.0, -1.0, len(x))


def test_host_memory_requests(ctx):
    x, y = synth.curve(5, 20000)
    check_instance(ctx, _plan(ctx), x, y, NAT, NAT, 20000, device_inputs=False)
    check_instance(ctx, _plan(ctx, 64), x, y, -1.0, 1.0, 777, device_inputs=False)


def test_validation_errors_reported(ctx):
    x, y = synth.curve(6, 3000)
    p = _plan(ctx, 64)
    bad = x.copy()
    bad[1700] = bad[1699]
    st, *_ = run_gpu(ctx, p, bad, y, NAT, NAT, 100)
    assert st == spl.ERR_NOT_INCREASING
    bad = y.copy()
    bad[2999] = np.nan
    st, *_ = run_gpu(ctx, p, x, bad, NAT, NAT, 100)
    assert st == spl.ERR_NONFINITE
    bad = x.copy()
    bad[0] = -np.inf
    st, *_ = run_gpu(ctx, p, bad, y, NAT, NAT, 100)
    assert st == spl.ERR_NONFINITE
    # the context keeps working after device-side errors
    check_instance(ctx, p, x, y, NAT, NAT, 3000)


def test_invalid_arguments_rejected_on_host(ctx):
    import torch
    p = _plan(ctx, 0, max_n=1000)
    x = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(spl.SplError) as e:
        ctx.submit(p, x, x, NAT, NAT, 0)
    assert e.value.status == spl.ERR_INVALID_ARG
    x, y = synth.curve(0, 10)
    xt = torch.from_numpy(x).cuda()
    yt = torch.from_numpy(y).cuda()
    out = torch.empty(10, dtype=torch.float64, device="cuda")
    for yp1 in (np.nan, -np.inf):
        with pytest.raises(spl.SplError) as e:
            ctx.submit(p, xt, yt, yp1, NAT, 10, None, out)
        assert e.value.status == spl.ERR_INVALID_ARG
    with pytest.raises(spl.SplError) as e:  # m > 0 needs an output
        ctx.submit(p, xt, yt, NAT, NAT, 10, None, None)
    assert e.value.status == spl.ERR_INVALID_ARG
    x2, y2 = synth.curve(0, 2000)
    with pytest.raises(spl.SplError) as e:  # beyond the plan's max_n
        ctx.submit(p, torch.from_numpy(x2).cuda(), torch.from_numpy(y2).cuda(), NAT, NAT, 0)
    assert e.value.status == spl.ERR_INVALID_ARG


def test_batch_many_instances_with_one_bad(ctx):
    import torch
    sizes = [3, 50, 1000, 4097, 100, 7, 20000, 333]
    plan = _plan(ctx, 128)
    reqs, keep, refs = [], [], []
    for i, n in enumerate(sizes):
        x, y = synth.curve(42, n, instance=i)
        if i == 5:
            y = y.copy()
            y[3] = np.inf
        bc = (NAT, NAT) if i % 2 == 0 else (-1.0, 1.0)
        m = n + (i * 37) % 101
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ypp = torch.empty(n, dtype=torch.float64, device="cuda")
        yq = torch.empty(m, dtype=torch.float64, device="cuda")
        jq = torch.empty(m, dtype=torch.int32, device="cuda")
        reqs.append(spl.make_request(xt, yt, bc[0], bc[1], m, ypp, yq, jq))
        keep.append((xt, yt, ypp, yq, jq))
        refs.append((x, y, bc, m))
    tickets = ctx.submit_batch(plan, reqs, keep)
    for i, t in enumerate(tickets):
        st, _ = ctx.wait(t)
        x, y, bc, m = refs[i]
        if i == 5:
            assert st == spl.ERR_NONFINITE
            continue
        assert st == 0
        ref = oracle.fit_eval(x, y, bc[0], bc[1], m)
        _, _, ypp, yq, jq = keep[i]
        assert ypp_error(ypp.cpu().numpy(), ref["ypp"]) <= TOL_F64
        assert np.array_equal(jq.cpu().numpy().astype(np.int64), ref["jq"])
        assert yq_error(x, y, ref["ypp"], ref["jq"], yq.cpu().numpy(), ref["yq"]) <= TOL_F64


def test_graph_batch_replays(ctx):
    import torch
    sizes = synth.sizes_loguniform(2, 64, 1e2, 1e4)
    plan = _plan(ctx)
    reqs, keep, refs = [], [], []
    for i, n in enumerate(sizes):
        x, y = synth.curve(2, int(n), instance=i)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ypp = torch.empty(int(n), dtype=torch.float64, device="cuda")
        yq = torch.empty(int(n), dtype=torch.float64, device="cuda")
        reqs.append(spl.make_request(xt, yt, NAT, NAT, int(n), ypp, yq))
        keep.append((xt, yt, ypp, yq))
        refs.append((x, y))
    b = ctx.batch(plan, reqs, keep)
    for rep in range(2):
        for k in keep:
            k[3].fill_(np.nan)
        b.launch()
        st = b.wait()
        assert (st == 0).all()
        for (x, y), k in zip(refs, keep):
            ref = oracle.fit_eval(x, y, NAT, NAT, len(x))
            assert ypp_error(k[2].cpu().numpy(), ref["ypp"]) <= TOL_F64
            assert yq_error(x, y, ref["ypp"], ref["jq"], k[3].cpu().numpy(), ref["yq"]) <= TOL_F64
    b.close()


@pytest.mark.parametrize("n", [1, 2, 3, 4096, 4097, 100000, 1000003])
def test_device_generator_bit_identical(n):
    x, y = spl.generate_curve(9, n, instance=3)
    hx, hy = synth.curve(9, n, instance=3)
    assert np.array_equal(x.cpu().numpy(), hx)
    assert np.array_equal(y.cpu().numpy(), hy)


def test_full_size_n1e7(ctx):
    """n = M = 10^7, seed 1 (the benchmark workload), in the benchmark's launch
    configuration; every output compared with the oracle."""
    import torch
    n = 10_000_000
    x, y = spl.generate_curve(1, n)
    hx, hy = synth.curve(1, n)
    assert np.array_equal(x.cpu().numpy(), hx)
    ypp = torch.empty(n, dtype=torch.float64, device="cuda")
    yq = torch.empty(n, dtype=torch.float64, device="cuda")
    jq = torch.empty(n, dtype=torch.int32, device="cuda")
    plan = _plan(ctx)
    t = ctx.submit(plan, x, y, NAT, NAT, n, ypp, yq, jq)
    st, _ = ctx.wait(t, 300)
    assert st == 0
    ref = oracle.fit_eval(hx, hy, NAT, NAT, n)
    assert ypp_error(ypp.cpu().numpy(), ref["ypp"]) <= TOL_F64
    assert np.array_equal(jq.cpu().numpy().astype(np.int64), ref["jq"])
    assert yq_error(hx, hy, ref["ypp"], ref["jq"], yq.cpu().numpy(), ref["yq"]) <= TOL_F64


@pytest.mark.parametrize("n", [3, 4, 5, 127, 128, 129, 255, 256, 257, 1000, 2047, 4095, 4096, 4097])
def test_small_instances_one_cta(ctx, n):
    """Automatic tiling sends single FP64 instances to the latency kernel: one CTA up to 512 knots
    (pieces of ceil(n / 128) rows, block scans of the d' and y'' maps), several CTAs above
    (test_parity_mid_f64.py).  Every end-condition pair, query counts below, at and above n."""
    x, y = synth.curve(4000 + n, n)
    plan = _plan(ctx, 0)
    for bc in ((NAT, NAT), (-1.0, 1.0), (NAT, 2.0), (-3.0, NAT)):
        for m in sorted({0, 1, 2, n, 2 * n + 1}):
            check_instance(ctx, plan, x, y, bc[0], bc[1], m)


def test_small_instances_adversarial_and_far_knots(ctx):
    """The latency kernels on 8-decade gaps and on knots near 5e6 with small gaps."""
    x, y = synth.curve_adversarial(7, 3000, decades=8)
    check_instance(ctx, _plan(ctx, 0), x, y, NAT, NAT, 4001)
    check_instance(ctx, _plan(ctx, 0), x, y, 0.5, -2.0, 2999)
    x, y = synth.curve(8, 2500)
    check_instance(ctx, _plan(ctx, 0), x + 5.0e6, y, -1.0, 1.0, 2500)


def test_many_small_instances_take_the_tiled_kernel(ctx):
    """More than two waves of small FP64 instances (700 > 4 x SMs on GB300) run the tiled kernel:
    a sample of them against the oracle, with clamped and natural ends."""
    import torch
    plan = _plan(ctx, 0)
    rng = np.random.default_rng(60)
    sizes = rng.integers(3, 2001, 700)
    reqs, keep, refs = [], [], []
    for i, n in enumerate(sizes):
        n = int(n)
        x, y = synth.curve(61, n, instance=i)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ypp = torch.empty(n, dtype=torch.float64, device="cuda")
        yq = torch.empty(n, dtype=torch.float64, device="cuda")
        bc = (NAT, NAT) if i % 2 else (-1.0, 0.5)
        reqs.append(spl.make_request(xt, yt, bc[0], bc[1], n, ypp, yq))
        keep.append((xt, yt, ypp, yq))
        refs.append((x, y, bc))
    tickets = ctx.submit_batch(plan, reqs, keep)
    for t in tickets:
        st, _ = ctx.wait(t)
        assert st == 0
    for i in rng.choice(len(sizes), size=60, replace=False):
        x, y, bc = refs[i]
        ref = oracle.fit_eval(x, y, bc[0], bc[1], len(x))
        assert ypp_error(keep[i][2].cpu().numpy(), ref["ypp"]) <= TOL_F64
        assert yq_error(x, y, ref["ypp"], ref["jq"], keep[i][3].cpu().numpy(), ref["yq"]) <= TOL_F64


def test_small_instances_batched_and_errors(ctx):
    """Several small FP64 instances in one launch (one CTA each) with one bad instance."""
    import torch
    plan = _plan(ctx, 0)
    sizes = [3, 1000, 17, 4096, 640]
    reqs, keep, refs = [], [], []
    for i, n in enumerate(sizes):
        x, y = synth.curve(50 + i, n)
        if i == 2:
            x = x.copy()
            x[5] = x[4]
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ypp = torch.empty(n, dtype=torch.float64, device="cuda")
        yq = torch.empty(n + 3, dtype=torch.float64, device="cuda")
        reqs.append(spl.make_request(xt, yt, NAT, NAT, n + 3, ypp, yq))
        keep.append((xt, yt, ypp, yq))
        refs.append((x, y))
    for i, (t, (x, y), k) in enumerate(zip(ctx.submit_batch(plan, reqs, keep), refs, keep)):
        st, _ = ctx.wait(t)
        if i == 2:
            assert st == spl.ERR_NOT_INCREASING
            continue
        assert st == 0
        ref = oracle.fit_eval(x, y, NAT, NAT, len(x) + 3)
        assert ypp_error(k[2].cpu().numpy(), ref["ypp"]) <= TOL_F64
        assert yq_error(x, y, ref["ypp"], ref["jq"], k[3].cpu().numpy(), ref["yq"]) <= TOL_F64
