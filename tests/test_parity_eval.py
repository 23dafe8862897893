"""GPU parity of the separate evaluation kernel against the oracle: explicit, unsorted query
arrays bracketed by bisection (bit-exact indices), the three forms of section "Fast
Interpolation" (orig / noinv / vol), and "fit once, evaluate many" with a stored y''."""
import numpy as np
import pytest

import oracle
from paper_2001_09253_gb300 import synth
from parity_util import TOL_F64, ypp_error, yq_error

pytestmark = pytest.mark.gpu

NAT = oracle.NATURAL


@pytest.fixture(scope="module")
def ctx():
    from paper_2001_09253_gb300 import spl
    c = spl.Context(0, arena_bytes=2 << 30, max_slots=64)
    yield c
    c.close()


def _queries(x, m, rng):
    """Unsorted positions: interior, exact knots, below x_0, above x_{n-1}, duplicates."""
    lo, hi = float(x[0]), float(x[-1])
    span = hi - lo
    q = [rng.uniform(lo, hi, size=m)]
    q.append(rng.choice(x, size=max(m // 10, 1)))
    q.append(lo - span * rng.random(max(m // 50, 1)))
    q.append(hi + span * rng.random(max(m // 50, 1)))
    q.append(np.array([lo, hi, np.nextafter(lo, -np.inf), np.nextafter(hi, np.inf)]))
    q = np.concatenate(q)
    q = np.concatenate([q, q[: max(m // 20, 1)]])  # duplicates
    rng.shuffle(q)
    return q.astype(np.float64)


def _run(ctx, plan, x, y, xq, yp1=NAT, ypn=NAT, ypp_in=None, want_ypp=True):
    import torch
    dev = torch.device("cuda", ctx.device)
    n, m = len(x), len(xq)
    xt = torch.from_numpy(np.ascontiguousarray(x)).to(dev)
    yt = torch.from_numpy(np.ascontiguousarray(y)).to(dev)
    qt = torch.from_numpy(np.ascontiguousarray(xq)).to(dev)
    ypp = torch.full((n,), np.nan, dtype=torch.float64, device=dev) if want_ypp else None
    yq = torch.full((max(m, 1),), np.nan, dtype=torch.float64, device=dev)
    jq = torch.full((max(m, 1),), -7, dtype=torch.int32, device=dev)
    pin = torch.from_numpy(np.ascontiguousarray(ypp_in)).to(dev) if ypp_in is not None else None
    t = ctx.submit(plan, xt, yt, yp1, ypn, m, ypp, yq if m else None, jq if m else None, xq=qt if m else None,
                   ypp_in=pin)
    st, _ = ctx.wait(t, 120.0)
    torch.cuda.synchronize(dev)
    return st, (ypp.cpu().numpy() if ypp is not None else None), yq.cpu().numpy()[:m], jq.cpu().numpy()[:m]


def _check(x, y, ypp_ref, xq, yq, jq, tol=TOL_F64):
    jref = oracle.bracket_any(x, xq)
    assert np.array_equal(jq.astype(np.int64), jref), np.nonzero(jq != jref)[0][:10]
    yref = oracle.evaluate(x, y, ypp_ref, xq, jref)
    e = yq_error(x, y, ypp_ref, jref, yq, yref)
    assert e <= tol, "S(x) error %.3e" % e
    return e


@pytest.mark.parametrize("variant", [0, 1, 2])
def test_explicit_unsorted_queries_all_variants(ctx, variant):
    rng = np.random.default_rng(10 + variant)
    x, y = synth.curve(21, 5000)
    xq = _queries(x, 7000, rng)
    from paper_2001_09253_gb300 import spl
    plan = ctx.plan(len(x), spl.PREC_F64, query_mode=spl.QUERY_EXPLICIT, eval_variant=variant)
    for yp1, ypn in ((NAT, NAT), (-0.75, 2.0)):
        ref = oracle.fit_eval(x, y, yp1, ypn, 0)
        st, ypp, yq, jq = _run(ctx, plan, x, y, xq, yp1, ypn)
        assert st == 0
        assert ypp_error(ypp, ref["ypp"]) <= TOL_F64
        _check(x, y, ref["ypp"], xq, yq, jq)


def test_explicit_adversarial_knots_and_tiles(ctx):
    from paper_2001_09253_gb300 import spl
    rng = np.random.default_rng(3)
    x, y = synth.curve_adversarial(4, 6000, decades=8)
    xq = _queries(x, 9000, rng)
    ref = oracle.fit_eval(x, y, NAT, NAT, 0)
    for L in (16, 300, 0):
        plan = ctx.plan(len(x), spl.PREC_F64, tile_rows=L, query_mode=spl.QUERY_EXPLICIT)
        st, ypp, yq, jq = _run(ctx, plan, x, y, xq)
        assert st == 0
        assert ypp_error(ypp, ref["ypp"]) <= TOL_F64
        _check(x, y, ref["ypp"], xq, yq, jq)


def test_fit_once_evaluate_many(ctx):
    """One fit (uniform plan, m = 0), then repeated evaluations from the stored y'': explicit
    batches and a uniform grid, every variant, without refitting."""
    import torch
    from paper_2001_09253_gb300 import spl
    x, y = synth.curve(22, 20000)
    ref = oracle.fit_eval(x, y, 1.5, -0.5, 0)
    fit_plan = ctx.plan(len(x), spl.PREC_F64)
    st, ypp, _, _ = _run(ctx, fit_plan, x, y, np.zeros(0), 1.5, -0.5)
    assert st == 0 and ypp_error(ypp, ref["ypp"]) <= TOL_F64
    launches0 = ctx.stats()["kernel_launches"]
    rng = np.random.default_rng(5)
    for variant in (0, 1, 2):
        ev = ctx.plan(len(x), spl.PREC_F64, query_mode=spl.QUERY_EXPLICIT, eval_variant=variant)
        for _ in range(2):
            xq = _queries(x, 3000, rng)
            st, out_ypp, yq, jq = _run(ctx, ev, x, y, xq, ypp_in=ypp, want_ypp=False)
            assert st == 0 and out_ypp is None
            # evaluated against the GPU's own y'' (the stored fit) and against the oracle's
            _check(x, y, ypp, xq, yq, jq)
            _check(x, y, ref["ypp"], xq, yq, jq)
    # one evaluation kernel per call, no fit
    assert ctx.stats()["kernel_launches"] - launches0 == 6
    # uniform grid from the stored y'': same brackets and values as the fused path
    dev = torch.device("cuda", ctx.device)
    m = 31337
    yq = torch.full((m,), np.nan, dtype=torch.float64, device=dev)
    jq = torch.full((m,), -7, dtype=torch.int32, device=dev)
    xt = torch.from_numpy(x).to(dev)
    yt = torch.from_numpy(y).to(dev)
    t = ctx.submit(fit_plan, xt, yt, 1.5, -0.5, m, None, yq, jq, ypp_in=torch.from_numpy(ypp).to(dev))
    st, _ = ctx.wait(t, 60.0)
    assert st == 0
    full = oracle.fit_eval(x, y, 1.5, -0.5, m)
    assert np.array_equal(jq.cpu().numpy().astype(np.int64), full["jq"])
    e = yq_error(x, y, full["ypp"], full["jq"], yq.cpu().numpy(), full["yq"])
    assert e <= TOL_F64


def test_explicit_batch_mixed_sizes(ctx):
    """Several instances in one launch: the query-to-instance map, an instance without queries."""
    import torch
    from paper_2001_09253_gb300 import spl
    dev = torch.device("cuda", ctx.device)
    plan = ctx.plan(50000, spl.PREC_F64, query_mode=spl.QUERY_EXPLICIT)
    rng = np.random.default_rng(9)
    reqs, keep, cases = [], [], []
    for i, (n, m) in enumerate([(3, 7), (100, 0), (4097, 5000), (50000, 1), (777, 2000)]):
        x, y = synth.curve(30, n, instance=i)
        xq = _queries(x, m, rng)[:m] if m else np.zeros(0)
        xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
        qt = torch.from_numpy(np.ascontiguousarray(xq)).to(dev)
        ypp = torch.full((n,), np.nan, dtype=torch.float64, device=dev)
        yq = torch.full((max(m, 1),), np.nan, dtype=torch.float64, device=dev)
        jq = torch.full((max(m, 1),), -7, dtype=torch.int32, device=dev)
        reqs.append(spl.make_request(xt, yt, NAT, NAT, m, ypp, yq if m else None, jq if m else None,
                                     xq=qt if m else None))
        keep += [xt, yt, qt, ypp, yq, jq]
        cases.append((x, y, xq, ypp, yq, jq, m))
    ts = ctx.submit_batch(plan, reqs, keep)
    for t in ts:
        st, _ = ctx.wait(t, 60.0)
        assert st == 0
    for x, y, xq, ypp, yq, jq, m in cases:
        ref = oracle.fit_eval(x, y, NAT, NAT, 0)
        assert ypp_error(ypp.cpu().numpy(), ref["ypp"]) <= TOL_F64
        if m:
            _check(x, y, ref["ypp"], xq, yq.cpu().numpy()[:m], jq.cpu().numpy()[:m])


def test_explicit_host_memory(ctx):
    from paper_2001_09253_gb300 import spl
    import torch
    x, y = synth.curve(23, 3000)
    rng = np.random.default_rng(4)
    xq = _queries(x, 2500, rng)
    ref = oracle.fit_eval(x, y, NAT, NAT, 0)
    plan = ctx.plan(len(x), spl.PREC_F64, query_mode=spl.QUERY_EXPLICIT, eval_variant=1)
    hx = torch.from_numpy(x).pin_memory()
    hy = torch.from_numpy(y).pin_memory()
    hq = torch.from_numpy(xq).pin_memory()
    ypp = torch.full((len(x),), np.nan, dtype=torch.float64).pin_memory()
    yq = torch.full((len(xq),), np.nan, dtype=torch.float64).pin_memory()
    jq = torch.full((len(xq),), -7, dtype=torch.int32).pin_memory()
    st, _ = ctx.wait(ctx.submit(plan, hx, hy, NAT, NAT, len(xq), ypp, yq, jq, xq=hq), 60.0)
    assert st == 0
    assert ypp_error(ypp.numpy(), ref["ypp"]) <= TOL_F64
    _check(x, y, ref["ypp"], xq, yq.numpy(), jq.numpy())
    # evaluation only, from a host copy of the stored y''
    hpp = torch.from_numpy(ref["ypp"].copy()).pin_memory()
    yq2 = torch.full((len(xq),), np.nan, dtype=torch.float64).pin_memory()
    jq2 = torch.full((len(xq),), -7, dtype=torch.int32).pin_memory()
    st, _ = ctx.wait(ctx.submit(plan, hx, hy, NAT, NAT, len(xq), None, yq2, jq2, xq=hq, ypp_in=hpp), 60.0)
    assert st == 0
    _check(x, y, ref["ypp"], xq, yq2.numpy(), jq2.numpy())


def test_explicit_errors(ctx):
    import torch
    from paper_2001_09253_gb300 import spl
    dev = torch.device("cuda", ctx.device)
    x, y = synth.curve(24, 500)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    # unknown modes and variants are refused
    for kw in ({"query_mode": 2}, {"eval_variant": 4}, {"eval_variant": -1}):
        with pytest.raises(spl.SplError) as ei:
            ctx.plan(500, **kw)
        assert ei.value.status == spl.ERR_INVALID_ARG
    uni = ctx.plan(500, spl.PREC_F64)
    exp = ctx.plan(500, spl.PREC_F64, query_mode=spl.QUERY_EXPLICIT)
    q = torch.linspace(float(x[0]), float(x[-1]), 10, dtype=torch.float64, device=dev)
    yq = torch.empty(10, dtype=torch.float64, device=dev)
    with pytest.raises(spl.SplError):  # positions given to a uniform plan
        ctx.submit(uni, xt, yt, NAT, NAT, 10, None, yq, None, xq=q)
    with pytest.raises(spl.SplError):  # explicit plan without positions
        ctx.submit(exp, xt, yt, NAT, NAT, 10, None, yq, None)
    # a non-finite query position completes with SPL_ERR_NONFINITE
    bad = q.clone()
    bad[3] = float("nan")
    st, _ = ctx.wait(ctx.submit(exp, xt, yt, NAT, NAT, 10, None, yq, None, xq=bad), 60.0)
    assert st == spl.ERR_NONFINITE
    # requests of one call must agree on a stored y''
    ypp = torch.zeros(500, dtype=torch.float64, device=dev)
    r1 = spl.make_request(xt, yt, NAT, NAT, 10, None, yq, None, xq=q, ypp_in=ypp)
    r2 = spl.make_request(xt, yt, NAT, NAT, 10, None, yq, None, xq=q)
    with pytest.raises(spl.SplError) as ei:
        ctx.submit_batch(exp, [r1, r2], (xt, yt, q, yq, ypp))
    assert ei.value.status == spl.ERR_INVALID_ARG


def test_explicit_large_sampled(ctx):
    """n = 2e6 knots, 2e6 unsorted queries (the full-size scale of the separate evaluation):
    every bracket against the oracle's bisection, values on a sample."""
    import torch
    from paper_2001_09253_gb300 import spl
    n = 2_000_000
    dev = torch.device("cuda", ctx.device)
    x, y = spl.generate_curve(25, n)
    torch.cuda.synchronize(dev)
    rng = np.random.default_rng(8)
    xh = x.cpu().numpy()
    xq = rng.uniform(float(xh[0]) - 1.0, float(xh[-1]) + 1.0, size=n)
    plan = ctx.plan(n, spl.PREC_F64, query_mode=spl.QUERY_EXPLICIT)
    qt = torch.from_numpy(xq).to(dev)
    ypp = torch.empty(n, dtype=torch.float64, device=dev)
    yq = torch.empty(n, dtype=torch.float64, device=dev)
    jq = torch.empty(n, dtype=torch.int32, device=dev)
    st, _ = ctx.wait(ctx.submit(plan, x, y, NAT, NAT, n, ypp, yq, jq, xq=qt), 120.0)
    assert st == 0
    jref = oracle.bracket_any(xh, xq)
    assert np.array_equal(jq.cpu().numpy().astype(np.int64), jref)
    yh = y.cpu().numpy()
    pick = rng.choice(n, size=4000, replace=False)
    ref = oracle.fit_eval(xh, yh, NAT, NAT, 0)
    yref = oracle.evaluate(xh, yh, ref["ypp"], xq[pick], jref[pick])
    e = yq_error(xh, yh, ref["ypp"], jref[pick], yq.cpu().numpy()[pick], yref)
    assert e <= TOL_F64


@pytest.mark.parametrize("n", [65535, 65536, 65537, 100003])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_explicit_coarse_key_table(ctx, n, precision):
    """Instances of 65,536 knots and more bisect explicit positions on a coarse table of every
    16th knot's key first, then within one 16-knot window: brackets must equal the oracle's on the
    hardest positions (every knot exactly, the binary64 neighbours on both sides of every knot,
    both ends and beyond), here and in a batch beside an instance without a table."""
    import torch
    from paper_2001_09253_gb300 import spl
    from parity_util import TOL_MIXED
    rng = np.random.default_rng(n)
    x, y = synth.curve(30, n)
    q = np.concatenate([x, np.nextafter(x, -np.inf), np.nextafter(x, np.inf), _queries(x, n // 4, rng)])
    rng.shuffle(q)
    prec = spl.PREC_F64 if precision == "f64" else spl.PREC_F32_REFINE
    tol = TOL_F64 if precision == "f64" else TOL_MIXED
    plan = ctx.plan(n, prec, query_mode=spl.QUERY_EXPLICIT)
    ref = oracle.fit_eval(x, y, NAT, NAT, 0)
    st, ypp, yq, jq = _run(ctx, plan, x, y, q)
    assert st == 0
    jref = oracle.bracket_any(x, q)
    assert np.array_equal(jq.astype(np.int64), jref)
    pick = rng.choice(len(q), size=5000, replace=False)
    yref = oracle.evaluate(x, y, ref["ypp"], q[pick], jref[pick])
    assert yq_error(x, y, ref["ypp"], jref[pick], yq[pick], yref) <= tol
    # the same positions in a batch beside a small instance (no table) with its own positions
    dev = torch.device("cuda", ctx.device)
    xs, ys = synth.curve(31, 1000)
    qs = _queries(xs, 3000, rng)
    big = [torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (x, y, q)]
    small = [torch.from_numpy(np.ascontiguousarray(v)).to(dev) for v in (xs, ys, qs)]
    outs = [(torch.full((len(v[2]),), np.nan, dtype=torch.float64, device=dev),
             torch.full((len(v[2]),), -7, dtype=torch.int32, device=dev)) for v in (small, big)]
    reqs = [spl.make_request(v[0], v[1], NAT, NAT, len(v[2]), None, o[0], o[1], xq=v[2])
            for v, o in zip((small, big), outs)]
    for t in ctx.submit_batch(plan, reqs, (big, small, outs)):
        st, _ = ctx.wait(t, 120.0)
        assert st == 0
    assert np.array_equal(outs[0][1].cpu().numpy().astype(np.int64), oracle.bracket_any(xs, qs))
    assert np.array_equal(outs[1][1].cpu().numpy().astype(np.int64), jref)


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("variant", [0, 1, 2])
def test_mixed_explicit_queries_and_stored_fit(ctx, refine, variant):
    """Binary32 plans: explicit unsorted queries after a binary32 fit (refined or not), and
    evaluation from a stored y'': brackets bit-exact, values within the mixed tolerance."""
    from paper_2001_09253_gb300 import spl
    from parity_util import TOL_MIXED
    rng = np.random.default_rng(30 + 3 * refine + variant)
    x, y = synth.curve(26, 6000)
    xq = _queries(x, 8000, rng)
    ref = oracle.fit_eval(x, y, NAT, NAT, 0)
    plan = ctx.plan(len(x), spl.PREC_F32_REFINE, refine_steps=refine, query_mode=spl.QUERY_EXPLICIT,
                    eval_variant=variant)
    st, ypp, yq, jq = _run(ctx, plan, x, y, xq)
    assert st == 0
    assert ypp_error(ypp, ref["ypp"]) <= (1e-8 if refine else TOL_MIXED)
    _check(x, y, ref["ypp"], xq, yq, jq, tol=TOL_MIXED)
    st, _, yq2, jq2 = _run(ctx, plan, x, y, xq, ypp_in=ypp, want_ypp=False)
    assert st == 0
    assert np.array_equal(yq2, yq) and np.array_equal(jq2, jq)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_uniform_grid_batch_from_stored_fits(ctx, precision):
    """Uniform grids evaluated from stored y'' for several instances in one launch: query counts
    that end inside a warp's run of queries (so runs cross from one instance into the next),
    an instance without queries, a single query, fewer and more queries than knots.  Brackets
    bit-exact against the oracle's monotone sweep, values within the plan's tolerance of the
    oracle's evaluation from the same y''."""
    import torch
    from paper_2001_09253_gb300 import spl
    from parity_util import TOL_MIXED
    dev = torch.device("cuda", ctx.device)
    prec = spl.PREC_F64 if precision == "f64" else spl.PREC_F32_REFINE
    tol = TOL_F64 if precision == "f64" else TOL_MIXED
    plan = ctx.plan(20000, prec)
    sizes = [(3, 1), (5, 300), (100, 0), (4097, 257), (777, 33), (64, 513), (20000, 5000), (1000, 2001)]
    reqs, keep, cases = [], [], []
    for i, (n, m) in enumerate(sizes):
        x, y = synth.curve(40, n, instance=i)
        yp1, ypn = (NAT, NAT) if i % 2 == 0 else (0.25 * i, -0.5)
        ref = oracle.fit_eval(x, y, yp1, ypn, m)
        xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
        pin = torch.from_numpy(np.ascontiguousarray(ref["ypp"])).to(dev)
        yq = torch.full((max(m, 1),), np.nan, dtype=torch.float64, device=dev)
        jq = torch.full((max(m, 1),), -7, dtype=torch.int32, device=dev)
        reqs.append(spl.make_request(xt, yt, yp1, ypn, m, None, yq if m else None, jq if m else None,
                                     ypp_in=pin))
        keep += [xt, yt, pin, yq, jq]
        cases.append((x, y, ref, yq, jq, m))
    launches0 = ctx.stats()["kernel_launches"]
    for t in ctx.submit_batch(plan, reqs, keep):
        st, _ = ctx.wait(t, 60.0)
        assert st == 0
    assert ctx.stats()["kernel_launches"] - launches0 == 1  # one evaluation launch, no fit
    for x, y, ref, yq, jq, m in cases:
        if not m:
            continue
        j = jq.cpu().numpy()[:m].astype(np.int64)
        assert np.array_equal(j, ref["jq"]), np.nonzero(j != ref["jq"])[0][:10]
        e = yq_error(x, y, ref["ypp"], ref["jq"], yq.cpu().numpy()[:m], ref["yq"])
        assert e <= tol, "S(x) error %.3e (n = %d, m = %d)" % (e, len(x), m)


@pytest.mark.parametrize("precision", [0, 1])
@pytest.mark.parametrize("mode", [0, 1])
def test_noop_control_brackets_only(ctx, precision, mode):
    """The paper's control loop (query generation and bracketing, no evaluation): brackets equal
    the oracle's, and the value written is the bracket's left knot; uniform and explicit queries,
    both precisions."""
    import torch
    from paper_2001_09253_gb300 import spl
    dev = torch.device("cuda", ctx.device)
    x, y = synth.curve(25, 3001)
    ref = oracle.fit_eval(x, y, NAT, NAT, 3001)
    xt, yt = torch.from_numpy(x).to(dev), torch.from_numpy(y).to(dev)
    ypp = torch.from_numpy(ref["ypp"]).to(dev)
    if mode == spl.QUERY_EXPLICIT:
        q = np.random.default_rng(3).uniform(x[0] - 1.0, x[-1] + 1.0, 4000)
        xq = torch.from_numpy(q).to(dev)
        jref = oracle.bracket_any(x, q)
    else:
        q, xq, jref = None, None, ref["jq"]
    m = len(jref)
    plan = ctx.plan(3001, precision, query_mode=mode, eval_variant=spl.EVAL_NOOP)
    yq = torch.full((m,), np.nan, dtype=torch.float64, device=dev)
    jq = torch.full((m,), -1, dtype=torch.int32, device=dev)
    st, _ = ctx.wait(ctx.submit(plan, xt, yt, NAT, NAT, m, None, yq, jq, xq=xq, ypp_in=ypp), 60.0)
    assert st == spl.OK
    j = jq.cpu().numpy().astype(np.int64)
    assert np.array_equal(j, jref)
    assert np.array_equal(yq.cpu().numpy(), x[jref])
