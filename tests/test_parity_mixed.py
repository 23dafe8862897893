"""GPU parity of the mixed-precision path (binary32 solve and cubic, exact binary64
differences and query positions) against the FP64 oracle, through the C ABI.
Tolerance 1e-5 (normwise for y'', per query for S(x_k)); bracket indices bit-exact."""
import numpy as np
import pytest

import oracle
from paper_2001_09253_gb300 import spl, synth
from parity_util import TOL_MIXED, check_instance, run_gpu, ypp_error, yq_error

pytestmark = pytest.mark.gpu

NAT = oracle.NATURAL


@pytest.fixture(scope="module")
def ctx():
    c = spl.Context(device=0, arena_bytes=2 << 30, max_slots=8192)
    yield c
    c.close()


def _plan(ctx, tile_rows=0, refine=0, max_n=1 << 26):
    return ctx.plan(max_n=max_n, precision=spl.PREC_F32_REFINE, refine_steps=refine, tile_rows=tile_rows)


@pytest.mark.parametrize("bc", [(NAT, NAT), (-1.0, 1.0), (0.0, 0.0), (NAT, 2.0)])
def test_smallest_config_n1000(ctx, bc):
    x, y = synth.curve(0, 1000)
    for L in (0, 16, 37, 150):
        check_instance(ctx, _plan(ctx, L), x, y, bc[0], bc[1], 1000, tol=TOL_MIXED)


@pytest.mark.parametrize("n", [3, 4, 5, 9, 31, 32, 33, 40, 64, 65, 129, 257])
@pytest.mark.parametrize("L", [16, 40])
def test_sizes_and_tiles(ctx, n, L):
    x, y = synth.curve(2000 + n, n)
    for m in sorted({0, 1, 2, 3, n, 2 * n + 1, max(2, n // 3)}):
        check_instance(ctx, _plan(ctx, L), x, y, -1.0, 1.0, m, tol=TOL_MIXED)
        check_instance(ctx, _plan(ctx, L), x, y, NAT, NAT, m, tol=TOL_MIXED)


def test_knots_far_from_zero_with_tiny_gaps(ctx):
    """Knots near 5e6 with gaps down to 2^-27: binary32 cannot hold the knots, the exact
    integer differences must carry the gaps."""
    x, y = synth.curve(11, 20000)
    x = x + 5.0e6
    check_instance(ctx, _plan(ctx), x, y, NAT, NAT, 20000, tol=TOL_MIXED)
    check_instance(ctx, _plan(ctx, 100), x, y, -1.0, 1.0, 33333, tol=TOL_MIXED)


@pytest.mark.parametrize("seed", [1, 2])
def test_adversarial_gap_ratios(ctx, seed):
    x, y = synth.curve_adversarial(seed, 5000, decades=6)
    for L in (16, 300, 0):
        check_instance(ctx, _plan(ctx, L), x, y, NAT, NAT, 7001, tol=TOL_MIXED)


def test_negative_and_mixed_sign_knots(ctx):
    x, y = synth.curve(12, 3000)
    x = x - x[1500]
    check_instance(ctx, _plan(ctx, 64), x, y, NAT, NAT, 4000, tol=TOL_MIXED)
    check_instance(ctx, _plan(ctx, 64), x, 1000.0 + y, 0.25, -0.25, 4000, tol=TOL_MIXED)


def test_validation_errors_reported(ctx):
    x, y = synth.curve(6, 3000)
    p = _plan(ctx, 64)
    bad = x.copy()
    bad[1700] = bad[1699]
    st, *_ = run_gpu(ctx, p, bad, y, NAT, NAT, 100)
    assert st == spl.ERR_NOT_INCREASING
    bad = y.copy()
    bad[5] = np.nan
    st, *_ = run_gpu(ctx, p, x, bad, NAT, NAT, 100)
    assert st == spl.ERR_NONFINITE


@pytest.mark.parametrize("bc", [(NAT, NAT), (-1.0, 1.0), (NAT, 0.5)])
def test_refinement_step(ctx, bc):
    """One refinement step against the double-float residual: parity at the mixed tolerance
    and a y'' error well below the unrefined one."""
    x, y = synth.curve(21, 50000)
    ref = oracle.fit_eval(x, y, bc[0], bc[1], 50000)
    errs = {}
    for refine in (0, 1):
        for L in (16, 0):
            st, ypp, yq, jq = run_gpu(ctx, _plan(ctx, L, refine), x, y, bc[0], bc[1], 50000)
            assert st == 0
            assert np.array_equal(jq.astype(np.int64), ref["jq"])
            e1 = ypp_error(ypp, ref["ypp"])
            e2 = yq_error(x, y, ref["ypp"], ref["jq"], yq, ref["yq"])
            assert e1 <= TOL_MIXED and e2 <= TOL_MIXED
            errs[(refine, L)] = e1
    assert errs[(1, 0)] < 0.1 * errs[(0, 0)], errs
    assert errs[(1, 16)] < 0.1 * errs[(0, 16)], errs
    assert errs[(1, 0)] < 1e-9, errs


def test_refinement_rescues_ill_conditioned_smooth_data(ctx):
    """Geometric gaps with smooth data: the binary32 slopes cancel in d_j; the refined path
    recovers the tolerance from the double-float residual."""
    g = np.concatenate([0.7 ** np.arange(40), 0.7 ** np.arange(40)[::-1]] * 25)
    x = np.concatenate([[1.0], 1.0 + np.cumsum(g)])
    y = np.sin(3 * x)
    ref = oracle.fit_eval(x, y, NAT, NAT, 3 * len(x))
    st, ypp, yq, jq = run_gpu(ctx, _plan(ctx, 0, 1), x, y, NAT, NAT, 3 * len(x))
    assert st == 0
    assert ypp_error(ypp, ref["ypp"]) <= TOL_MIXED
    assert yq_error(x, y, ref["ypp"], ref["jq"], yq, ref["yq"]) <= TOL_MIXED


def test_refined_batch(ctx):
    import torch
    plan = _plan(ctx, 0, 1)
    sizes = [3, 17, 1000, 5000, 64, 129]
    reqs, keep, refs = [], [], []
    for i, n in enumerate(sizes):
        x, y = synth.curve(31, n, instance=i)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ypp = torch.empty(n, dtype=torch.float64, device="cuda")
        yq = torch.empty(2 * n, dtype=torch.float64, device="cuda")
        bc = (NAT, NAT) if i % 2 else (-1.0, 2.0)
        reqs.append(spl.make_request(xt, yt, bc[0], bc[1], 2 * n, ypp, yq))
        keep.append((xt, yt, ypp, yq))
        refs.append((x, y, bc))
    for t, (x, y, bc), k in zip(ctx.submit_batch(plan, reqs, keep), refs, keep):
        st, _ = ctx.wait(t)
        assert st == 0
        ref = oracle.fit_eval(x, y, bc[0], bc[1], 2 * len(x))
        assert ypp_error(k[2].cpu().numpy(), ref["ypp"]) <= 1e-8
        assert yq_error(x, y, ref["ypp"], ref["jq"], k[3].cpu().numpy(), ref["yq"]) <= TOL_MIXED


def test_consecutive_single_requests_reuse_the_tile_counter(ctx):
    """A single request in device memory launches the binary32 kernel(s) with a tile counter that
    no memset clears: the kernel's last tile claim leaves it at zero for the next launch.  Requests
    whose tile counts change from one launch to the next, with and without the refinement step,
    all equal the oracle (a counter left non-zero would skip tiles, leaving the NaN fill)."""
    for i, n in enumerate([100_000, 1_000, 1_000_000, 3, 50_000, 129, 300_001]):
        x, y = synth.curve(950 + i, n)
        check_instance(ctx, _plan(ctx, refine=i % 2), x, y, NAT, NAT, n, tol=TOL_MIXED)
        check_instance(ctx, _plan(ctx, refine=1 - i % 2), x, y, -1.0, 1.0, n // 3 + 1, tol=TOL_MIXED)


@pytest.mark.parametrize("refine", [0, 1])
def test_small_instance_batch(ctx, refine):
    """A batch of mostly small instances (sizes 3..1000, one or two tiles each, a warp per tile):
    clamped and natural ends, against the oracle."""
    import torch
    plan = _plan(ctx, 0, refine)
    rng = np.random.default_rng(40 + refine)
    sizes = [3, 4, 5, 16, 17, 31, 33, 64, 127, 128, 129, 500, 999, 1000] + list(rng.integers(3, 1000, 50))
    reqs, keep, refs = [], [], []
    for i, n in enumerate(sizes):
        n = int(n)
        x, y = synth.curve(41, n, instance=i)
        xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        ypp = torch.full((n,), np.nan, dtype=torch.float64, device="cuda")
        m = n + i % 3
        yq = torch.full((m,), np.nan, dtype=torch.float64, device="cuda")
        jq = torch.full((m,), -7, dtype=torch.int32, device="cuda")
        bc = [(NAT, NAT), (-1.0, 2.0), (NAT, 0.5)][i % 3]
        reqs.append(spl.make_request(xt, yt, bc[0], bc[1], m, ypp, yq, jq))
        keep.append((xt, yt, ypp, yq, jq))
        refs.append((x, y, bc, m))
    for t, (x, y, bc, m), k in zip(ctx.submit_batch(plan, reqs, keep), refs, keep):
        st, _ = ctx.wait(t)
        assert st == 0
        ref = oracle.fit_eval(x, y, bc[0], bc[1], m)
        assert np.array_equal(k[4].cpu().numpy().astype(np.int64), ref["jq"])
        assert ypp_error(k[2].cpu().numpy(), ref["ypp"]) <= (1e-8 if refine else TOL_MIXED)
        assert yq_error(x, y, ref["ypp"], ref["jq"], k[3].cpu().numpy(), ref["yq"]) <= TOL_MIXED


@pytest.mark.parametrize("refine", [0, 1])
def test_full_size_n1e7(ctx, refine):
    """n = M = 10^7, seed 1, in the benchmark's launch configurations (no refinement, one
    refinement step); all outputs compared."""
    import torch
    n = 10_000_000
    x, y = spl.generate_curve(1, n)
    hx, hy = synth.curve(1, n)
    ypp = torch.empty(n, dtype=torch.float64, device="cuda")
    yq = torch.empty(n, dtype=torch.float64, device="cuda")
    jq = torch.empty(n, dtype=torch.int32, device="cuda")
    t = ctx.submit(_plan(ctx, refine=refine), x, y, NAT, NAT, n, ypp, yq, jq)
    st, _ = ctx.wait(t, 300)
    assert st == 0
    ref = oracle.fit_eval(hx, hy, NAT, NAT, n)
    e1 = ypp_error(ypp.cpu().numpy(), ref["ypp"])
    assert np.array_equal(jq.cpu().numpy().astype(np.int64), ref["jq"])
    e2 = yq_error(hx, hy, ref["ypp"], ref["jq"], yq.cpu().numpy(), ref["yq"])
    print("mixed n=1e7, %d refinement steps: y'' err %.3e  S err %.3e" % (refine, e1, e2))
    assert e1 <= (1e-8 if refine else TOL_MIXED) and e2 <= TOL_MIXED


def test_batched_workload_4096(ctx):
    """The batched workload in the benchmark's launch configuration: 4,096 instances with n
    log-uniform in [1e2, 1e5] (seed 2, instance i its own curve), natural ends, M = n, binary32
    + one refinement step, one reusable batch replayed from a CUDA graph.  Every status OK; all
    outputs of 64 sampled instances (and the largest and smallest) compared with the oracle."""
    import torch
    count = 4096
    sizes = synth.sizes_loguniform(2, count, 1e2, 1e5)
    total = int(sizes.sum())
    off = np.concatenate([[0], np.cumsum(sizes)])
    X, Y, P, Q = (torch.empty(total, dtype=torch.float64, device="cuda") for _ in range(4))
    for i, nn in enumerate(sizes):
        xi, yi = spl.generate_curve(2, int(nn), instance=i)
        X[off[i]:off[i + 1]].copy_(xi)
        Y[off[i]:off[i + 1]].copy_(yi)
    torch.cuda.synchronize()
    plan = _plan(ctx, refine=1, max_n=int(sizes.max()))
    reqs = [spl.make_request(X[off[i]:off[i + 1]], Y[off[i]:off[i + 1]], NAT, NAT, int(nn),
                             P[off[i]:off[i + 1]], Q[off[i]:off[i + 1]]) for i, nn in enumerate(sizes)]
    b = ctx.batch(plan, reqs, keep=(X, Y, P, Q))
    first = None
    for _ in range(2):  # the second replay gives the same outputs, bit for bit
        P.fill_(np.nan)
        Q.fill_(np.nan)
        torch.cuda.synchronize()
        b.launch()
        assert (b.wait() == 0).all()
        if first is None:
            first = (P.clone(), Q.clone())
    b.close()
    assert torch.equal(first[0], P) and torch.equal(first[1], Q)
    rng = np.random.default_rng(11)
    pick = set(rng.choice(count, 64, replace=False).tolist()) | {int(np.argmax(sizes)), int(np.argmin(sizes))}
    for i in sorted(pick):
        x, y = synth.curve(2, int(sizes[i]), instance=i)
        ref = oracle.fit_eval(x, y, NAT, NAT, len(x))
        ypp = P[off[i]:off[i + 1]].cpu().numpy()
        yq = Q[off[i]:off[i + 1]].cpu().numpy()
        assert ypp_error(ypp, ref["ypp"]) <= 1e-8, i
        assert yq_error(x, y, ref["ypp"], ref["jq"], yq, ref["yq"]) <= TOL_MIXED, i
