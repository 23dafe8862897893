"""GPU tests of the continuous-batching server (spl_serve_*): results equal a single-instance
submission bit for bit, alone and in the mix; admission under a small budget; relaunch of the
device loop after it went idle; per-request error isolation; trace replay; failure detection
through the loop's bounded waits."""
import time

import numpy as np
import pytest

import oracle
from paper_2001_09253_gb300 import spl, synth
from parity_util import TOL_MIXED, yq_error, ypp_error

pytestmark = pytest.mark.gpu

NAT = spl.NATURAL
TILE = 256


@pytest.fixture(scope="module")
def ctx():
    c = spl.Context(device=0, arena_bytes=2 << 30, max_slots=4096)
    yield c
    c.close()


def _pool(count, seed, lo=1e2, hi=2e5):
    import torch
    sizes = synth.sizes_loguniform(seed, count, lo, hi)
    pool = []
    for i, n in enumerate(sizes):
        n = int(max(n, 3))
        x, y = synth.curve(seed, n, instance=i)
        m = n + (i * 13) % 97
        bc = (NAT, NAT) if i % 3 else (-1.0, 0.5)
        pool.append(dict(x=x, y=y, n=n, m=m, bc=bc, xt=torch.from_numpy(x).cuda(), yt=torch.from_numpy(y).cuda()))
    return pool


def _outputs(p):
    import torch
    return (torch.full((p["n"],), np.nan, dtype=torch.float64, device="cuda"),
            torch.full((p["m"],), np.nan, dtype=torch.float64, device="cuda"))


def _reference(ctx, p, tile=TILE):
    """The same request served alone: a fresh server with nothing else in flight."""
    srv = spl.Server(ctx, max_inflight=1, tile_rows=tile, idle_timeout_ms=20)
    ypp, yq = _outputs(p)
    s, _ = srv.wait(srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], ypp, yq))
    srv.close()
    assert s == spl.OK
    return ypp.cpu().numpy(), yq.cpu().numpy()


@pytest.mark.parametrize("tile", [TILE, 0])  # 0: tile length chosen per request
def test_alone_and_in_the_mix_are_identical(ctx, tile):
    import torch
    pool = _pool(48, 5)
    refs = [_reference(ctx, p, tile) for p in pool]
    srv = spl.Server(ctx, max_inflight=64, tile_rows=tile, budget_bytes=1 << 34)
    # alone: one request at a time
    for p, ref in zip(pool, refs):
        ypp, yq = _outputs(p)
        t = srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], ypp, yq)
        s, _ = srv.wait(t)
        assert s == spl.OK
        assert np.array_equal(ypp.cpu().numpy(), ref[0]) and np.array_equal(yq.cpu().numpy(), ref[1])
    # in the mix: all in flight together
    outs, tickets = [], []
    for p in pool:
        o = _outputs(p)
        outs.append(o)
        tickets.append(srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1]))
    for t in tickets:
        s, _ = srv.wait(t)
        assert s == spl.OK
    torch.cuda.synchronize()
    for o, ref, p in zip(outs, refs, pool):
        assert np.array_equal(o[0].cpu().numpy(), ref[0]) and np.array_equal(o[1].cpu().numpy(), ref[1])
    # and both agree with the oracle at the mixed tolerance
    for o, p in list(zip(outs, pool))[:8]:
        r = oracle.fit_eval(p["x"], p["y"], p["bc"][0], p["bc"][1], p["m"])
        assert ypp_error(o[0].cpu().numpy(), r["ypp"]) <= TOL_MIXED
        assert yq_error(p["x"], p["y"], r["ypp"], r["jq"], o[1].cpu().numpy(), r["yq"]) <= TOL_MIXED
    srv.close()


def test_admission_under_a_small_budget(ctx):
    import torch
    # requests long enough (1e6..2e6 points) and submitted back to back (outputs made ready
    # beforehand) so that later ones arrive while the budget is held by earlier ones
    pool = _pool(16, 6, lo=1e6, hi=2e6)
    biggest = max(16 * p["n"] + 8 * p["n"] + 8 * p["m"] for p in pool)
    srv = spl.Server(ctx, max_inflight=64, tile_rows=TILE, budget_bytes=2 * biggest)
    outs = [_outputs(p) for p in pool]
    torch.cuda.synchronize()
    tickets = []
    waited = 0
    for p, o in zip(pool, outs):
        tickets.append(srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1], sync=False))
        waited = max(waited, srv.stats()["waiting"])
    assert waited > 0  # some requests had to wait for memory
    for t in tickets:
        s, _ = srv.wait(t)
        assert s == spl.OK
    for o, p in zip(outs, pool):
        ref = _reference(ctx, p)
        assert np.array_equal(o[1].cpu().numpy(), ref[1])
    # a request larger than the whole budget is refused
    big = pool[0]
    with pytest.raises(spl.SplError) as e:
        srv2 = spl.Server(ctx, max_inflight=4, budget_bytes=1000)
        try:
            srv2.submit(big["xt"], big["yt"], NAT, NAT, big["m"], *_outputs(big))
        finally:
            srv2.close()
    assert e.value.status == spl.ERR_BUDGET
    srv.close()


def test_loop_relaunches_after_idle(ctx):
    pool = _pool(4, 7, lo=1e3, hi=1e4)
    srv = spl.Server(ctx, max_inflight=8, tile_rows=TILE, idle_timeout_ms=20)
    for p in pool[:2]:
        o = _outputs(p)
        s, _ = srv.wait(srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1]))
        assert s == spl.OK
    time.sleep(0.2)  # the device loop leaves after 20 ms without work
    for p in pool[2:]:
        o = _outputs(p)
        s, _ = srv.wait(srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1]))
        assert s == spl.OK
        assert np.array_equal(o[1].cpu().numpy(), _reference(ctx, p)[1])
    assert srv.stats()["loop_launches"] >= 2
    srv.close()


def test_worker_wait_runs_out_and_the_context_stays_usable(ctx):
    """Failure detection without a GPU fault: the scheduler warp is told to leave at once
    (fault_flags bit 0), so nothing publishes work and the workers' bounded waits run out one
    second after the loop's 100 ms deadline; the host reads the loop's error flag and completes
    the request with SPL_ERR_TIMEOUT.  The context stays usable: a normal server on it then
    finishes its requests with the expected results."""
    pool = _pool(3, 8, lo=1e3, hi=1e4)
    bad = spl.Server(ctx, max_inflight=4, tile_rows=TILE, idle_timeout_ms=20, deadline_ms=100, fault_flags=1)
    p = pool[0]
    o = _outputs(p)
    t = bad.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1])
    s, _ = bad.poll(t)
    assert s == spl.PENDING
    t0 = time.time()
    while s == spl.PENDING and time.time() - t0 < 20.0:
        time.sleep(0.05)
        s, _ = bad.poll(t)
    assert s == spl.ERR_TIMEOUT  # completed by the failure path, not by a host-side wait limit
    assert 0.5 < time.time() - t0 < 10.0
    bad.close()
    good = spl.Server(ctx, max_inflight=4, tile_rows=TILE, idle_timeout_ms=20)
    for p in pool:
        o = _outputs(p)
        s, _ = good.wait(good.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1]))
        assert s == spl.OK
        ref = _reference(ctx, p)
        assert np.array_equal(o[1].cpu().numpy(), ref[1]) and np.array_equal(o[0].cpu().numpy(), ref[0])
    good.close()


def test_bad_request_is_isolated(ctx):
    import torch
    pool = _pool(6, 8, lo=1e3, hi=1e4)
    bad = dict(pool[2])
    y = bad["y"].copy()
    y[5] = np.nan
    bad["yt"] = torch.from_numpy(y).cuda()
    srv = spl.Server(ctx, max_inflight=16, tile_rows=TILE)
    items = pool[:2] + [bad] + pool[3:]
    outs = [_outputs(p) for p in items]
    tickets = [srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1]) for p, o in zip(items, outs)]
    for i, t in enumerate(tickets):
        s, _ = srv.wait(t)
        assert s == (spl.ERR_NONFINITE if i == 2 else spl.OK)
    # host arrays are refused at submission (the loop reads device memory only)
    p, o = pool[0], outs[0]
    with pytest.raises(spl.SplError) as ei:
        srv.submit(torch.from_numpy(p["x"]), torch.from_numpy(p["y"]), p["bc"][0], p["bc"][1], p["m"], o[0], o[1])
    assert ei.value.status == spl.ERR_INVALID_ARG
    srv.close()


def test_trace_replay(ctx):
    pool = _pool(64, 9, lo=1e2, hi=1e5)
    reqs, keep = [], []
    for p in pool:
        o = _outputs(p)
        keep.append(o)
        reqs.append(spl.make_request(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1]))
    srv = spl.Server(ctx, max_inflight=256, tile_rows=TILE)
    count = 2000
    arrivals = synth.poisson_arrivals(3, 20000.0, count)
    pick = np.arange(count) % len(pool)
    s, lat, makespan = srv.replay(reqs, pick, arrivals)
    assert s == spl.OK
    assert np.all(lat > 0) and np.all(np.isfinite(lat))
    assert makespan >= arrivals[-1]
    srv.close()


@pytest.mark.parametrize("tile", [TILE, 0])
def test_refined_serving_alone_and_in_the_mix(ctx, tile):
    """Served with one refinement step (two passes over each request's tiles, the second once
    the first is complete): y'' within the refined tolerance of the oracle, S(x_k) within the
    mixed one, and each result the same alone and in the mix, bit for bit."""
    import torch
    pool = _pool(24, 9)
    refs = []
    for p in pool:  # alone: a server with nothing else in flight
        srv = spl.Server(ctx, max_inflight=1, tile_rows=tile, idle_timeout_ms=20, refine_steps=1)
        ypp, yq = _outputs(p)
        s, _ = srv.wait(srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], ypp, yq))
        srv.close()
        assert s == spl.OK
        refs.append((ypp.cpu().numpy(), yq.cpu().numpy()))
    srv = spl.Server(ctx, max_inflight=64, tile_rows=tile, budget_bytes=1 << 34, refine_steps=1)
    outs, tickets = [], []
    for p in pool:
        o = _outputs(p)
        outs.append(o)
        tickets.append(srv.submit(p["xt"], p["yt"], p["bc"][0], p["bc"][1], p["m"], o[0], o[1]))
    for t in tickets:
        s, _ = srv.wait(t)
        assert s == spl.OK
    torch.cuda.synchronize()
    srv.close()
    for o, ref in zip(outs, refs):
        assert np.array_equal(o[0].cpu().numpy(), ref[0]) and np.array_equal(o[1].cpu().numpy(), ref[1])
    for o, p in zip(outs, pool):
        r = oracle.fit_eval(p["x"], p["y"], p["bc"][0], p["bc"][1], p["m"])
        assert ypp_error(o[0].cpu().numpy(), r["ypp"]) <= 1e-8
        assert yq_error(p["x"], p["y"], r["ypp"], r["jq"], o[1].cpu().numpy(), r["yq"]) <= TOL_MIXED


def test_refined_serving_rejects_bad_option(ctx):
    with pytest.raises(spl.SplError) as ei:
        spl.Server(ctx, max_inflight=4, refine_steps=2)
    assert ei.value.status == spl.ERR_INVALID_ARG
