"""GPU parity of the two tile decompositions of long instances.

FP64 kernel, grouped and chained tiles: every lane but the first of a warp group starts from
the exact c' and a corrected d', every lane but the last takes its back-substitution start from
the next lane's rows.  Group size for the forced tile length L = 200: 32 L - 48 - 56 = 6296
rows; the size below gives 7 groups, the last one ragged, with padding under the 1/8 the runtime
allows, so the grouped geometry is used.

Binary32 warp-cooperative kernel: a warp solves one tile 32 rows at a time (warp scans for the
recurrences, lane-parallel queries); tiles of L rows (a multiple of 32) start their forward sweep
64 rows early and their back substitution 32 rows past their end.  The sizes below give many
tiles with a ragged last tile and ragged last chunk."""
import numpy as np
import pytest

import oracle
from paper_2001_09253_gb300 import spl, synth
from parity_util import TOL_F64, TOL_MIXED, check_instance, run_gpu, ypp_error, yq_error

pytestmark = pytest.mark.gpu

NAT = spl.NATURAL
N64, L64 = 6296 * 7 - 1000, 200
N32, L32 = 256 * 37 + 19, 256


@pytest.fixture(scope="module")
def ctx():
    c = spl.Context(device=0, arena_bytes=2 << 30, max_slots=64)
    yield c
    c.close()


def test_group_sizes_are_grouped():
    """The FP64 size above meets the runtime's grouping rule (32-tile groups, padding <= 1/8)."""
    plain = -(-N64 // L64)
    groups = -(-N64 // (32 * L64 - 48 - 56))
    assert plain >= 32 and 8 * 32 * groups <= 9 * plain and groups >= 5


@pytest.mark.parametrize("bc", [(NAT, NAT), (-1.0, 1.0), (NAT, 0.25)])
def test_fp64_grouped_chained(ctx, bc):
    x, y = synth.curve(71, N64)
    plan = ctx.plan(N64, spl.PREC_F64, tile_rows=L64)
    for m in (N64, 3 * N64 + 7, 1001):
        check_instance(ctx, plan, x, y, bc[0], bc[1], m)


def test_fp64_grouped_adversarial(ctx):
    for seed in (1, 2):
        x, y = synth.curve_adversarial(seed, N64, decades=8)
        plan = ctx.plan(N64, spl.PREC_F64, tile_rows=L64)
        check_instance(ctx, plan, x, y, NAT, NAT, N64 + 5)
        check_instance(ctx, plan, x, y, 0.5, -2.0, N64 // 3)


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("bc", [(NAT, NAT), (-1.0, 1.0), (NAT, 0.25)])
def test_mixed_warp_tiles(ctx, refine, bc):
    x, y = synth.curve(72, N32)
    plan = ctx.plan(N32, spl.PREC_F32_REFINE, refine_steps=refine, tile_rows=L32)
    for m in (N32, 2 * N32 + 3, 77, 2):
        check_instance(ctx, plan, x, y, bc[0], bc[1], m, tol=TOL_MIXED)


@pytest.mark.parametrize("refine", [0, 1])
def test_mixed_warp_tiles_adversarial(ctx, refine):
    x, y = synth.curve_adversarial(3, N32, decades=6)
    plan = ctx.plan(N32, spl.PREC_F32_REFINE, refine_steps=refine, tile_rows=L32)
    ref = oracle.fit_eval(x, y, NAT, NAT, N32)
    st, ypp, yq, jq = run_gpu(ctx, plan, x, y, NAT, NAT, N32)
    assert st == 0
    assert np.array_equal(jq.astype(np.int64), ref["jq"])
    assert ypp_error(ypp, ref["ypp"]) <= TOL_MIXED
    assert yq_error(x, y, ref["ypp"], ref["jq"], yq, ref["yq"]) <= TOL_MIXED
    if refine:  # the refinement brings y'' to FP64 accuracy
        assert ypp_error(ypp, ref["ypp"]) <= 1e-8


@pytest.mark.parametrize("precision,n,L,row", [(spl.PREC_F64, N64, L64, 2 * (32 * L64 - 104) + 5 * L64 - 56 + L64 // 2),
                                               (spl.PREC_F32_REFINE, N32, L32, 5 * L32 + 77)])
def test_errors_inside_a_tile(ctx, precision, n, L, row):
    """Input errors in the middle of a tile (FP64: group 2, lane 5; binary32: tile 5) are reported."""
    x, y = synth.curve(73, n)
    plan = ctx.plan(n, precision, tile_rows=L)
    bad_y = y.copy()
    bad_y[row] = np.nan
    st, _, _, _ = run_gpu(ctx, plan, x, bad_y, NAT, NAT, n)
    assert st == spl.ERR_NONFINITE
    bad_x = x.copy()
    bad_x[row] = bad_x[row - 1]
    st, _, _, _ = run_gpu(ctx, plan, bad_x, y, NAT, NAT, n)
    assert st == spl.ERR_NOT_INCREASING


def test_fp64_group_boundaries_sweep(ctx):
    """Sizes around whole FP64 groups (exactly k groups, one row more or less, a lone row past a
    group, the last lane's tile cut short), seeded, both end conditions."""
    L = 128
    G = 32 * L - 104
    sizes = sorted({k * G + d for k in (1, 2, 3) for d in (-1, 0, 1, 2, 17, -L + 1, L - 1)})
    plan = ctx.plan(4 * G, spl.PREC_F64, tile_rows=L)
    for i, n in enumerate(sizes):
        x, y = synth.curve(80 + i, n)
        bc = (NAT, NAT) if i % 2 else (0.75, -1.25)
        check_instance(ctx, plan, x, y, bc[0], bc[1], n + (i % 3), tol=TOL_F64)


@pytest.mark.parametrize("refine", [0, 1])
def test_mixed_tile_boundaries_sweep(ctx, refine):
    """Sizes around whole binary32 tiles and chunks (k tiles exactly, one row more or less, a lone
    row or chunk past a tile, a tile one row short of its last chunk), seeded, both end
    conditions."""
    L = 96
    sizes = sorted({k * L + d for k in (12, 13, 33) for d in (-1, 0, 1, 2, 17, 31, 32, 33, -L + 1, L - 1)})
    plan = ctx.plan(34 * L, spl.PREC_F32_REFINE, refine_steps=refine, tile_rows=L)
    for i, n in enumerate(sizes):
        x, y = synth.curve(90 + i, n)
        bc = (NAT, NAT) if i % 2 else (0.75, -1.25)
        check_instance(ctx, plan, x, y, bc[0], bc[1], n + (i % 3), tol=TOL_MIXED)


@pytest.mark.parametrize("refine", [0, 1])
@pytest.mark.parametrize("n", [1024, 1057, 1311])
def test_mixed_warp_tiles_query_counts(ctx, refine, n):
    """The warp-cooperative kernel (instances of 1,024 rows or more) with few and many queries:
    none, one (the grid's single point x_0), two, three, a third of n, more than twice n; both
    end conditions, tiles of 96 rows."""
    x, y = synth.curve(3000 + n, n)
    plan = ctx.plan(n, spl.PREC_F32_REFINE, refine_steps=refine, tile_rows=96)
    for m in sorted({0, 1, 2, 3, n // 3, 2 * n + 1}):
        check_instance(ctx, plan, x, y, -1.0, 1.0, m, tol=TOL_MIXED)
        check_instance(ctx, plan, x, y, NAT, NAT, m, tol=TOL_MIXED)
