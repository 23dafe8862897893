"""The runtime's launch-geometry rules through spl_launch_geometry, a pure function of the plan
options, the instance sizes and the SM count (no GPU): which kernel fits a submission, how it is
tiled, the invariants each kernel relies on, and which submissions launch their kernel alone."""
import numpy as np
import pytest

from paper_2001_09253_gb300 import spl

SMS = (152, 148, 8)
F32 = dict(precision=spl.PREC_F32_REFINE, refine_steps=1)


def geo(sizes, sms, **kw):
    return spl.launch_geometry(sizes, sms, **kw)


@pytest.mark.parametrize("sms", SMS)
def test_fp64_single_instance_on_the_cooperative_grid(sms):
    """One CTA up to 512 knots (pieces of up to 4 rows), 1-row pieces (128 rows per CTA) up to
    SMs x 128 knots, then the fewest rows per CTA that keep one CTA per SM, up to 9,600."""
    for n in (3, 4, 127, 128, 129, 300, 511, 512):
        g = geo([n], sms)
        assert g["fit_kernel"] == spl.KERNEL_MID_F64 and g["ctas"] == 1
        assert g["cta_rows"] == 128 * -(-n // 128)
    for n in (513, 1000, 128 * sms):
        g = geo([n], sms)
        assert g["cta_rows"] == 128 and g["ctas"] == -(-n // 128)
    rng = np.random.default_rng(5)
    edges = [128 * sms + 1, 4096 * sms, 4096 * sms + 1, 9600 * sms - 1, 9600 * sms]
    for n in [int(v) for v in rng.integers(513, 9600 * sms + 1, 400)] + edges:
        g = geo([n], sms)
        assert g["fit_kernel"] == spl.KERNEL_MID_F64 and g["direct"] and not g["separate_eval"]
        r, c = g["cta_rows"], g["ctas"]
        assert r % 128 == 0 and 128 <= r <= 9600
        assert 1 <= c <= sms and (c - 1) * r < n <= c * r
        assert r // 128 == max(1, -(-n // (128 * sms)))  # the shortest pieces that fit the SMs
    g = geo([9600 * sms + 1], sms)
    assert g["fit_kernel"] == spl.KERNEL_FUSED_F64 and g["cta_rows"] == 0 and not g["direct"]


def test_fp64_tiled_kernel_tile_length():
    """The tiled FP64 kernel: one instance of n = 1e7 on 152 SMs takes 151-row tiles (one group of
    32 tiles, 32 L - 104 rows, per warp of 14 per SM); an explicit tile length is kept; several
    instances take 128-row tiles; short tiles for the small instances that stay on this kernel."""
    g = geo([10_000_000], 152)
    assert g["fit_kernel"] == spl.KERNEL_FUSED_F64 and g["tile_rows"] == 151
    assert (32 * 151 - 104) * (152 * 14) >= 10_000_000 > (32 * 150 - 104) * (152 * 14)
    for n in (1000, 50_000, 2_000_000):
        assert geo([n], 152, tile_rows=64)["fit_kernel"] == spl.KERNEL_FUSED_F64
        assert geo([n], 152, tile_rows=64)["tile_rows"] == 64
    assert geo([5000, 7000], 152, tile_rows=0)["tile_rows"] == 128
    # explicit queries keep the fit on the tiled kernel, with the short-tile rule
    g = geo([1000], 152, query_mode=spl.QUERY_EXPLICIT)
    assert g["fit_kernel"] == spl.KERNEL_FUSED_F64 and g["separate_eval"] and g["tile_rows"] == 16
    assert geo([152 * 2000 + 1], 152, query_mode=spl.QUERY_EXPLICIT)["tile_rows"] == 32
    assert geo([152 * 8000 + 1], 152, query_mode=spl.QUERY_EXPLICIT)["tile_rows"] >= 128


@pytest.mark.parametrize("sms", SMS)
def test_fp64_batches_of_small_instances(sms):
    """Up to 4 x SMs instances of at most 4,096 knots: one CTA each; one more instance, or one
    larger instance, and the batch takes the tiled kernel."""
    assert geo([4096] * (4 * sms), sms)["fit_kernel"] == spl.KERNEL_SMALL_F64
    assert geo([3, 4096], sms)["fit_kernel"] == spl.KERNEL_SMALL_F64
    assert geo([100] * (4 * sms + 1), sms)["fit_kernel"] == spl.KERNEL_FUSED_F64
    assert geo([100, 4097], sms)["fit_kernel"] == spl.KERNEL_FUSED_F64
    assert not geo([100, 200], sms)["direct"]


@pytest.mark.parametrize("sms", SMS)
def test_binary32_tile_length(sms):
    """The warp-cooperative kernel: 32-row tiles for one instance of at most 32 rows per resident
    warp (20 per SM); beyond, about two tiles per warp within [128, 544] rows, a multiple of 32;
    544 rows for several instances; an explicit length rounded up to 32 and capped at 544."""
    cap = 32 * 20 * sms
    for n in (3, 100, 1000, cap):
        g = geo([n], sms, **F32)
        assert g["fit_kernel"] == spl.KERNEL_SCAN_MIXED and g["tile_rows"] == 32 and g["direct"]
    rng = np.random.default_rng(7)
    for n in [cap + 1] + [int(v) for v in rng.integers(cap + 1, 10**8, 200)]:
        L = geo([n], sms, max_n=10**8, **F32)["tile_rows"]
        assert L % 32 == 0 and 128 <= L <= 544
        assert L == min(max(-(-(-(-n // (2 * 20 * sms))) // 32) * 32, 128), 544)
    assert geo([1000, 2000], sms, **F32)["tile_rows"] == 544
    assert geo([5000], sms, tile_rows=40, **F32)["tile_rows"] == 64
    assert geo([5000], sms, tile_rows=4000, **F32)["tile_rows"] == 544


def test_direct_launch_only_for_single_device_fit_and_evaluate():
    """A submission is launched as its kernel alone only for one instance in device memory, fitted
    and evaluated on the uniform grid by the multi-CTA FP64 kernel or the binary32 kernel."""
    assert geo([5000], 152)["direct"]
    assert geo([5000], 152, **F32)["direct"]
    assert not geo([5000], 152, mem=spl.MEM_HOST)["direct"]
    assert not geo([5000], 152, mem=spl.MEM_HOST, **F32)["direct"]
    assert not geo([5000], 152, query_mode=spl.QUERY_EXPLICIT)["direct"]
    assert not geo([5000], 152, query_mode=spl.QUERY_EXPLICIT, **F32)["direct"]
    g = geo([5000], 152, stored_fit=True)
    assert g["fit_kernel"] == spl.KERNEL_NONE and g["separate_eval"] and not g["direct"]
    assert not geo([5000], 152, tile_rows=64)["direct"]  # an explicit FP64 tile length: tiled kernel
    assert geo([5000], 152, tile_rows=64, **F32)["direct"]
    assert not geo([5000, 5000], 152, **F32)["direct"]


def test_invalid_arguments_rejected():
    with pytest.raises(spl.SplError):
        geo([], 152)
    with pytest.raises(spl.SplError):
        geo([2], 152)
    with pytest.raises(spl.SplError):
        geo([1000], 0)
    with pytest.raises(spl.SplError):
        geo([1000], 152, max_n=999)
    with pytest.raises(spl.SplError):
        geo([1000], 152, precision=7)
    with pytest.raises(spl.SplError):
        geo([1000], 152, refine_steps=1)  # FP64 takes no refinement step
    with pytest.raises(spl.SplError):
        geo([1000], 152, mem=5)
    with pytest.raises(spl.SplError):
        geo([1000], 152, tile_rows=8)
