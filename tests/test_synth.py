"""The seeded input generator: reproducible, strictly increasing, exact prefix sums."""
from fractions import Fraction

import numpy as np

from paper_2001_09253_gb300 import synth


def test_splitmix64_reference_values():
    # SplitMix64 with state 0: the first outputs of the published generator
    # (state += 0x9E3779B97F4A7C15, then the mix) are these constants.
    out = synth.draws(np.uint64(0), 3)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_curve_shape_and_determinism():
    x, y = synth.curve(1, 100000)
    x2, y2 = synth.curve(1, 100000)
    assert np.array_equal(x, x2) and np.array_equal(y, y2)
    assert x[0] == 0.0
    assert np.all(np.diff(x) > 0)
    assert np.all(np.diff(x) <= 1.0)
    assert np.all((y >= 0) & (y < 1))
    # knots sit on the 2^-27 grid, so every partial sum is exact
    assert np.all(np.floor(x * 2 ** 27) == x * 2 ** 27)
    xs, _ = synth.curve(1, 1000)
    assert np.array_equal(xs, x[:1000])  # prefixes agree across sizes


def test_prefix_sums_exact():
    x, _ = synth.curve(3, 5000)
    r = synth.draws(synth.stream_key(3, 0, synth.STREAM_X), 4999)
    inc = [int(v >> np.uint64(37)) + 1 for v in r]
    acc = Fraction(0)
    for i, v in enumerate(inc):
        acc += Fraction(v, 2 ** 27)
        assert Fraction(x[i + 1]) == acc


def test_instances_and_streams_independent():
    a, _ = synth.curve(1, 100, instance=0)
    b, _ = synth.curve(1, 100, instance=1)
    assert not np.array_equal(a, b)


def test_loguniform_sizes_and_arrivals():
    s = synth.sizes_loguniform(2, 4096, 1e2, 1e5)
    assert s.min() >= 100 and s.max() <= 100000
    lg = np.log10(s)
    assert abs(lg.mean() - 3.5) < 0.05
    t = synth.poisson_arrivals(3, 20000.0, 200000)
    gaps = np.diff(t)
    assert abs(gaps.mean() - 5e-5) < 1e-6
    assert np.all(gaps > 0)
