"""Seeded synthetic inputs shaped like the benchmark workload of arXiv 2001.09253.

This module holds no arithmetic of the spline method: it only draws knots,
values, instance sizes and arrival times.  Tests feed its arrays to both the
CPU oracle and the CUDA path; the CUDA library carries a bit-identical device
copy of ``curve`` (same counter-based generator, same integer prefix sum) for
workloads too large to generate on the host.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-style: draw i of a stream with
key k is mix64(k + (i + 1) * 0x9E3779B97F4A7C15).

Curve recipe (section "Curve Interpolation", benchmark steps 5-6), with the
readings of this implementation:
  * x_0 = 0 and x_i = x_{i-1} + eps_i.  eps_i is uniform on the dyadic grid
    {1, 2, ..., 2^27} * 2^-27, a subset of (0, 1]: zero never occurs, so the
    paper's "eps = 0 -> 1e-4" guard never fires, and every partial sum is a
    multiple of 2^-27 below 2^26, hence exact in binary64 whatever the order
    of summation (knots up to n = 6.7e7 are reproducible bit for bit by a
    parallel prefix sum).
  * y_i is an independent uniform draw on [0, 1) with 53 random bits.
"""
from __future__ import annotations

import numpy as np

GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_INST = np.uint64(0xD1B54A32D192ED03)
STREAM_X, STREAM_Y = 0, 1
EPS_BITS = 27


def mix64(z):
    """SplitMix64 output function (finaliser) on uint64 numpy values."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def stream_key(seed: int, instance: int, stream: int) -> np.uint64:
    """Key of one (seed, instance, stream) draw sequence."""
    with np.errstate(over="ignore"):
        k = mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + GOLDEN)
        k = mix64(k + np.uint64(instance) * _INST + np.uint64(stream))
    return np.uint64(k)


def draws(key, count: int, start: int = 0) -> np.ndarray:
    """Draws start..start+count-1 of the stream with the given key."""
    i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(key) + i * GOLDEN)


def curve(seed: int, n: int, instance: int = 0):
    """Knots x[n] (strictly increasing, x_0 = 0) and values y[n] of one random curve."""
    if n <= 0:
        return np.zeros(0), np.zeros(0)
    rx = draws(stream_key(seed, instance, STREAM_X), n - 1)
    inc = (rx >> np.uint64(64 - EPS_BITS)).astype(np.int64) + 1
    xi = np.zeros(n, dtype=np.int64)
    np.cumsum(inc, out=xi[1:])
    x = xi.astype(np.float64) * (2.0 ** -EPS_BITS)
    ry = draws(stream_key(seed, instance, STREAM_Y), n)
    y = (ry >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return x, y


def curve_continuous(seed: int, n: int, instance: int = 0):
    """The benchmark curve with the paper's continuous increments (section "Curve
    Interpolation", step 5, read literally): eps_i uniform on [0, 1) with 53 random bits (an
    eps of exactly 0 becomes 1e-4), x_i = x_{i-1} + eps_i summed left to right in binary64, so
    knot gaps carry up to 53 significant bits and the partial sums round.  Host-only (the
    sequential rounded sum has no bit-identical parallel form)."""
    if n <= 0:
        return np.zeros(0), np.zeros(0)
    rx = draws(stream_key(seed, instance, STREAM_X), n - 1)
    eps = (rx >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    eps[eps == 0.0] = 1e-4
    x = np.concatenate([[0.0], eps]).cumsum()
    ry = draws(stream_key(seed, instance, STREAM_Y), n)
    y = (ry >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return x, y


def curve_adversarial(seed: int, n: int, decades: float = 8.0):
    """Knots with gap ratios spread over many decades (log-uniform gaps in
    [10^-decades, 1]) and values in [-1, 1): stresses the conditioning of the
    fit and the halo truncation of the chunked solve.  Host-only."""
    rng = np.random.default_rng(seed)
    gaps = 10.0 ** (-decades * rng.random(n - 1))
    x = np.concatenate([[rng.random()], gaps]).cumsum()
    y = 2.0 * rng.random(n) - 1.0
    return x, y


def sizes_loguniform(seed: int, count: int, lo: float, hi: float) -> np.ndarray:
    """Instance sizes n = round(10^(log10 lo + u (log10 hi - log10 lo))) (host-only)."""
    r = draws(stream_key(seed, 0, 7), count)
    u = (r >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    e = np.log10(lo) + u * (np.log10(hi) - np.log10(lo))
    return np.rint(10.0 ** e).astype(np.int64)


def poisson_arrivals(seed: int, rate: float, count: int) -> np.ndarray:
    """Arrival times (seconds from 0) of a Poisson process: exponential gaps (host-only)."""
    r = draws(stream_key(seed, 0, 8), count)
    u = ((r >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)
    return np.cumsum(-np.log(u) / rate)
