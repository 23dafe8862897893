"""The division replacement of the plain FP64 kernel against IEEE division, through the C ABI
(spl_selftest_div64).

The FP64 kernel forms slopes s_j = (y_{j+1} - y_j) / h_j (eq. (init_val)) as a MUFU-seeded
reciprocal refined by a Newton step plus a Markstein correction.  The slopes feed the cancelling
difference s_j - s_{j-1}, so the kernel claims they equal the correctly rounded quotient bit for
bit.  Here that claim is checked on 1.3e7 operand pairs: the benchmark generator's dyadic widths,
continuous and 8-decade gaps with value differences, random significands over +-1000 binades,
powers of two and their neighbours, all-ones significands, zeros, and the ends of the exponent
range (where the fast routines hand over to the IEEE ones).  CUDA's __ddiv_rn / __drcp_rn results
are themselves checked against numpy's IEEE division on the host."""
import numpy as np
import pytest

from paper_2001_09253_gb300 import spl

pytestmark = pytest.mark.gpu


def operand_sets(rng, per=2_000_000):
    out = []
    k = rng.integers(1, 2 ** 27 + 1, per).astype(np.float64) * 2.0 ** -27
    out.append(("dyadic widths", rng.random(per) - rng.random(per), k))
    x = np.concatenate([[0.0], rng.random(per)]).cumsum()
    h = np.diff(x)
    h = h[h > 0]
    out.append(("continuous widths", rng.random(len(h)) - rng.random(len(h)), h))
    g = 10.0 ** (-8.0 * rng.random(per))
    x = np.concatenate([[rng.random()], g]).cumsum()
    h = np.diff(x)
    h = h[h > 0]
    out.append(("8-decade widths", 2 * rng.random(len(h)) - 1, h))
    num = np.ldexp(1 + rng.random(per), rng.integers(-1000, 1001, per)) * rng.choice([-1.0, 1.0], per)
    out.append(("random binades", num, np.ldexp(1 + rng.random(per), rng.integers(-1000, 1001, per))))
    e = rng.integers(-1000, 1001, per // 4)
    p2 = np.ldexp(1.0, e)
    dens = np.concatenate([p2, np.nextafter(p2, np.inf), np.nextafter(p2, 0), np.ldexp(2.0 - 2.0 ** -52, e)])
    out.append(("powers of two, neighbours, all-ones", 1 + rng.random(len(dens)), dens))
    nums = np.concatenate([np.ldexp(2.0 - 2.0 ** -52, rng.integers(-500, 500, per // 4)),
                           np.ldexp(1.0, rng.integers(-500, 500, per // 4)),
                           np.zeros(1000), -np.zeros(1000)])
    out.append(("special numerators", nums, 1 + rng.random(len(nums))))
    ee = np.concatenate([rng.integers(1010, 1024, per // 8), rng.integers(-1074, -1000, per // 8)])
    edge = np.ldexp(1 + rng.random(len(ee)), ee)
    out.append(("ends of the exponent range", 1 + rng.random(len(edge)), edge))
    return out


def _bits(a):
    return np.ascontiguousarray(a).view(np.uint64)


def test_quotients_bit_exact_and_reciprocals_faithful():
    import torch
    rng = np.random.default_rng(7)
    total = 0
    for name, num, den in operand_sets(rng):
        nt = torch.from_numpy(np.ascontiguousarray(num)).cuda()
        dt = torch.from_numpy(np.ascontiguousarray(den)).cuda()
        qf, rf, qi, ri = [t.cpu().numpy() for t in spl.selftest_div64(nt, dt)]
        with np.errstate(all="ignore"):
            qh, rh = num / den, 1.0 / den
        assert np.array_equal(_bits(qi), _bits(qh)), name   # CUDA's IEEE division is numpy's
        assert np.array_equal(_bits(ri), _bits(rh)), name
        bad = np.nonzero(_bits(qf) != _bits(qi))[0]
        assert bad.size == 0, "%s: %d quotients differ, e.g. %r / %r" % (name, bad.size, num[bad[0]], den[bad[0]])
        # the reciprocal alone is within one ulp of the IEEE one
        d_ulp = np.abs(_bits(rf).astype(np.int64) - _bits(ri).astype(np.int64))
        assert int(d_ulp.max()) <= 1, name
        total += len(num)
    assert total >= 10_000_000


@pytest.mark.gpu
def test_dfma_probe_counts_and_converges():
    """spl_selftest_dfma: the lane-operation count it reports is SMs x warps x 32 threads x trips x
    16 steps x 4 chains, and every chain of a <- a/2 + 1/2 reaches the fixed point 1 exactly (the
    sum of a thread's four chains is 4); a sink shorter than one value per thread is refused."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sink = torch.full((sms * 4 * 32,), float("nan"), dtype=torch.float64, device="cuda")
    ops = spl.selftest_dfma(100, 4, sink, mul=0.5, add=0.5)
    torch.cuda.synchronize()
    assert ops == sms * 4 * 32 * 100 * 16 * 4
    assert bool((sink == 4.0).all())
    with pytest.raises(spl.SplError):
        spl.selftest_dfma(1, 4, sink[:100])
    with pytest.raises(spl.SplError):
        spl.selftest_dfma(1, 0, sink)
