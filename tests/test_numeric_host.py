"""The integer-pipe numerics of the mixed-precision kernels, compiled for the host from the
same header and checked against exact rational arithmetic (no GPU needed)."""
import ctypes
import math
import os
import subprocess
import tempfile
from fractions import Fraction

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2001_09253_gb300", "csrc")


@pytest.fixture(scope="module")
def lib():
    d = tempfile.mkdtemp(prefix="splnum_")
    so = os.path.join(d, "libnum.so")
    # no contraction of a*b + c: the error-free transformations must round each step as written
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fPIC", "-shared", "-I", CSRC, "-o", so,
                    os.path.join(HERE, "numeric_driver.cpp")], check=True)
    L = ctypes.CDLL(so)
    L.t_diff_f32.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_float)]
    L.t_diff_f32.restype = ctypes.c_int
    L.t_f32_to_f64.argtypes = [ctypes.c_float]
    L.t_f32_to_f64.restype = ctypes.c_double
    L.t_f64_to_f32.argtypes = [ctypes.c_double]
    L.t_f64_to_f32.restype = ctypes.c_float
    return L


def rn32(v: Fraction) -> float:
    """Exact round-to-nearest-even of a rational to binary32 (normal range)."""
    if v == 0:
        return 0.0
    s = -1 if v < 0 else 1
    a = abs(v)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    while Fraction(2) ** (e + 1) <= a:
        e += 1
    scaled = a / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    q, r = divmod(scaled.numerator, scaled.denominator)
    rem = Fraction(r, scaled.denominator)
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and q % 2 == 1):
        q += 1
    return float(np.float32(s * q * 2.0 ** (e - 23)))


def diff(L, b, a):
    out = ctypes.c_float()
    ok = L.t_diff_f32(b, a, ctypes.byref(out))
    return bool(ok), out.value


def _exp(v):
    return math.frexp(v)[1]


def test_diff_exact_on_close_operands(lib):
    rng = np.random.default_rng(0)
    cases = []
    for _ in range(4000):
        a = rng.normal() * 10.0 ** rng.integers(-6, 8)
        kind = rng.integers(0, 5)
        if kind == 0:
            b = np.nextafter(a, np.inf) if rng.random() < 0.5 else a + abs(a) * 1e-12 * rng.random()
        elif kind == 1:
            b = a * (1 + rng.random())
        elif kind == 2:
            b = a + rng.normal() * abs(a) * 10.0 ** rng.integers(-15, 1)
        elif kind == 3:
            b = -a * rng.random()
        else:
            b = a * 2.0 ** rng.integers(-9, 10) * rng.random()
        cases.append((float(b), float(a)))
    # knots of the benchmark curve and crossings of powers of two
    for v in [1.0, 2.0, 1024.0, 4194304.0]:
        cases += [(v, float(np.nextafter(v, 0))), (float(np.nextafter(v, np.inf)), float(np.nextafter(v, 0)))]
    for b, a in cases:
        if b == 0 or a == 0:
            continue
        ok, got = diff(lib, b, a)
        exact = Fraction(b) - Fraction(a)
        if exact != 0 and not (2.0 ** -126 <= abs(float(exact)) < 2.0 ** 127):
            assert not ok
            continue
        assert ok, (b, a)
        ref = rn32(exact)
        if abs(_exp(b) - _exp(a)) <= 9:
            assert got == ref, (b, a, got, ref)
        else:
            ulp = abs(float(np.spacing(np.float32(ref))))
            assert abs(got - float(exact)) <= ulp, (b, a, got, float(exact))


def test_same_binade_difference(lib):
    lib.t_diff_same_f32.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_float)]
    lib.t_diff_same_f32.restype = ctypes.c_int
    rng = np.random.default_rng(7)
    hits = 0
    for _ in range(6000):
        a = rng.normal() * 10.0 ** rng.integers(-20, 20)
        b = a + rng.normal() * abs(a) * 10.0 ** rng.integers(-16, 0)
        out = ctypes.c_float()
        ok = lib.t_diff_same_f32(float(b), float(a), ctypes.byref(out))
        same = (np.sign(a) == np.sign(b)) and _exp(a) == _exp(b) and a != 0
        if not same:
            assert not ok
            continue
        exact = Fraction(float(b)) - Fraction(float(a))
        if exact != 0 and not (2.0 ** -126 <= abs(float(exact)) < 2.0 ** 127):
            assert not ok
            continue
        assert ok
        hits += 1
        assert out.value == rn32(exact), (a, b)
    assert hits > 3000


def test_small_same_binade_difference(lib):
    lib.t_diff_small_f32.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_float)]
    lib.t_diff_small_f32.restype = ctypes.c_int
    rng = np.random.default_rng(8)
    hits = 0
    for _ in range(6000):
        a = rng.normal() * 10.0 ** rng.integers(-12, 12)
        b = a + abs(a) * rng.random() * 10.0 ** rng.integers(-16, -5)
        if rng.random() < 0.2:
            b = a
        out = ctypes.c_float()
        ok = lib.t_diff_small_f32(float(b), float(a), ctypes.byref(out))
        if not ok:
            continue
        hits += 1
        exact = Fraction(float(b)) - Fraction(float(a))
        assert out.value == rn32(exact), (a, b)
    assert hits > 3000
    # refused: different binades, negative differences, large exponents
    o = ctypes.c_float()
    assert not lib.t_diff_small_f32(2.0, 1.9, ctypes.byref(o))
    assert not lib.t_diff_small_f32(1.0, 1.5, ctypes.byref(o))
    assert not lib.t_diff_small_f32(1e300, 1e300 * (1 - 1e-15), ctypes.byref(o))


def test_ordered_difference_split_fma(lib):
    """The ordered same-binade route (b >= a) with the split ulp count and one FMA: exact
    rounding of b - a for positive and negative operands, up to 2^39 ulps apart; b < a, wider
    gaps and other binades refused."""
    lib.t_diff_up_f32.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_float)]
    lib.t_diff_up_f32.restype = ctypes.c_int
    rng = np.random.default_rng(9)
    hits = 0
    for _ in range(8000):
        a = rng.normal() * 10.0 ** rng.integers(-20, 20)
        b = a + abs(a) * rng.random() * 10.0 ** rng.integers(-16, -3)
        if rng.random() < 0.1:
            b = a
        out = ctypes.c_float()
        if not lib.t_diff_up_f32(float(b), float(a), ctypes.byref(out)):
            continue
        hits += 1
        exact = Fraction(float(b)) - Fraction(float(a))
        assert out.value == rn32(exact), (a, b)
        if exact == 0:
            assert math.copysign(1.0, out.value) == 1.0
    assert hits > 4000
    # the split boundary: D = 2^39 - 1 accepted, 2^39 refused; ties of the single rounding
    one = 1.0
    ulp = 2.0 ** -52
    o = ctypes.c_float()
    b = one + (2 ** 39 - 1) * ulp
    assert lib.t_diff_up_f32(b, one, ctypes.byref(o)) and o.value == rn32(Fraction(b) - 1)
    assert not lib.t_diff_up_f32(one + 2 ** 39 * ulp, one, ctypes.byref(o))
    for d in ((1 << 24) + 1, (1 << 24) + 3, (1 << 30) + (1 << 6), (1 << 30) + (3 << 6), (1 << 38) + (1 << 14)):
        b = one + d * ulp
        assert lib.t_diff_up_f32(b, one, ctypes.byref(o)) and o.value == rn32(Fraction(b) - 1), d
        assert lib.t_diff_up_f32(-one, -b, ctypes.byref(o)) and o.value == rn32(Fraction(b) - 1), d
        assert not lib.t_diff_up_f32(one, b, ctypes.byref(o)), d           # b < a
        assert not lib.t_diff_up_f32(-b, -one, ctypes.byref(o)), d         # b < a, negative
    assert not lib.t_diff_up_f32(2.0, 1.9, ctypes.byref(o))
    assert not lib.t_diff_up_f32(1e300, 1e300 * (1 - 1e-15), ctypes.byref(o))
    assert not lib.t_diff_up_f32(1.5e-300, 1e-300, ctypes.byref(o))


def test_diff_far_apart_and_signs(lib):
    rng = np.random.default_rng(1)
    for _ in range(2000):
        b = rng.normal() * 10.0 ** rng.integers(-10, 10)
        a = rng.normal() * 10.0 ** rng.integers(-30, 30)
        ok, got = diff(lib, b, a)
        exact = Fraction(float(b)) - Fraction(float(a))
        if exact == 0 or not (2.0 ** -126 <= abs(float(exact)) < 2.0 ** 127):
            continue
        assert ok
        ref = rn32(exact)
        ulp = abs(float(np.spacing(np.float32(ref))))
        assert abs(got - float(exact)) <= ulp


def test_diff_special_inputs_refused(lib):
    for b, a in [(0.0, 1.0), (1.0, 0.0), (5e-324, 1.0), (np.inf, 1.0), (1.0, np.nan), (1e300, -1e300),
                 (1.0 + 2 ** -52, 1.0 + 2 ** -51 - 2 ** -52 * 0)]:
        ok, got = diff(lib, b, a)
        exact = Fraction(float(b)) - Fraction(float(a)) if np.isfinite(b) and np.isfinite(a) else None
        if b == 0 or a == 0 or not np.isfinite(b) or not np.isfinite(a) or abs(b) < 2.2250738585072014e-308:
            assert not ok
        elif exact is not None and abs(float(exact)) >= 2.0 ** 128:
            assert not ok
    ok, got = diff(lib, 3.0, 3.0)
    assert ok and got == 0.0


def _f2(L, name, *args):
    a = ctypes.c_float()
    b = ctypes.c_float()
    getattr(L, name)(*args, ctypes.byref(a), ctypes.byref(b))
    return Fraction(a.value) + Fraction(b.value)


def _setup_df(L):
    f, pf = ctypes.c_float, ctypes.POINTER(ctypes.c_float)
    L.t_diff_f2.argtypes = [ctypes.c_double, ctypes.c_double, pf, pf]
    L.t_diff_f2.restype = ctypes.c_int
    L.t_df_div.argtypes = [f, f, f, f, pf, pf]
    L.t_df_add.argtypes = [f, f, f, f, pf, pf]
    L.t_df_mul_f.argtypes = [f, f, f, pf, pf]
    L.t_df_mul.argtypes = [f, f, f, f, pf, pf]
    L.t_two_sum.argtypes = [f, f, pf, pf]
    L.t_two_prod.argtypes = [f, f, pf, pf]
    for nm in ("t_df_div", "t_df_add", "t_df_mul_f", "t_df_mul", "t_two_sum", "t_two_prod"):
        getattr(L, nm).restype = None


def _pair(L, name, *args):
    a = ctypes.c_float()
    b = ctypes.c_float()
    getattr(L, name)(*args, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def _rand_f2(rng):
    hi = np.float32(rng.normal() * 10.0 ** rng.integers(-8, 8))
    lo = np.float32(float(hi) * rng.normal() * 2.0 ** -25)
    return float(hi), float(lo)


def test_double_float_difference_and_arithmetic(lib):
    _setup_df(lib)
    rng = np.random.default_rng(3)
    for _ in range(3000):
        a = rng.normal() * 10.0 ** rng.integers(-6, 7)
        b = a + rng.normal() * abs(a) * 10.0 ** rng.integers(-14, 1)
        hi, lo = ctypes.c_float(), ctypes.c_float()
        if not lib.t_diff_f2(b, a, ctypes.byref(hi), ctypes.byref(lo)):
            continue
        exact = Fraction(float(b)) - Fraction(float(a))
        got = Fraction(hi.value) + Fraction(lo.value)
        if exact == 0:
            assert got == 0
        else:
            assert abs(got - exact) <= abs(exact) * Fraction(1, 2 ** 47), (a, b)
            assert hi.value == rn32(exact)
    for _ in range(3000):
        ah, al = _rand_f2(rng)
        bh, bl = _rand_f2(rng)
        A, B = Fraction(ah) + Fraction(al), Fraction(bh) + Fraction(bl)
        q = _f2(lib, "t_df_div", ah, al, bh, bl)
        assert abs(q - A / B) <= abs(A / B) * Fraction(1, 2 ** 44)
        s = _f2(lib, "t_df_add", ah, al, bh, bl)
        assert abs(s - (A + B)) <= (abs(A) + abs(B)) * Fraction(1, 2 ** 46)
        c = float(np.float32(rng.normal()))
        p = _f2(lib, "t_df_mul_f", ah, al, c)
        assert abs(p - A * Fraction(c)) <= abs(A * Fraction(c)) * Fraction(1, 2 ** 46)


def test_error_free_sum_and_product(lib):
    """TwoSum and TwoProduct return the rounded result and its exact error: s + e == a + b and
    p + e == a * b exactly (operands within binary32's normal range, products not underflowing),
    with s and p the binary32 roundings; the double-float product carries ~46 bits."""
    _setup_df(lib)
    rng = np.random.default_rng(5)
    for _ in range(4000):
        a = float(np.float32(rng.normal() * 2.0 ** int(rng.integers(-30, 31))))
        b = float(np.float32(rng.normal() * 2.0 ** int(rng.integers(-30, 31))))
        s, e = _pair(lib, "t_two_sum", a, b)
        assert Fraction(s) + Fraction(e) == Fraction(a) + Fraction(b)
        assert s == rn32(Fraction(a) + Fraction(b)) or Fraction(a) + Fraction(b) == 0
        p, e = _pair(lib, "t_two_prod", a, b)
        assert Fraction(p) + Fraction(e) == Fraction(a) * Fraction(b)
        assert p == rn32(Fraction(a) * Fraction(b))
    for _ in range(3000):
        ah, al = _rand_f2(rng)
        bh, bl = _rand_f2(rng)
        A, B = Fraction(ah) + Fraction(al), Fraction(bh) + Fraction(bl)
        q = _f2(lib, "t_df_mul", ah, al, bh, bl)
        assert abs(q - A * B) <= abs(A * B) * Fraction(1, 2 ** 45)


def test_float_double_conversions(lib):
    rng = np.random.default_rng(2)
    vals = np.concatenate([rng.normal(size=3000) * 10.0 ** rng.integers(-37, 38, size=3000),
                           [0.0, -0.0, 1.0, -1.0, 3.4e38, 1.2e-38]])
    for v in vals.astype(np.float32):
        assert lib.t_f32_to_f64(float(v)) == float(v)
        assert math.copysign(1, lib.t_f32_to_f64(float(v))) == math.copysign(1, float(v))
    for v in rng.normal(size=5000) * 10.0 ** rng.integers(-37, 38, size=5000):
        assert lib.t_f64_to_f32(float(v)) == float(np.float32(v))
    # ties round to even
    for base in [1.0, 1.5, 3.0]:
        tie = base + 2.0 ** -24 * (1 if base < 2 else 2)
        assert lib.t_f64_to_f32(tie) == float(np.float32(tie))


def _f2_call(lib, name, *args):
    fn = getattr(lib, name)
    hi, lo = ctypes.c_float(), ctypes.c_float()
    ok = fn(*args, ctypes.byref(hi), ctypes.byref(lo))
    return bool(ok), Fraction(hi.value) + Fraction(lo.value), hi.value


def test_ordered_difference_as_double_float(lib):
    """The same-binade double-float width (b >= a): hi is b - a rounded to binary32, hi + lo is
    within 2^-47 of the exact difference; other binades, b < a and out-of-range scales refused."""
    lib.t_diff_up_f2.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_float)]
    lib.t_diff_up_f2.restype = ctypes.c_int
    rng = np.random.default_rng(12)
    hits = 0
    for _ in range(8000):
        a = rng.normal() * 10.0 ** rng.integers(-20, 20)
        b = a + abs(a) * rng.random() * 10.0 ** rng.integers(-16, 0)
        if rng.random() < 0.05:
            b = a
        ok, got, hi = _f2_call(lib, "t_diff_up_f2", float(b), float(a))
        if not ok:
            continue
        hits += 1
        exact = Fraction(float(b)) - Fraction(float(a))
        assert abs(got - exact) <= abs(exact) * Fraction(1, 2 ** 47), (a, b)
        assert hi == rn32(exact), (a, b)
    assert hits > 5000
    one, ulp = 1.0, 2.0 ** -52
    for d in (1, 2 ** 24 - 1, 2 ** 24, 2 ** 24 + 1, 2 ** 24 + 3, 3 * 2 ** 30 + 2 ** 6, 2 ** 51 + 12345, 2 ** 52 - 1):
        b = one + d * ulp
        for (bb, aa) in ((b, one), (-one, -b)):
            ok, got, hi = _f2_call(lib, "t_diff_up_f2", bb, aa)
            assert ok and got == Fraction(bb) - Fraction(aa) or abs(got - (Fraction(bb) - Fraction(aa))) <= \
                (Fraction(bb) - Fraction(aa)) * Fraction(1, 2 ** 47), d
        assert not _f2_call(lib, "t_diff_up_f2", one, b)[0], d          # b < a
    assert not _f2_call(lib, "t_diff_up_f2", 2.0, 1.9)[0]                # two binades
    assert not _f2_call(lib, "t_diff_up_f2", 1e300, 1e300 * (1 - 1e-15))[0]


def test_binary64_as_double_float(lib):
    """A binary64 value split into hi = RN32(d) and lo = RN32(d - hi): hi + lo within 2^-48 |d|,
    signs and zeros kept; values outside the range refused."""
    lib.t_f64_to_f2.argtypes = [ctypes.c_double, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]
    lib.t_f64_to_f2.restype = ctypes.c_int
    rng = np.random.default_rng(13)
    for _ in range(8000):
        d = float(rng.normal() * 10.0 ** rng.integers(-20, 30))
        ok, got, hi = _f2_call(lib, "t_f64_to_f2", d)
        assert ok == (2.0 ** -74 <= abs(d) < 2.0 ** 126), d  # binary64 exponents 949 .. 1149
        if not ok:
            continue
        assert hi == rn32(Fraction(d)), d
        assert abs(got - Fraction(d)) <= abs(Fraction(d)) * Fraction(1, 2 ** 48), d
    for d in (1.0, -1.0, 1.0 + 2.0 ** -52, 2.0 - 2.0 ** -52, -(2.0 - 2.0 ** -52), 1.0 + 2.0 ** -24, 1.0 + 3 * 2.0 ** -25,
              2.0 ** -70, 2.0 ** 100 * 1.7):
        ok, got, hi = _f2_call(lib, "t_f64_to_f2", d)
        assert ok and hi == rn32(Fraction(d)) and abs(got - Fraction(d)) <= abs(Fraction(d)) * Fraction(1, 2 ** 48), d
    ok, got, hi = _f2_call(lib, "t_f64_to_f2", -0.0)
    assert ok and got == 0 and math.copysign(1.0, hi) == -1.0
    for d in (1e-200, 1e200, 2.0 ** -80, 2.0 ** 127, float("inf"), float("nan"), 5e-324):
        assert not _f2_call(lib, "t_f64_to_f2", d)[0], d


def test_newint_in_double_float_against_exact(lib):
    """The one-division form of "Fast Interpolation" in double-float arithmetic against the same
    form evaluated exactly on the binary64 operands: within 2^-40 of the largest term magnitude
    (|y_j|, |y_{j+1}|, h^2 max|y''| / 6), far inside the FP64 path's 1e-12."""
    lib.t_newint_f2.argtypes = [ctypes.c_double] * 8 + [ctypes.POINTER(ctypes.c_double)]
    lib.t_newint_f2.restype = ctypes.c_int
    rng = np.random.default_rng(14)
    hits = 0
    for _ in range(4000):
        x0 = float(rng.random() * 10.0 ** rng.integers(-2, 7))
        h = float(abs(x0) * 10.0 ** rng.uniform(-9, -1) + 1e-3 * rng.random())
        x1 = x0 + h
        if not x1 > x0:
            continue
        q = x0 + (x1 - x0) * float(rng.random())
        q = min(max(q, x0), x1)
        y0, y1 = (float(v) for v in rng.normal(size=2) * 10.0 ** rng.integers(-3, 3))
        p0, p1 = (float(v) for v in rng.normal(size=2) * 10.0 ** rng.integers(-3, 6))
        inv = 1.0 / (x1 - x0)
        out = ctypes.c_double()
        if not lib.t_newint_f2(q, x0, x1, y0, y1, p0, p1, inv, ctypes.byref(out)):
            continue
        hits += 1
        Q, X0, X1 = Fraction(q), Fraction(x0), Fraction(x1)
        xa, bx, ba = Q - X0, X1 - Q, X1 - X0
        exact = (xa * Fraction(y1) + bx * Fraction(y0) + ((xa * xa - ba * ba) * xa * Fraction(p1) +
                 (bx * bx - ba * ba) * bx * Fraction(p0)) / 6) * Fraction(inv)
        scale = max(abs(Fraction(y0)), abs(Fraction(y1)), ba * ba * max(abs(Fraction(p0)), abs(Fraction(p1))) / 6)
        assert abs(Fraction(out.value) - exact) <= scale * Fraction(1, 2 ** 40), (q, x0, x1)
    assert hits > 2500
