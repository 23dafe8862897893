"""Pins that tie the FP64 oracle to the paper and to the mathematics (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, a swapped end-row coefficient)
fails at least one of them; ``test_oracle_mutants.py`` plants such slips in a
copy of the oracle and confirms it.
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from exact_spline import ExactSpline
from paper_2001_09253_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# Section "Quality Checks": the hand-made 13-knot test curve.
TEST_KNOTS = [0, 0.5, 1, 1.01, 1.25, 1.5, 1.58, 1.79, 2.12, 2.30, 2.402, 2.451, 2.5]
TEST_VALUES = [1, 1.2, 2, 0.25, 0.25, 0.25, 0.63, 0.96, 1.17, 1.23, 1.245, 1.249, 1.25]
# The three end conditions exercised there: natural, y'_1 = y'_n = 0, and y'_1 = -1, y'_n = 1.
BC_CASES = [(None, None), (0.0, 0.0), (-1.0, 1.0)]


def _slope(s):
    return oracle.NATURAL if s is None else s


def _normwise(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


def load_golden_table():
    rows = []
    with open(os.path.join(GOLDEN, "test_compare_nat1.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(v) for v in line.split()])
    return np.array(rows)


def test_golden_fixture_matches_curve():
    t = load_golden_table()
    assert t.shape == (13, 3)
    assert np.array_equal(t[:, 0], np.array(TEST_KNOTS, float))
    assert np.array_equal(t[:, 1], np.array(TEST_VALUES, float))


def test_printed_natural_table():
    """Table tbl:test_compare_nat1 prints y'' to 6 decimals for the natural spline."""
    t = load_golden_table()
    st, ypp = oracle.fit(t[:, 0], t[:, 1])
    assert st == oracle.OK
    np.testing.assert_array_less(np.abs(ypp - t[:, 2]), 5.0e-7 + 1e-12)
    # and the rounded values agree digit for digit
    assert [round(v, 6) for v in ypp] == [round(v, 6) for v in t[:, 2]]


def load_true_tables():
    """Per-knot deltas (13 x 8: x, y, then NR and "our" for natural, flat, twist), the six
    printed mean square errors of y'' and the two of the interpolated curve."""
    rows, mse, mse_full = [], None, None
    with open(os.path.join(GOLDEN, "test_compare_true.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("mse_full"):
                mse_full = np.array([float(v) for v in line.split()[1:]])
            elif line.startswith("mse"):
                mse = np.array([float(v) for v in line.split()[1:]])
            else:
                rows.append([float(v) for v in line.split()])
    return np.array(rows), mse, mse_full


def test_true_tables_fixture_consistent():
    """The transcribed deltas of Tables tbl:test_compare_nat / _flat / _twist reproduce the
    mean square errors the paper prints for them (Tables tbl:mse_nat / _flat / _twist)."""
    t, mse, mse_full = load_true_tables()
    assert t.shape == (13, 8) and mse.shape == (6,) and mse_full.shape == (2,)
    assert np.array_equal(t[:, 0], np.array(TEST_KNOTS, float))
    assert np.array_equal(t[:, 1], np.array(TEST_VALUES, float))
    np.testing.assert_allclose(np.mean(t[:, 2:] ** 2, axis=0), mse, rtol=2e-5)


@pytest.mark.parametrize("case", range(3))
def test_oracle_rounding_matches_printed_true_tables(case):
    """Section "Quality Checks" compares both double routines with a 30-digit solve.  Its
    high-precision knots and values are created before the working precision is raised, at
    mpmath's default 53 bits, so its "true" is the exact spline of the binary64 inputs; the
    exact rational spline stands in for it here.  The oracle's deltas are no larger in mean
    square than the worse of the paper's two routines, and at most knots equal the printed
    delta of one of them to its 5 digits: the oracle performs the paper's operations in the
    paper's order (a changed operation or order moves the deltas; a wrong term moves them by
    orders of magnitude)."""
    t, mse, _ = load_true_tables()
    bc = BC_CASES[case]
    ex = ExactSpline(TEST_KNOTS, TEST_VALUES, bc[0], bc[1])
    st, ypp = oracle.fit(TEST_KNOTS, TEST_VALUES, _slope(bc[0]), _slope(bc[1]))
    assert st == oracle.OK
    d = np.array([float(Fraction(float(a)) - e) for a, e in zip(ypp, ex.second_derivatives())])
    nr, our = t[:, 2 + 2 * case], t[:, 3 + 2 * case]
    assert np.mean(d ** 2) <= 1.01 * max(mse[2 * case], mse[2 * case + 1])
    assert np.max(np.abs(d)) <= 1.01 * max(np.max(np.abs(nr)), np.max(np.abs(our)))
    same = [np.isclose(v, p, rtol=1e-4, atol=0.0) or (v == 0.0 and p == 0.0)
            for v, pair in zip(d, zip(nr, our)) for p in pair]
    knots_same = sum(any(same[2 * k: 2 * k + 2]) for k in range(13))
    assert knots_same >= 9, knots_same


def test_interpolated_curve_error_matches_printed_mse():
    """Table tbl:mse_full: the twist-end spline of the 13-knot curve evaluated at 2048 evenly
    spaced queries (monotone sweep, one-division form) against the "true" curve.  The oracle's
    mean square error against the exact spline of the binary64 inputs is within the printed
    ones (~1e-30; a wrong term in the cubic or a wrong bracket gives errors many orders larger)."""
    _, _, mse_full = load_true_tables()
    ex = ExactSpline(TEST_KNOTS, TEST_VALUES, -1.0, 1.0)
    res = oracle.fit_eval(TEST_KNOTS, TEST_VALUES, -1.0, 1.0, 2048)
    assert res["status"] == oracle.OK
    d = np.array([float(Fraction(float(v)) - ex.piece_value(int(j), float(q)))
                  for v, j, q in zip(res["yq"], res["jq"], res["xq"])])
    assert np.mean(d ** 2) <= 1.01 * np.max(mse_full)


@pytest.mark.parametrize("bc", BC_CASES)
def test_paper_curve_matches_exact_spline(bc):
    """All three end-condition cases of the quality checks against the exact rational spline."""
    ex = ExactSpline(TEST_KNOTS, TEST_VALUES, bc[0], bc[1])
    exact = [float(v) for v in ex.second_derivatives()]
    st, ypp = oracle.fit(TEST_KNOTS, TEST_VALUES, _slope(bc[0]), _slope(bc[1]))
    assert st == oracle.OK
    assert _normwise(ypp, exact) < 1e-14


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("bc", BC_CASES + [(None, 2.5), (-3.0, None)])
def test_random_curves_match_exact_spline(seed, bc):
    n = 3 + (seed * 5) % 17
    x, y = synth.curve(100 + seed, n)
    ex = ExactSpline(x, y, bc[0], bc[1])
    exact = [float(v) for v in ex.second_derivatives()]
    st, ypp = oracle.fit(x, y, _slope(bc[0]), _slope(bc[1]))
    assert st == oracle.OK
    assert _normwise(ypp, exact) < 1e-13
    # interpolated values on the uniform grid against the exact piecewise cubic
    res = oracle.fit_eval(x, y, _slope(bc[0]), _slope(bc[1]), m=3 * n + 1)
    ev = [float(ex.piece_value(int(j), q)) for j, q in zip(res["jq"], res["xq"])]
    scale = np.maximum(np.abs(ev), np.max(np.abs(y)))
    assert np.max(np.abs(res["yq"] - ev) / scale) < 1e-13


def test_adversarial_gaps_match_exact_spline():
    x, y = synth.curve_adversarial(7, 14, decades=6)
    for bc in BC_CASES:
        ex = ExactSpline(x, y, bc[0], bc[1])
        exact = [float(v) for v in ex.second_derivatives()]
        st, ypp = oracle.fit(x, y, _slope(bc[0]), _slope(bc[1]))
        assert st == oracle.OK
        assert _normwise(ypp, exact) < 1e-12


def test_scipy_cubic_spline_cross_check():
    """Library cross-check: scipy's CubicSpline solves the same interpolation problem."""
    from scipy.interpolate import CubicSpline
    x, y = synth.curve(3, 2000)
    for bc, bc_sp in [((None, None), "natural"), ((-1.0, 1.0), ((1, -1.0), (1, 1.0)))]:
        cs = CubicSpline(x, y, bc_type=bc_sp)
        st, ypp = oracle.fit(x, y, _slope(bc[0]), _slope(bc[1]))
        assert st == oracle.OK
        assert _normwise(ypp, cs(x, 2)) < 1e-10
        res = oracle.fit_eval(x, y, _slope(bc[0]), _slope(bc[1]), m=5000)
        ref = cs(res["xq"])
        assert np.max(np.abs(res["yq"] - ref)) / np.max(np.abs(ref)) < 1e-10


@pytest.mark.parametrize("seed", range(4))
def test_clamped_spline_reproduces_cubics(seed):
    """A clamped spline with the end slopes of a cubic p reproduces p exactly: y'' = p''."""
    rng = np.random.default_rng(seed)
    c = rng.normal(size=4)
    x = np.sort(rng.random(40)) * 3.0 - 1.0
    p = np.polynomial.Polynomial(c)
    d1, d2 = p.deriv(1), p.deriv(2)
    st, ypp = oracle.fit(x, p(x), d1(x[0]), d1(x[-1]))
    assert st == oracle.OK
    assert _normwise(ypp, d2(x)) < 1e-9
    res = oracle.fit_eval(x, p(x), d1(x[0]), d1(x[-1]), m=301)
    assert np.max(np.abs(res["yq"] - p(res["xq"]))) / np.max(np.abs(p(x))) < 1e-11


def test_natural_spline_of_a_line_is_the_line():
    x, _ = synth.curve(5, 500)
    y = 3.0 - 0.25 * x
    st, ypp = oracle.fit(x, y)
    assert st == oracle.OK
    assert np.max(np.abs(ypp)) < 1e-12
    res = oracle.fit_eval(x, y, m=777)
    np.testing.assert_allclose(res["yq"], 3.0 - 0.25 * res["xq"], rtol=0, atol=1e-12 * np.max(np.abs(y)))


def test_uniform_knots_reduce_to_textbook_141_system():
    """Equal spacing h turns the interior rows into h/6 [1 4 1] y'' = second differences / h;
    solved here by LAPACK's banded solver."""
    from scipy.linalg import solve_banded
    n, h = 200, 0.125
    x = np.arange(n) * h
    y = np.sin(3 * x) + 0.1 * np.cos(17 * x)
    st, ypp = oracle.fit(x, y)
    assert st == oracle.OK
    m = n - 2
    ab = np.zeros((3, m))
    ab[0, 1:] = 1.0
    ab[1, :] = 4.0
    ab[2, :-1] = 1.0
    rhs = 6.0 * (y[2:] - 2 * y[1:-1] + y[:-2]) / h ** 2
    inner = solve_banded((1, 1), ab, rhs)
    assert ypp[0] == 0.0 and ypp[-1] == 0.0
    assert _normwise(ypp[1:-1], inner) < 1e-13


@pytest.mark.parametrize("bc", BC_CASES)
def test_defining_conditions_hold(bc):
    """S(x_j) = y_j, S' continuous at interior knots, end conditions; evaluated exactly
    from the oracle's y'' with the textbook one-sided slopes of the second-derivative form."""
    x, y = synth.curve(11, 60)
    st, ypp = oracle.fit(x, y, _slope(bc[0]), _slope(bc[1]))
    assert st == oracle.OK
    X = [Fraction(v) for v in x]
    Y = [Fraction(v) for v in y]
    P = [Fraction(v) for v in ypp]
    n = len(x)

    def slope_right(j):  # S'(x_j) from the piece [x_j, x_{j+1}]
        h = X[j + 1] - X[j]
        return (Y[j + 1] - Y[j]) / h - h * (2 * P[j] + P[j + 1]) / 6

    def slope_left(j):  # S'(x_j) from the piece [x_{j-1}, x_j]
        h = X[j] - X[j - 1]
        return (Y[j] - Y[j - 1]) / h + h * (P[j - 1] + 2 * P[j]) / 6

    scale = max(abs(float(slope_right(j))) for j in range(n - 1))
    jumps = [abs(float(slope_left(j) - slope_right(j))) for j in range(1, n - 1)]
    assert max(jumps) < 1e-12 * scale
    if bc[0] is None:
        assert ypp[0] == 0.0
    else:
        assert abs(float(slope_right(0)) - bc[0]) < 1e-12 * scale
    if bc[1] is None:
        assert ypp[-1] == 0.0
    else:
        assert abs(float(slope_left(n - 1)) - bc[1]) < 1e-12 * scale
    # interpolation at the knots: a query equal to x_j takes the interval on its left
    yk = oracle.evaluate(x, y, ypp, x)
    assert np.max(np.abs(yk - y)) < 1e-13


def test_interpolation_form_equals_nr_form_exactly():
    """The paper's cancelled form against eq. (nr_formula) with its A, B, C, D, evaluated in
    exact rationals on random intervals."""
    rng = np.random.default_rng(1)
    worst = 0.0
    for _ in range(2000):
        a = rng.normal() * 10.0 ** rng.integers(-3, 4)
        b = a + rng.random() * 10.0 ** rng.integers(-4, 2) + 1e-12
        if not b > a:
            continue
        q = a + (b - a) * rng.random()
        u, v, up, vp = rng.normal(size=4) * np.array([1, 1, 100, 100])
        got = oracle.interp(q, a, b, u, v, up, vp)
        A_, B_, Q = Fraction(a), Fraction(b), Fraction(q)
        A = (B_ - Q) / (B_ - A_)
        B = (Q - A_) / (B_ - A_)
        C = (A ** 3 - A) * (B_ - A_) ** 2 / 6
        D = (B ** 3 - B) * (B_ - A_) ** 2 / 6
        ref = A * Fraction(u) + B * Fraction(v) + C * Fraction(up) + D * Fraction(vp)
        scale = max(abs(u), abs(v), abs(float(ref)), abs(float(C * Fraction(up))), abs(float(D * Fraction(vp))))
        worst = max(worst, abs(got - float(ref)) / scale)
    assert worst < 1e-13


def test_query_grid_is_numpy_linspace():
    for n, m, seed in [(10, 2, 0), (1000, 1000, 1), (777, 4096, 2), (50, 3, 3)]:
        x, _ = synth.curve(seed, n)
        xq = oracle.grid(x, m)
        assert np.array_equal(xq, np.linspace(x[0], x[-1], m))
    x, _ = synth.curve(0, 9)
    assert np.array_equal(oracle.grid(x, 1), np.linspace(x[0], x[-1], 1))
    # grids whose last product-and-sum point misses the last knot by rounding: the last query
    # is the knot itself (numpy.linspace sets it so too)
    for knots, m in (([0.1, 0.4, 0.7, 1.0], 4), ([-1.1, 0.5, 3.3], 2), ([0.0, 1.0, 2.5], 78)):
        x = np.array(knots)
        assert (m - 1) * ((x[-1] - x[0]) / (m - 1)) + x[0] != x[-1]  # the case meant
        xq = oracle.grid(x, m)
        assert np.array_equal(xq, np.linspace(x[0], x[-1], m)) and xq[-1] == x[-1]


def test_bracket_sweep_and_bisection_match_brute_force():
    rng = np.random.default_rng(5)
    for trial in range(30):
        n = int(rng.integers(3, 60))
        x = np.sort(rng.choice(np.arange(-50, 50) * 0.25, size=n, replace=False))
        # queries hit knots exactly, fall between them and lie past both ends
        xq = np.sort(np.concatenate([x, x + 0.1, [x[0] - 1, x[-1] + 1], rng.random(20) * 30 - 15]))
        brute = []
        for q in xq:
            below = [i for i in range(n - 1) if x[i] < q]
            brute.append(max(below) if below else 0)
        assert np.array_equal(oracle.bracket_sweep(x, xq), brute)
        assert np.array_equal(oracle.bracket_any(x, xq), brute)
        perm = rng.permutation(len(xq))
        assert np.array_equal(oracle.bracket_any(x, xq[perm]), np.array(brute)[perm])


def test_validation_codes():
    x = np.array([0.0, 1.0, 2.0, 3.0])
    y = np.array([0.0, 1.0, 0.0, 1.0])
    assert oracle.validate(x, y) == oracle.OK
    assert oracle.validate(x[:2], y[:2]) == oracle.INVALID_ARG
    assert oracle.validate(x, y, np.nan, 0.0) == oracle.INVALID_ARG
    assert oracle.validate(x, y, 0.0, -np.inf) == oracle.INVALID_ARG
    assert oracle.validate(x, y, np.inf, np.inf) == oracle.OK
    bad = x.copy()
    bad[2] = 1.0
    assert oracle.validate(bad, y) == oracle.NOT_INCREASING
    bad = y.copy()
    bad[1] = np.nan
    assert oracle.validate(x, bad) == oracle.NONFINITE
    bad = x.copy()
    bad[3] = np.inf
    assert oracle.validate(bad, y) == oracle.NONFINITE


def test_natural_sentinel_threshold():
    x, y = synth.curve(2, 30)
    st_a, a = oracle.fit(x, y, 0.99e30, 0.99e30)   # not above the threshold: clamped
    st_b, b = oracle.fit(x, y, 1.0e31, 1.0e31)     # above: natural
    assert st_a == st_b == oracle.OK
    assert b[0] == 0.0 and b[-1] == 0.0
    assert a[0] != 0.0
