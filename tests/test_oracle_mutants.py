"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check that the
pins of ``test_oracle_pins.py`` catch every one of them."""
import inspect
import os
import shutil
import tempfile

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "spline_oracle.c")

MUTANTS = [
    ("diagonal loses its factor 2", "*b = 2.0 * (aj + cj);", "*b = (aj + cj);"),
    ("sign of the slope difference", "*d = 6.0 * ((y[j + 1] - y[j]) / cj - (y[j] - y[j - 1]) / aj);",
     "*d = 6.0 * ((y[j + 1] - y[j]) / cj + (y[j] - y[j - 1]) / aj);"),
    ("sign of the start slope", "*d = 6.0 * ((y[1] - y[0]) / h - yp1);", "*d = 6.0 * ((y[1] - y[0]) / h + yp1);"),
    ("last clamped row with a_n and b_n swapped as printed", "*a = h;\n    *b = 2.0 * h;", "*a = 2.0 * h;\n    *b = h;"),
    ("elimination uses c instead of a", "double den = b - a * cp[i - 1];", "double den = b - c * cp[i - 1];"),
    ("back substitution off by one", "ypp[i] = ypp[i] - cp[i] * ypp[i + 1];", "ypp[i] = ypp[i] - cp[i + 1] * ypp[i + 1];"),
    ("transposed operand in the cubic term", "ppj * right * (right * right - w2)", "ppj * left * (right * right - w2)"),
    ("dropped 1/6", "v / 6.0", "v"),
    ("swapped node values", "yj * right + yj1 * left", "yj * left + yj1 * right"),
    ("tie goes to the right interval", "x[i + 1] < xq[k]", "x[i + 1] <= xq[k]"),
    ("natural sentinel not strict", "slope > 0.99e30", "slope >= 0.99e30"),
    ("grid product and sum fused order", "double t = (double)k * step;\n    xq[k] = t + x[0];",
     "xq[k] = x[0] + (double)k * (x[n - 1] - x[0]) / (double)(m - 1);"),
    ("first clamped row with b and c swapped", "*b = 2.0 * h;\n    *c = h;", "*b = h;\n    *c = 2.0 * h;"),
    ("sign of the end slope", "*d = 6.0 * (ypn - (y[n - 1] - y[n - 2]) / h);",
     "*d = 6.0 * ((y[n - 1] - y[n - 2]) / h - ypn);"),
    ("interior widths transposed in the slopes", "/ cj - (y[j] - y[j - 1]) / aj);", "/ aj - (y[j] - y[j - 1]) / cj);"),
    ("interior a and c swapped", "*a = aj;\n  *c = cj;", "*a = cj;\n  *c = aj;"),
    ("first c' formed from d", "cp[0] = c / b;", "cp[0] = d / b;"),
    ("back substitution skips the second-to-last row", "for (int64_t i = n - 2; i >= 0; --i)",
     "for (int64_t i = n - 3; i >= 0; --i)"),
    ("grid step over m instead of m - 1", "/ (double)(m - 1);", "/ (double)m;"),
    ("last grid point not forced to the last knot", "  xq[m - 1] = x[n - 1];\n", ""),
    ("y''_{j+1} replaced by y''_j in the cubic", "ppj1 * left * (left * left - w2)", "ppj * left * (left * left - w2)"),
    ("squared width taken from the left offset", "double w2 = width * width;", "double w2 = left * left;"),
    ("equal knots let through", "if (!(x[i] > x[i - 1])) return ORC_NOT_INCREASING;",
     "if (!(x[i] >= x[i - 1])) return ORC_NOT_INCREASING;"),
    ("bisection sends a tie to the right", "if (x[mid] < q) lo = mid + 1;", "if (x[mid] <= q) lo = mid + 1;"),
    ("bisection never reaches the last interval", "int64_t lo = 0, hi = n - 1;", "int64_t lo = 0, hi = n - 2;"),
    ("sweep never reaches the last interval", "while (i + 1 < n - 1 && x[i + 1] < xq[k]) ++i;",
     "while (i + 1 < n - 2 && x[i + 1] < xq[k]) ++i;"),
    ("evaluation takes y''_j at both ends of the interval", "ypp[j], ypp[j + 1]);", "ypp[j], ypp[j]);"),
    ("evaluation takes the right knot's value twice", "y[j], y[j + 1], ypp[j]", "y[j + 1], y[j + 1], ypp[j]"),
    ("non-finite values let through", "if (!isfinite(x[i]) || !isfinite(y[i])) return ORC_NONFINITE;",
     "if (!isfinite(x[i])) return ORC_NONFINITE;"),
    ("whole path brackets against the first knot only", "orc_bracket_sweep(n, x, m, xq, jq);\n  orc_eval",
     "for (int64_t k = 0; k < m; ++k) jq[k] = 0;\n  orc_eval"),
]


def _pin_functions():
    out = []
    for name, fn in inspect.getmembers(pins, inspect.isfunction):
        if not name.startswith("test_"):
            continue
        params = inspect.signature(fn).parameters
        marks = getattr(fn, "pytestmark", [])
        grid = {}
        for mk in marks:
            if mk.name == "parametrize":
                grid[mk.args[0]] = list(mk.args[1])
        if not params:
            out.append((name, fn, {}))
        else:
            import itertools
            keys = list(params)
            for combo in itertools.product(*[grid[k] for k in keys]):
                out.append((name, fn, dict(zip(keys, combo))))
    return out


@pytest.fixture(scope="module")
def workdir():
    d = tempfile.mkdtemp(prefix="oracle_mut_")
    yield d
    shutil.rmtree(d, ignore_errors=True)


@pytest.mark.parametrize("desc,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(desc, old, new, workdir):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor not unique: %r" % old
    tag = str(abs(hash(desc)))
    cpath = os.path.join(workdir, "mut_%s.c" % tag)
    with open(cpath, "w") as f:
        f.write(src.replace(old, new))
    so = oracle.compile_source(cpath, os.path.join(workdir, "mut_%s.so" % tag))
    caught = None
    with oracle.swapped(so):
        for name, fn, kw in _pin_functions():
            try:
                fn(**kw)
            except (AssertionError, ValueError, FloatingPointError, ZeroDivisionError):
                caught = name
                break
    assert caught is not None, "no pin caught: " + desc
