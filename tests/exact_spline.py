"""Exact-rational reference for the interpolating cubic spline, used to pin the oracle.

This is deliberately NOT the paper's tridiagonal formulation: every piece is an
unknown cubic  S_i(t) = p0 + p1 t + p2 t^2 + p3 t^3  in t = x - x_i, and the
4(n-1) unknowns are fixed by the defining conditions of a C2 interpolating
spline (values at both ends of every piece, equal first and second derivatives
at every interior knot, and one condition per end: S'' = 0 for a natural end,
S' = the given slope for a clamped end).  The dense system is solved by
Gaussian elimination over Fractions, so the result is exact for the rational
values of the double inputs.  It is slow (cubic in n) and meant for n <= ~30.
"""
from __future__ import annotations

from fractions import Fraction


def _solve_exact(A, b):
    n = len(A)
    M = [row[:] + [b[i]] for i, row in enumerate(A)]
    for col in range(n):
        piv = None
        for r in range(col, n):
            if M[r][col] != 0:
                piv = r
                break
        if piv is None:
            raise ValueError("singular system")
        if piv != col:
            M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        for r in range(col + 1, n):
            f = M[r][col]
            if f != 0:
                f = f / pv
                Mr, Mc = M[r], M[col]
                for c in range(col, n + 1):
                    if Mc[c] != 0:
                        Mr[c] -= f * Mc[c]
    x = [Fraction(0)] * n
    for r in range(n - 1, -1, -1):
        s = M[r][n]
        for c in range(r + 1, n):
            if M[r][c] != 0:
                s -= M[r][c] * x[c]
        x[r] = s / M[r][r]
    return x


def _rational(v):
    """A Fraction or a decimal string is taken as given; anything else as its binary64 value."""
    return v if isinstance(v, Fraction) else Fraction(v) if isinstance(v, str) else Fraction(float(v))


class ExactSpline:
    """The exact spline through (x_i, y_i); slopes None mean a natural end."""

    def __init__(self, x, y, slope0=None, slope1=None):
        X = [_rational(v) for v in x]
        Y = [_rational(v) for v in y]
        n = len(X)
        assert n >= 3
        npc = n - 1
        N = 4 * npc
        rows, rhs = [], []

        def row():
            return [Fraction(0)] * N

        H = [X[i + 1] - X[i] for i in range(npc)]
        for i in range(npc):
            r = row()
            r[4 * i] = Fraction(1)
            rows.append(r)
            rhs.append(Y[i])
            r = row()
            h = H[i]
            r[4 * i:4 * i + 4] = [Fraction(1), h, h * h, h * h * h]
            rows.append(r)
            rhs.append(Y[i + 1])
        for i in range(npc - 1):
            h = H[i]
            r = row()  # S_i'(h) - S_{i+1}'(0) = 0
            r[4 * i + 1], r[4 * i + 2], r[4 * i + 3] = Fraction(1), 2 * h, 3 * h * h
            r[4 * (i + 1) + 1] = Fraction(-1)
            rows.append(r)
            rhs.append(Fraction(0))
            r = row()  # S_i''(h) - S_{i+1}''(0) = 0
            r[4 * i + 2], r[4 * i + 3] = Fraction(2), 6 * h
            r[4 * (i + 1) + 2] = Fraction(-2)
            rows.append(r)
            rhs.append(Fraction(0))
        r = row()
        if slope0 is None:
            r[2] = Fraction(2)
            rhs.append(Fraction(0))
        else:
            r[1] = Fraction(1)
            rhs.append(Fraction(float(slope0)))
        rows.append(r)
        r = row()
        h = H[-1]
        k = 4 * (npc - 1)
        if slope1 is None:
            r[k + 2], r[k + 3] = Fraction(2), 6 * h
            rhs.append(Fraction(0))
        else:
            r[k + 1], r[k + 2], r[k + 3] = Fraction(1), 2 * h, 3 * h * h
            rhs.append(Fraction(float(slope1)))
        rows.append(r)
        sol = _solve_exact(rows, rhs)
        self.X, self.Y, self.H = X, Y, H
        self.coef = [sol[4 * i:4 * i + 4] for i in range(npc)]

    def second_derivatives(self):
        """S''(x_j) for every knot (the last one from the last piece)."""
        out = [2 * c[2] for c in self.coef]
        c = self.coef[-1]
        h = self.H[-1]
        out.append(2 * c[2] + 6 * c[3] * h)
        return out

    def piece_value(self, i, q):
        c = self.coef[i]
        t = Fraction(float(q)) - self.X[i]
        return c[0] + t * (c[1] + t * (c[2] + t * c[3]))

    def piece_slope(self, i, q):
        c = self.coef[i]
        t = Fraction(float(q)) - self.X[i]
        return c[1] + t * (2 * c[2] + 3 * t * c[3])
