"""Central finite-difference coefficients for the second derivative, derived
exactly from the Taylor conditions (part of the oracle; test infrastructure).

For a symmetric stencil f''(0) h^2 ~ a_0 f(0) + sum_{j=1..r} a_j (f(jh) + f(-jh)),
expanding f(+-jh) in Taylor series gives, for the even powers 2q (q = 0..r):

    q = 0:  a_0 + 2 sum_j a_j          = 0
    q = 1:  2 sum_j a_j j^2 / 2!       = 1
    q > 1:  2 sum_j a_j j^(2q) / (2q)! = 0

r + 1 linear equations in r + 1 unknowns, solved here by Gaussian elimination
over the rationals, so the result is exact.  For r = 4 this is the 8th-order
star stencil of the acoustic wave configuration.
"""
from __future__ import annotations

from fractions import Fraction
from math import factorial


def taylor_second_derivative_coeffs(radius: int = 4) -> list[Fraction]:
    r = int(radius)
    if r < 1:
        raise ValueError("radius >= 1")
    n = r + 1
    # rows: q = 0..r ; columns: a_0..a_r
    rows = []
    for q in range(n):
        row = [Fraction(0)] * n
        if q == 0:
            row[0] = Fraction(1)
        for j in range(1, n):
            row[j] = Fraction(2 * j ** (2 * q), factorial(2 * q))
        rhs = Fraction(1) if q == 1 else Fraction(0)
        rows.append(row + [rhs])
    # Gaussian elimination with exact arithmetic
    for c in range(n):
        piv = next(i for i in range(c, n) if rows[i][c] != 0)
        rows[c], rows[piv] = rows[piv], rows[c]
        pv = rows[c][c]
        rows[c] = [v / pv for v in rows[c]]
        for i in range(n):
            if i != c and rows[i][c] != 0:
                f = rows[i][c]
                rows[i] = [vi - f * vc for vi, vc in zip(rows[i], rows[c])]
    return [rows[i][n] for i in range(n)]
