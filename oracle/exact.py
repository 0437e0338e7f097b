"""Exact rational evaluation of a constant-weight stencil sweep on tiny grids
(part of the oracle; test infrastructure).

Used only to write golden fixtures: with dyadic weights and boundary values
(Example 1 of Sec. III-A uses weight 1/4 and boundary 1) every intermediate is
a dyadic rational, so a double-precision evaluation must reproduce these
values exactly.  Pure-Python loops over ``fractions.Fraction``.
"""
from __future__ import annotations

from fractions import Fraction


def sweep_exact_2d(u0, offsets, weights, bc_value, nsteps: int, periodic: bool = False):
    ny = len(u0)
    nx = len(u0[0])
    u = [[Fraction(v) for v in row] for row in u0]
    w = [Fraction(v) for v in weights]
    bc = Fraction(bc_value)
    for _ in range(nsteps):
        new = [[Fraction(0)] * nx for _ in range(ny)]
        for y in range(ny):
            for x in range(nx):
                acc = Fraction(0)
                for (dy, dx), wk in zip(offsets, w):
                    yy, xx = y + dy, x + dx
                    if periodic:
                        v = u[yy % ny][xx % nx]
                    elif 0 <= yy < ny and 0 <= xx < nx:
                        v = u[yy][xx]
                    else:
                        v = bc
                    acc += wk * v
                new[y][x] = acc
        u = new
    return u
