"""Stencil descriptions of the workloads in the affine-weight form of the C ABI,
w_k(p) = alpha_k + beta_k * kappa[p]  (beta = None: constant weights).

Offsets are in C order, (dy, dx) in 2D and (dz, dy, dx) in 3D, in the orders
given by paper_2512_19851_gb300.inputs.
"""
from __future__ import annotations

from fractions import Fraction

from .inputs import OFFSETS_5PT, OFFSETS_7PT, OFFSETS_BOX9

# 8th-order central second-derivative coefficients a_0..a_4 (radius 4):
# f''(0) h^2 ~ a_0 f(0) + sum_j a_j (f(jh) + f(-jh)).
STAR8_COEFFS = (Fraction(-205, 72), Fraction(8, 5), Fraction(-1, 5), Fraction(8, 315), Fraction(-1, 560))


def heat2d(a: float = 0.2):
    """u + a (N + S + E + W - 4u): the 2D 5-point Jacobi heat step."""
    return OFFSETS_5PT, [1.0 - 4.0 * a, a, a, a, a], None


def heat3d(alpha: float = 0.1):
    """u + alpha (sum of 6 neighbours - 6u): the 3D 7-point heat step."""
    return OFFSETS_7PT, [1.0 - 6.0 * alpha] + [alpha] * 6, None


def varcoef7():
    """(1 - 6 kappa_p) u + kappa_p (sum of 6 neighbours): per-cell diffusivity."""
    return OFFSETS_7PT, [1.0] + [0.0] * 6, [-6.0] + [1.0] * 6


def box9(weights):
    """3x3 box with the given nine weights (row-major over (dy, dx))."""
    return OFFSETS_BOX9, [float(w) for w in weights], None


def star8_offsets():
    offs = [(0, 0, 0)]
    for ax in range(3):
        for j in range(1, 5):
            for sgn in (1, -1):
                o = [0, 0, 0]
                o[ax] = sgn * j
                offs.append(tuple(o))
    return offs


def wave25():
    """Leapfrog radius-4 star: u^{n+1} = 2u^n - u^{n-1} + m_p L8 u^n (+ source),
    as w_k(p) = alpha_k + beta_k m_p with alpha = 2 at the centre and beta the
    star coefficients (3 a_0 at the centre: one a_0 per axis)."""
    a = [float(c) for c in STAR8_COEFFS]
    offs = star8_offsets()
    alpha = [2.0] + [0.0] * 24
    beta = [3.0 * a[0]]
    for _ax in range(3):
        for j in range(1, 5):
            beta += [a[j], a[j]]
    return offs, alpha, beta
