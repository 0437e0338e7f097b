"""Lid-driven cavity flow (incompressible Navier-Stokes) on a uniform 2D grid
(part of the oracle; TEST INFRASTRUCTURE ONLY, see the package header).

The paper's second benchmark (Sec. V-B) runs a cavity-flow solver written as
NumPy slice assignments on several arrays per step.  This is the standard
explicit projection-style scheme for the square cavity with a moving lid,
written from the equations

    du/dt + u du/dx + v du/dy = -(1/rho) dp/dx + nu (d2u/dx2 + d2u/dy2)
    dv/dt + u dv/dx + v dv/dy = -(1/rho) dp/dy + nu (d2v/dx2 + d2v/dy2)
    d2p/dx2 + d2p/dy2 = -rho (ux^2 + 2 uy vx + vy^2) + (rho/dt)(ux + vy)

on arrays of shape (ny, nx) that include their boundary rows and columns
(y along axis 0, x along axis 1, spacings dy and dx).  Per time step:

1. the pressure source at interior points, central differences
   b = rho * ((ux + vy) / dt - ux^2 - 2 uy vx - vy^2),
   ux = (u[j, i+1] - u[j, i-1]) / (2 dx), uy = (u[j+1, i] - u[j-1, i]) / (2 dy),
   vx, vy likewise;
2. nit Jacobi iterations of the pressure Poisson equation on the interior,
   p[j, i] = ((p[j, i+1] + p[j, i-1]) dy^2 + (p[j+1, i] + p[j-1, i]) dx^2
              - b dx^2 dy^2) / (2 (dx^2 + dy^2)),
   each followed by the boundary rule, applied in this order: right column
   copies its left neighbour, bottom row copies the row above, left column
   copies its right neighbour, top row (the lid) is set to 0;
3. the velocities at interior points from the previous step's u, v and the
   new p: backward (upwind for positive velocities) differences for
   advection, central differences for the pressure gradient and the
   diffusion,
   u' = u - u dt/dx (u - u[j, i-1]) - v dt/dy (u - u[j-1, i])
          - dt / (2 rho dx) (p[j, i+1] - p[j, i-1])
          + nu (dt/dx^2 (u[j, i+1] - 2u + u[j, i-1]) + dt/dy^2 (u[j+1, i] - 2u + u[j-1, i])),
   v' likewise with - dt / (2 rho dy) (p[j+1, i] - p[j-1, i]);
   then u = 0 on the bottom, left and right walls and u = lid on the top
   row, v = 0 on all four walls.

Plain numpy, float64: each formula evaluated on shifted interior views in
the order written above.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass(frozen=True)
class CavityParams:
    dx: float
    dy: float
    dt: float
    rho: float = 1.0
    nu: float = 0.1
    nit: int = 50
    lid: float = 1.0


def _views(a):
    """Interior view and its four neighbours: (centre, east, west, north, south)
    with east = +x (axis 1), north = +y (axis 0)."""
    return a[1:-1, 1:-1], a[1:-1, 2:], a[1:-1, :-2], a[2:, 1:-1], a[:-2, 1:-1]


def pressure_source(u, v, P: CavityParams):
    b = np.zeros_like(u)
    _, ue, uw, un, us = _views(u)
    _, ve, vw, vn, vs = _views(v)
    ux = (ue - uw) / (2 * P.dx)
    uy = (un - us) / (2 * P.dy)
    vx = (ve - vw) / (2 * P.dx)
    vy = (vn - vs) / (2 * P.dy)
    b[1:-1, 1:-1] = P.rho * ((ux + vy) / P.dt - ux * ux - 2 * uy * vx - vy * vy)
    return b


def pressure_boundary(p):
    p[:, -1] = p[:, -2]
    p[0, :] = p[1, :]
    p[:, 0] = p[:, 1]
    p[-1, :] = 0.0


def pressure_iterations(p, b, P: CavityParams, nit=None):
    p = np.array(p, copy=True)
    dx2, dy2 = P.dx * P.dx, P.dy * P.dy
    for _ in range(P.nit if nit is None else nit):
        pn = p.copy()
        _, pe, pw, pnn, ps = _views(pn)
        p[1:-1, 1:-1] = ((pe + pw) * dy2 + (pnn + ps) * dx2 - b[1:-1, 1:-1] * dx2 * dy2) / (2 * (dx2 + dy2))
        pressure_boundary(p)
    return p


def velocity_update(u, v, p, P: CavityParams):
    un, vn = u.copy(), v.copy()
    uc, ue, uw, unn, us = _views(un)
    vc, ve, vw, vnn, vs = _views(vn)
    _, pe, pw, pnn, ps = _views(p)
    cx, cy = P.dt / P.dx, P.dt / P.dy
    dxx, dyy = P.dt / (P.dx * P.dx), P.dt / (P.dy * P.dy)
    u2 = u.copy()
    v2 = v.copy()
    u2[1:-1, 1:-1] = (uc - uc * cx * (uc - uw) - vc * cy * (uc - us)
                      - P.dt / (2 * P.rho * P.dx) * (pe - pw)
                      + P.nu * (dxx * (ue - 2 * uc + uw) + dyy * (unn - 2 * uc + us)))
    v2[1:-1, 1:-1] = (vc - uc * cx * (vc - vw) - vc * cy * (vc - vs)
                      - P.dt / (2 * P.rho * P.dy) * (pnn - ps)
                      + P.nu * (dxx * (ve - 2 * vc + vw) + dyy * (vnn - 2 * vc + vs)))
    u2[0, :] = 0.0
    u2[:, 0] = 0.0
    u2[:, -1] = 0.0
    u2[-1, :] = P.lid
    v2[0, :] = 0.0
    v2[-1, :] = 0.0
    v2[:, 0] = 0.0
    v2[:, -1] = 0.0
    return u2, v2


def cavity_run(u0, v0, p0, P: CavityParams, nsteps: int, dtype=np.float64):
    """nsteps time steps from (u0, v0, p0); returns (u, v, p).  dtype=float32
    evaluates the same expressions in single precision (the parameters act as
    weak Python scalars), to measure the drift inherent to FP32."""
    u = np.array(u0, dtype=dtype, copy=True)
    v = np.array(v0, dtype=dtype, copy=True)
    p = np.array(p0, dtype=dtype, copy=True)
    for _ in range(int(nsteps)):
        b = pressure_source(u, v, P)
        p = pressure_iterations(p, b, P)
        u, v = velocity_update(u, v, p, P)
    return u, v, p
