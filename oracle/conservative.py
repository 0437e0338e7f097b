"""Conservative (face-averaged) variable-coefficient diffusion, its transpose
and the coefficient gradient (part of the oracle; TEST INFRASTRUCTURE ONLY,
see the package header).

The operator is the per-cell-coefficient stencil of the paper's model
(Sec. III-A: u_{t+1}[p] = sum_k w_k(p) u_t[p + o_k], two arrays swapped each
step) written in flux form, so that whatever the coefficient field the sum of
u is conserved on a periodic grid:

    u'[p] = u[p] + sum over the 2 * ndim axis neighbours q of p of
                   k_pq * (u[q] - u[p]),
    k_pq  = (kappa[p] + kappa[q]) / 2   for an interior (or wrapped) q,
    k_pq  = kappa[p]                    for a Dirichlet ghost q (u[q] = bc).

Plain numpy, float64: shifted views of padded arrays (u padded with the
boundary value or wrapped, kappa padded with its edge values, which makes a
ghost face's coefficient (kappa[p] + kappa[p]) / 2 = kappa[p]); the
neighbours are taken in the order -z, +z, -y, +y, -x, +x (2D: -y, +y, -x,
+x), each term a multiply then an add.

The transpose and the gradient are written as scatters (every row p sends
its face terms to the points they touch), a different formulation from the
forward gather, with every state of the forward run kept.
"""
from __future__ import annotations

import numpy as np


def _dirs(nd):
    out = []
    for ax in range(nd):
        for s in (-1, 1):
            o = [0] * nd
            o[ax] = s
            out.append(tuple(o))
    return out


def _pad(a, periodic, value=None):
    if periodic:
        return np.pad(a, 1, mode="wrap")
    if value is None:
        return np.pad(a, 1, mode="edge")
    return np.pad(a, 1, mode="constant", constant_values=value)


def _shift(padded, o, shape):
    return padded[tuple(slice(1 + c, 1 + c + n) for c, n in zip(o, shape))]


def cons_step(u, kappa, periodic: bool, bc_value: float):
    """One step of the conservative operator on a dense interior."""
    u = np.asarray(u, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    up, kp = _pad(u, periodic, bc_value), _pad(kappa, periodic)
    acc = np.zeros_like(u)
    for o in _dirs(u.ndim):
        w = (kappa + _shift(kp, o, u.shape)) / 2
        acc = acc + w * (_shift(up, o, u.shape) - u)
    return u + acc


def cons_forward(u0, kappa, periodic: bool, bc_value: float, nsteps: int, keep=False):
    u = np.array(u0, dtype=np.float64)
    states = [u]
    for _ in range(int(nsteps)):
        u = cons_step(u, kappa, periodic, bc_value)
        if keep:
            states.append(u)
    return states if keep else u


def _interior_mask(shape, o, periodic):
    """True where p + o is an interior (or wrapped) point."""
    m = np.ones(shape, dtype=bool)
    if periodic:
        return m
    for ax, c in enumerate(o):
        if c < 0:
            idx = [slice(None)] * len(shape)
            idx[ax] = slice(0, -c)
            m[tuple(idx)] = False
        elif c > 0:
            idx = [slice(None)] * len(shape)
            idx[ax] = slice(shape[ax] - c, shape[ax])
            m[tuple(idx)] = False
    return m


def _scatter_add(dst, vals, o, periodic):
    """dst[p + o] += vals[p] for every p whose p + o is interior (wrapped)."""
    if periodic:
        dst += np.roll(vals, shift=o, axis=tuple(range(dst.ndim)))
        return
    src = tuple(slice(max(0, -c), n - max(0, c)) for c, n in zip(o, dst.shape))
    tgt = tuple(slice(max(0, c), n - max(0, -c)) for c, n in zip(o, dst.shape))
    dst[tgt] += vals[src]


def cons_transpose(lam, kappa, periodic: bool):
    """S^T lam by scatter: row p of S is u[p] (1 - sum_q k_pq) + sum over
    interior q of k_pq u[q] (ghost values are constants, not variables)."""
    lam = np.asarray(lam, dtype=np.float64)
    kappa = np.asarray(kappa, dtype=np.float64)
    kp = _pad(kappa, periodic)
    out = lam.copy()
    for o in _dirs(lam.ndim):
        w = (kappa + _shift(kp, o, lam.shape)) / 2
        out -= w * lam                                     # row p, its own column
        inner = _interior_mask(lam.shape, o, periodic)
        _scatter_add(out, np.where(inner, w * lam, 0.0), o, periodic)   # row p, column q
    return out


def cons_gradient_step(u, lam_next, kappa, periodic: bool, bc_value: float):
    """d/dkappa of lam_next . (S u + b) by scatter: row p's face term
    k_pq (u[q] - u[p]) weighted by lam_next[p] sends dk_pq/dkappa_p to p and
    dk_pq/dkappa_q to q (1/2 each for an interior q; 1 to p for a ghost q)."""
    u = np.asarray(u, dtype=np.float64)
    lam = np.asarray(lam_next, dtype=np.float64)
    up = _pad(u, periodic, bc_value)
    g = np.zeros_like(u)
    for o in _dirs(u.ndim):
        inner = _interior_mask(u.shape, o, periodic)
        t = lam * (_shift(up, o, u.shape) - u)             # lam_p (u_q - u_p)
        g += np.where(inner, 0.5 * t, t)                   # dk_pq / dkappa_p
        _scatter_add(g, np.where(inner, 0.5 * t, 0.0), o, periodic)   # dk_pq / dkappa_q
    return g


def cons_loss_gradient(u0, kappa, target, periodic: bool, bc_value: float, nsteps: int):
    """L = 0.5 ||u_T - target||^2: returns (L, u_T, dL/du0, dL/dkappa)."""
    states = cons_forward(u0, kappa, periodic, bc_value, nsteps, keep=True)
    uT = states[-1]
    r = uT - np.asarray(target, dtype=np.float64)
    loss = 0.5 * float(np.sum(r * r))
    lam = r
    g = np.zeros_like(uT)
    for t in range(int(nsteps) - 1, -1, -1):
        g += cons_gradient_step(states[t], lam, kappa, periodic, bc_value)
        lam = cons_transpose(lam, kappa, periodic)
    return loss, uT, lam, g
