"""Constant-weight sweeps with arbitrary Dirichlet ghost values and with a
zero-flux (Neumann) boundary, and the transpose of the zero-flux sweep (part
of the oracle; TEST INFRASTRUCTURE ONLY, see the package header).

Example 1 of Sec. III-A sets the boundary ring of both arrays once by slice
assignment and never writes it again; the update reads the ring wherever a
neighbour falls outside the interior.  The ring may hold any values (one per
cell), not only one constant.  This module evaluates that definition
literally on a padded array:

    for every interior p:  out[p] = sum_k w_k * in[p + o_k]   (offset order)

with ``in`` and ``out`` both padded by r cells on every side, the ring copied
unchanged from step to step, and the two arrays swapped after each step
(Sec. III-A's ``u1, u2 = u2, u1``).  Plain numpy: for each offset the shifted
interior view of ``in`` is multiplied by w_k and added to the accumulator in
offset order (a multiply, then an add: no fused multiply-add), which is the
order the C oracle uses.  Float64 unless ``dtype`` says otherwise.
"""
from __future__ import annotations

import numpy as np


def sweep_ghosts(u_padded, radius: int, offsets, weights, nsteps: int, dtype=np.float64):
    """Run ``nsteps`` sweeps on a padded array (interior plus ``radius`` ghost
    cells per side on every axis); returns the padded array after the last
    step (ring unchanged)."""
    r = int(radius)
    u = np.array(u_padded, dtype=dtype, copy=True)
    nd = u.ndim
    offs = [tuple(int(c) for c in o) for o in offsets]
    if any(len(o) != nd for o in offs):
        raise ValueError("one offset component per axis")
    if any(abs(c) > r for o in offs for c in o):
        raise ValueError("an offset reaches beyond the ghost ring")
    w = [dtype(x) for x in weights]
    if len(w) != len(offs):
        raise ValueError("one weight per offset")
    n = [s - 2 * r for s in u.shape]
    if min(n) < 1:
        raise ValueError("empty interior")
    inner = tuple(slice(r, r + m) for m in n)
    tmp = u.copy()
    for _ in range(int(nsteps)):
        tmp[inner] = _sweep_once(u, r, offs, w, n, dtype)
        u, tmp = tmp, u
        # the ring of the array that now holds the older level is still the
        # initial ring (sweeps write interiors only)
    return u


def _sweep_once(u, r, offs, w, n, dtype):
    """The new interior from the padded array u (offset order, multiply then add)."""
    acc = np.zeros(n, dtype=dtype)
    for o, wk in zip(offs, w):
        src = tuple(slice(r + c, r + c + m) for c, m in zip(o, n))
        acc = acc + wk * u[src]
    return acc


def sweep_neumann(u0, offsets, weights, nsteps: int, dtype=np.float64):
    """Zero-flux (Neumann) boundary: before every sweep the ghost ring of
    the input is its mirror image across each boundary face (cell-centred
    reflection: index -1 - i for i < 0, 2n - 1 - i for i >= n, per axis),
    which numpy's symmetric padding is; then the sweep of sweep_ghosts.
    Takes and returns the dense interior."""
    offs = [tuple(int(c) for c in o) for o in offsets]
    r = max(abs(c) for o in offs for c in o)
    u = np.array(u0, dtype=dtype, copy=True)
    if r > min(u.shape):
        raise ValueError("a mirror image must be interior (extent >= radius)")
    w = [dtype(x) for x in weights]
    for _ in range(int(nsteps)):
        u = _sweep_once(np.pad(u, r, mode="symmetric"), r, offs, w, list(u.shape), dtype)
    return u


def _mirror_index(i, n):
    """Cell-centred reflection of index array i into [0, n): -1 - i below,
    2n - 1 - i above (the zero-flux ghost rule, for i within n of the edge)."""
    return np.where(i < 0, -1 - i, np.where(i >= n, 2 * n - 1 - i, i))


def neumann_transpose(lam, offsets, weights, dtype=np.float64):
    """Transpose of one zero-flux sweep, by scatter: the sweep reads, for
    every interior p and offset k, the cell mirror(p + o_k) with weight w_k,
    so its transpose sends w_k * lam[p] to that cell.  Plain numpy: for each
    offset (in order) the mirrored target index of every p is formed and
    the products are added there (np.add.at, which accumulates repeated
    targets)."""
    lam = np.asarray(lam, dtype=dtype)
    offs = [tuple(int(c) for c in o) for o in offsets]
    if any(len(o) != lam.ndim for o in offs):
        raise ValueError("one offset component per axis")
    r = max(abs(c) for o in offs for c in o)
    if r > min(lam.shape):
        raise ValueError("a mirror image must be interior (extent >= radius)")
    idx = np.indices(lam.shape)
    out = np.zeros_like(lam)
    for o, wk in zip(offs, weights):
        tgt = tuple(_mirror_index(idx[a] + o[a], lam.shape[a]) for a in range(lam.ndim))
        np.add.at(out, tgt, dtype(wk) * lam)
    return out


def neumann_loss_gradient(u0, target, offsets, weights, nsteps: int):
    """L = 0.5 ||u_n - target||^2 for n zero-flux sweeps from u0, and
    dL/du0 = (S^T)^n (u_n - target), in double precision."""
    un = sweep_neumann(u0, offsets, weights, nsteps)
    d = un - np.asarray(target, dtype=np.float64)
    lam = d
    for _ in range(int(nsteps)):
        lam = neumann_transpose(lam, offsets, weights)
    return 0.5 * float(np.sum(d * d)), un, lam
