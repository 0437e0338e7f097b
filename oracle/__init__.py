"""Plain CPU oracle for the stencil sweeps of "An Adaptive Distributed Stencil
Abstraction for GPUs" (CharmStencil).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2512_19851_gb300``) never imports, links or runs it, and the two share
no code: the oracle is plain C loops (``stencil_oracle.c``) evaluated in double
precision, in a stated summation order, with ``-ffp-contract=off``.

Conventions: arrays are dense interiors (no ghost cells), C order, shape
``(nz, ny, nx)`` in 3D or ``(ny, nx)`` in 2D; a neighbour offset is
``(dz, dy, dx)`` (or ``(dy, dx)`` in 2D).  Points outside the interior read the
Dirichlet value or wrap (periodic).

Functions and the passage each follows:

* :func:`sweep_const` -- u_{t+1}[p] = sum_k w_k u_t[p+o_k], two arrays swapped
  each step (Example 1 and the dependency rule of Sec. III-A; boundary ring set
  once and held, Example 1).
* :func:`varcoef7_forward` / :func:`varcoef7_adjoint` -- per-cell-coefficient
  7-point diffusion and its transpose with the coefficient gradient; the
  checkpoint-every-m recomputation is :func:`varcoef7_gradient`.
* :func:`wave25` -- radius-4 star Laplacian in a leapfrog update.
* :func:`reduce` -- sum, sum of squares and max-abs in double precision.
* :func:`sweep_ghosts` (in :mod:`oracle.ghosts`) -- the sweep of
  :func:`sweep_const` on a padded array whose Dirichlet ring holds arbitrary
  per-cell values (Example 1's boundary ring set by slice assignment, Sec.
  III-A), plain numpy; :func:`sweep_neumann` the same update with a
  zero-flux boundary (mirror-image ghosts refreshed before every step, the
  ghost exchange of Sec. III-C on one domain); :func:`neumann_transpose` its
  transpose by scatter and :func:`neumann_loss_gradient` the gradient of a
  loss of the last state with respect to the first.
* :func:`cons_forward`, :func:`cons_transpose`, :func:`cons_loss_gradient`
  (in :mod:`oracle.conservative`) -- the per-cell diffusion in conservative
  face-averaged form, its transpose and the coefficient gradient, plain
  numpy (forward by gather, transpose and gradient by scatter).
* :mod:`oracle.cavity` -- the lid-driven cavity flow (pressure source,
  Jacobi pressure iterations with their boundary rule, momentum updates),
  the paper's multi-field benchmark (Sec. V-B), plain numpy.
* :func:`taylor_second_derivative_coeffs` (in :mod:`oracle.taylor`) -- the
  8th-order central coefficients from the Taylor conditions.

Parity pins for every function live in ``tests/test_oracle_pins.py``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

from .conservative import cons_forward, cons_loss_gradient, cons_step, cons_transpose  # noqa: F401
from .ghosts import neumann_loss_gradient, neumann_transpose, sweep_ghosts, sweep_neumann  # noqa: F401
from .taylor import taylor_second_derivative_coeffs  # noqa: F401

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "stencil_oracle.c")
_LIBS = {np.float64: os.path.join(_HERE, "_oracle_f64.so"),
         np.float32: os.path.join(_HERE, "_oracle_f32.so")}
_SUFFIX = {np.float64: "_f64", np.float32: "_f32"}
_CTYPE = {np.float64: "double", np.float32: "float"}
_loaded: dict = {}


def build(force: bool = False) -> None:
    """Compile the oracle twice (double and single precision) with gcc."""
    for dt, path in _LIBS.items():
        if (not force and os.path.exists(path)
                and os.path.getmtime(path) >= os.path.getmtime(_SRC)):
            continue
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
               "-fPIC", "-shared", f"-DREAL={_CTYPE[dt]}", f"-DORC_SUFFIX={_SUFFIX[dt]}",
               _SRC, "-o", path + ".tmp"]
        subprocess.check_call(cmd)
        os.replace(path + ".tmp", path)


def _lib(dt):
    dt = np.dtype(dt).type
    if dt not in _loaded:
        build()
        _loaded[dt] = ctypes.CDLL(_LIBS[dt])
    return _loaded[dt]


def default_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _shape3(shape):
    if len(shape) == 3:
        return tuple(int(s) for s in shape)
    if len(shape) == 2:
        return (1, int(shape[0]), int(shape[1]))
    if len(shape) == 1:
        return (1, 1, int(shape[0]))
    raise ValueError("1D, 2D or 3D grids only")


def _off3(offsets, ndim):
    off = np.asarray(offsets, dtype=np.int32).reshape(-1, ndim)
    pad = np.zeros((off.shape[0], 3 - ndim), dtype=np.int32)
    return np.ascontiguousarray(np.concatenate([pad, off], axis=1))


def _fn(dt, name, restype=None):
    f = getattr(_lib(dt), name + _SUFFIX[np.dtype(dt).type])
    f.restype = restype
    return f


I64, INT, DBL, VP = ctypes.c_int64, ctypes.c_int, ctypes.c_double, ctypes.c_void_p


def sweep_const(u0, offsets, weights, periodic: bool, bc_value: float, nsteps: int,
                dtype=np.float64, threads: int | None = None):
    """Run ``nsteps`` constant-weight sweeps from ``u0``; returns u_nsteps."""
    dt = np.dtype(dtype).type
    u = np.ascontiguousarray(u0, dtype=dt).copy()
    tmp = np.empty_like(u)
    nz, ny, nx = _shape3(u.shape)
    off = _off3(offsets, u.ndim)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if w.shape[0] != off.shape[0] or off.shape[0] > 64:
        raise ValueError("one weight per offset, at most 64 points")
    f = _fn(dt, "orc_sweep_const")
    f.argtypes = [I64, I64, I64, INT, VP, VP, INT, DBL, INT, VP, VP, INT]
    f(nz, ny, nx, off.shape[0], _ptr(off), _ptr(w), int(bool(periodic)), float(bc_value),
      int(nsteps), _ptr(u), _ptr(tmp), int(threads or default_threads()))
    return u


def sweep_const_into(u, tmp, offsets, weights, periodic: bool, bc_value: float, nsteps: int,
                     threads: int | None = None):
    """:func:`sweep_const` on caller-owned arrays, for timing the oracle on a
    resident field: ``u`` (C-contiguous float64 or float32) holds u_0 on entry
    and u_nsteps on return, ``tmp`` (same shape and dtype) is scratch.  The
    arithmetic is the same C loop; only the copies of the wrapper are left
    out (an even nsteps also skips the C loop's final copy)."""
    if not (u.flags.c_contiguous and tmp.flags.c_contiguous) or u.dtype != tmp.dtype or u.shape != tmp.shape:
        raise ValueError("u and tmp: C-contiguous arrays of one shape and dtype")
    dt = u.dtype.type
    nz, ny, nx = _shape3(u.shape)
    off = _off3(offsets, u.ndim)
    w = np.ascontiguousarray(weights, dtype=np.float64)
    if w.shape[0] != off.shape[0] or off.shape[0] > 64:
        raise ValueError("one weight per offset, at most 64 points")
    f = _fn(dt, "orc_sweep_const")
    f.argtypes = [I64, I64, I64, INT, VP, VP, INT, DBL, INT, VP, VP, INT]
    f(nz, ny, nx, off.shape[0], _ptr(off), _ptr(w), int(bool(periodic)), float(bc_value),
      int(nsteps), _ptr(u), _ptr(tmp), int(threads or default_threads()))
    return u


def varcoef7_forward(u0, kappa, periodic: bool, bc_value: float, nsteps: int,
                     store_states: bool = False, dtype=np.float64, threads: int | None = None):
    """Per-cell 7-point diffusion; returns u_nsteps (and u_0..u_nsteps if asked)."""
    dt = np.dtype(dtype).type
    u = np.ascontiguousarray(u0, dtype=dt).copy()
    k = np.ascontiguousarray(kappa, dtype=dt)
    tmp = np.empty_like(u)
    nz, ny, nx = _shape3(u.shape)
    states = np.empty((nsteps + 1,) + u.shape, dtype=dt) if store_states else None
    f = _fn(dt, "orc_varcoef7")
    f.argtypes = [I64, I64, I64, VP, INT, DBL, INT, VP, VP, VP, INT]
    f(nz, ny, nx, _ptr(k), int(bool(periodic)), float(bc_value), int(nsteps), _ptr(u),
      _ptr(tmp), _ptr(states), int(threads or default_threads()))
    return (u, states) if store_states else u


def varcoef7_adjoint(states, kappa, lam_T, periodic: bool, bc_value: float,
                     gk=None, dtype=np.float64, threads: int | None = None):
    """Transpose sweep over ``len(states)`` steps (states = u_0 .. u_{S-1}).

    Returns (lambda_0, gk) with gk += sum_t lambda_{t+1} * du_{t+1}/dkappa.
    """
    dt = np.dtype(dtype).type
    st = np.ascontiguousarray(states, dtype=dt)
    nsteps = st.shape[0]
    lam = np.ascontiguousarray(lam_T, dtype=dt).copy()
    k = np.ascontiguousarray(kappa, dtype=dt)
    tmp = np.empty_like(lam)
    g = np.zeros_like(lam) if gk is None else np.ascontiguousarray(gk, dtype=dt)
    nz, ny, nx = _shape3(lam.shape)
    f = _fn(dt, "orc_varcoef7_adjoint")
    f.argtypes = [I64, I64, I64, VP, INT, DBL, INT, VP, VP, VP, VP, INT]
    f(nz, ny, nx, _ptr(k), int(bool(periodic)), float(bc_value), int(nsteps), _ptr(st),
      _ptr(lam), _ptr(tmp), _ptr(g), int(threads or default_threads()))
    return lam, g


def varcoef7_gradient(u0, kappa, u_target, periodic: bool, bc_value: float, nsteps: int,
                      ckpt_every: int, threads: int | None = None):
    """Loss 0.5*||u_S - u_target||^2 and its gradients (d/du_0, d/dkappa).

    Checkpoint-every-m recomputation: the forward keeps u_0, u_m, u_2m, ...;
    the reverse pass recomputes each segment's states from its checkpoint and
    runs the transpose sweep over that segment.  ``ckpt_every = nsteps`` is
    the store-everything special case.  Everything in double precision.
    """
    m = int(ckpt_every)
    if m < 1:
        raise ValueError("ckpt_every >= 1")
    u = np.ascontiguousarray(u0, dtype=np.float64)
    k = np.ascontiguousarray(kappa, dtype=np.float64)
    ckpts = {}
    t = 0
    while t < nsteps:
        ckpts[t] = u.copy()
        seg = min(m, nsteps - t)
        u = varcoef7_forward(u, k, periodic, bc_value, seg, threads=threads)
        t += seg
    uT = u
    diff = uT - np.asarray(u_target, dtype=np.float64)
    loss = 0.5 * reduce(uT, u_target)[1]
    lam = diff
    gk = np.zeros_like(k)
    for t0 in sorted(ckpts.keys(), reverse=True):
        seg = min(m, nsteps - t0)
        _, states = varcoef7_forward(ckpts[t0], k, periodic, bc_value, seg, store_states=True,
                                     threads=threads)
        lam, gk = varcoef7_adjoint(states[:seg], k, lam, periodic, bc_value, gk=gk,
                                   threads=threads)
    return loss, uT, lam, gk


def wave25(u_n, u_nm1, m, a, src_index, src_amps, periodic: bool, bc_value: float,
           nsteps: int, dtype=np.float64, threads: int | None = None):
    """Leapfrog radius-4 star update; returns (u^nsteps, u^{nsteps-1})."""
    dt = np.dtype(dtype).type
    un = np.ascontiguousarray(u_n, dtype=dt).copy()
    unm1 = np.ascontiguousarray(u_nm1, dtype=dt).copy()
    mm = np.ascontiguousarray(m, dtype=dt)
    nz, ny, nx = _shape3(un.shape)
    aa = np.ascontiguousarray(a, dtype=np.float64)
    if aa.shape != (5,):
        raise ValueError("five coefficients a_0..a_4")
    if src_index is None:
        src = -1
        s = np.zeros(max(nsteps, 1), dtype=np.float64)
    else:
        src = int(np.ravel_multi_index(tuple(int(i) for i in src_index), un.shape))
        s = np.ascontiguousarray(src_amps, dtype=np.float64)
        if s.shape[0] < nsteps:
            raise ValueError("one source amplitude per step")
    f = _fn(dt, "orc_wave25")
    f.argtypes = [I64, I64, I64, VP, VP, INT, DBL, I64, VP, INT, VP, VP, INT]
    f(nz, ny, nx, _ptr(aa), _ptr(mm), int(bool(periodic)), float(bc_value), src, _ptr(s),
      int(nsteps), _ptr(un), _ptr(unm1), int(threads or default_threads()))
    return un, unm1


def reduce(a, b=None):
    """(sum(a-b), sum((a-b)^2), max|a-b|) accumulated in double, index order."""
    aa = np.ascontiguousarray(a)
    dt = np.float32 if aa.dtype == np.float32 else np.float64
    aa = np.ascontiguousarray(aa, dtype=dt).reshape(-1)
    bb = None if b is None else np.ascontiguousarray(b, dtype=dt).reshape(-1)
    out = np.zeros(3, dtype=np.float64)
    f = _fn(dt, "orc_reduce")
    f.argtypes = [I64, VP, VP, VP]
    f(aa.shape[0], _ptr(aa), _ptr(bb), _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def normwise_error(x, ref) -> float:
    """max|x - ref| / max|ref| (the error metric used for every parity check)."""
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref)))
    num = float(np.max(np.abs(x - ref)))
    return num / den if den > 0 else num


if __name__ == "__main__":  # pragma: no cover
    build(force="--force" in sys.argv)
