"""Seeded synthetic inputs for the five stencil workloads.

This module only draws and lays out input data (initial fields, coefficient
fields, source time series, grid sizes).  It holds none of the stencil
arithmetic, imports neither the CUDA library nor the oracle, and is the one
piece of code both the GPU path and the CPU oracle are fed from.

All arrays are dense interiors in C order, float64 unless stated; the GPU
path casts them to its own storage type.  The recipes follow the workload
descriptions (Laplace/Jacobi, Example 1 of Sec. III-A, and the four derived
configurations), with the seeds and draw orders fixed here:

* heat2d      -- u0 ~ U[0,1) over the 256x256 interior, default_rng(0).
* heat3d      -- 8 product-of-sines modes, integer wavenumbers 1..16 per axis,
                 amplitudes U[0,1), plus N(0, 0.01) noise; default_rng(1),
                 drawn in the order wavenumbers, amplitudes, noise.
* wave3d      -- 8 equal-thickness layers along z, velocity U[1.5, 4.5) per
                 layer (default_rng(2)); h = 1/n, dt = 0.4 h / max(c);
                 per-cell factor m = (c dt / h)^2; Ricker source
                 r(t) = (1 - 2 pi^2 f^2 (t-t0)^2) exp(-pi^2 f^2 (t-t0)^2),
                 f = 15, t0 = 1/f, amplitude dt^2 r(n dt) at the centre cell.
* varcoef3d   -- u0 ~ U[0,1) then kappa = clip(0.05 exp(0.5 Z), 0, 0.16),
                 Z ~ N(0,1) (default_rng(3)); target ~ U[0,1) (default_rng(5)).
* batch2d     -- 512 grids, ny then nx drawn as round(exp(U(ln 64, ln 2048)))
                 (default_rng(4)), then 9 weights U[0,1) per grid normalised to
                 sum 1, then u0 ~ U[0,1) grid by grid.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# Neighbour offsets in the orders the workloads use.  (dy, dx) in 2D,
# (dz, dy, dx) in 3D.  These are input descriptions, shared by both sides.
OFFSETS_5PT = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
OFFSETS_7PT = [(0, 0, 0), (0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
OFFSETS_BOX9 = [(dy, dx) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def heat2d(n: int = 256, seed: int = 0, shape=None) -> np.ndarray:
    """Initial field of the 2D Jacobi heat workload: U[0,1) interior."""
    shp = tuple(shape) if shape is not None else (n, n)
    return np.random.default_rng(seed).random(shp)


def _sine_modes_1d(k: int, n: int) -> np.ndarray:
    return np.sin(2.0 * np.pi * k * np.arange(n, dtype=np.float64) / n)


@dataclass
class Heat3D:
    u0: np.ndarray
    wavenumbers: np.ndarray  # (modes, 3): kz, ky, kx
    amplitudes: np.ndarray   # (modes,)


def heat3d(n: int = 512, seed: int = 1, noise: bool = True, modes: int = 8,
           shape=None, sigma: float = 0.01) -> Heat3D:
    """Sum of product-of-sines modes plus Gaussian noise on a periodic grid."""
    shp = tuple(shape) if shape is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    ks = rng.integers(1, 17, size=(modes, 3))
    amps = rng.random(modes)
    u = np.zeros(shp, dtype=np.float64)
    for m in range(modes):
        sz = _sine_modes_1d(int(ks[m, 0]), shp[0])
        sy = _sine_modes_1d(int(ks[m, 1]), shp[1])
        sx = _sine_modes_1d(int(ks[m, 2]), shp[2])
        plane = (amps[m] * sy)[:, None] * sx[None, :]
        u += sz[:, None, None] * plane[None, :, :]
    if noise:
        u += rng.normal(0.0, sigma, size=shp)
    return Heat3D(u, ks, amps)


@dataclass
class Wave3D:
    m: np.ndarray          # per-cell (c dt / h)^2, shape (nz, ny, nx)
    c_layers: np.ndarray   # velocity per layer
    layer_of_z: np.ndarray # layer index of each z-plane
    h: float
    dt: float
    src: tuple             # interior index of the source cell
    amps: np.ndarray       # source amplitude per step, dt^2 r(n dt)


def ricker(t, f: float = 15.0, t0: float | None = None):
    t0 = 1.0 / f if t0 is None else t0
    a = (np.pi * f * (np.asarray(t, dtype=np.float64) - t0)) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def wave3d(n: int = 512, steps: int = 1000, seed: int = 2, layers: int = 8,
           cfl: float = 0.4, f: float = 15.0) -> Wave3D:
    """Layered velocity model and Ricker source on an n^3 interior."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(1.5, 4.5, size=layers)
    h = 1.0 / n
    dt = cfl * h / float(c.max())
    layer_of_z = (np.arange(n) * layers) // n
    m_layer = (c * dt / h) ** 2
    m = np.empty((n, n, n), dtype=np.float64)
    m[...] = m_layer[layer_of_z][:, None, None]
    amps = dt * dt * ricker(np.arange(steps, dtype=np.float64) * dt, f=f)
    return Wave3D(m, c, layer_of_z, h, dt, (n // 2, n // 2, n // 2), amps)


@dataclass
class VarCoef3D:
    u0: np.ndarray
    kappa: np.ndarray
    target: np.ndarray


KAPPA_MAX = 0.16


def varcoef3d(n: int = 256, seed: int = 3, target_seed: int = 5, shape=None) -> VarCoef3D:
    """Diffusivity field, initial field and target of the adjoint workload."""
    shp = tuple(shape) if shape is not None else (n, n, n)
    rng = np.random.default_rng(seed)
    u0 = rng.random(shp)
    z = rng.standard_normal(shp)
    kappa = np.clip(0.05 * np.exp(0.5 * z), 0.0, KAPPA_MAX)
    target = np.random.default_rng(target_seed).random(shp)
    return VarCoef3D(u0, kappa, target)


@dataclass
class Batch2D:
    shapes: np.ndarray     # (ngrids, 2): ny, nx
    weights: np.ndarray    # (ngrids, 9), rows sum to 1
    fields: list           # u0 per grid (or empty)


def batch2d(ngrids: int = 512, seed: int = 4, lo: int = 64, hi: int = 2048,
            with_fields: bool = True) -> Batch2D:
    """Uneven 2D grids with per-grid normalised 3x3 box weights."""
    rng = np.random.default_rng(seed)
    ny = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=ngrids))).astype(np.int64)
    nx = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=ngrids))).astype(np.int64)
    w = rng.random((ngrids, 9))
    w = w / w.sum(axis=1, keepdims=True)
    fields = [rng.random((int(ny[g]), int(nx[g]))) for g in range(ngrids)] if with_fields else []
    return Batch2D(np.stack([ny, nx], axis=1), w, fields)
