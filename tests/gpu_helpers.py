"""Helpers shared by the GPU parity tests: run a workload through the C ABI
(via the torch-facing Grid object) and fetch interiors as numpy arrays."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2512_19851_gb300 import inputs  # noqa: E402
from paper_2512_19851_gb300.grid import Grid  # noqa: E402


def require_cuda():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")


def five_point(a):
    return inputs.OFFSETS_5PT, [1 - 4 * a, a, a, a, a]


def seven_point(a):
    return inputs.OFFSETS_7PT, [1 - 6 * a] + [a] * 6


def run_const(u0, offsets, weights, periodic, bc_value, nsteps, dtype, generic=False, chunks=None, two_step=False):
    """Run nsteps sweeps on the GPU; chunks splits the run into several
    stencil_step calls (graph and direct paths, odd/even parities)."""
    g = Grid(u0.shape, offsets, weights, periodic=periodic, bc_value=bc_value, dtype=dtype, generic=generic,
             two_step=two_step)
    g.set_field(u0)
    for n in (chunks or [nsteps]):
        g.step(n)
    g.sync()
    out = g.current().double().cpu().numpy()
    kern = g.kernel
    g.close()
    return out, kern


def cone_box(field, center, half):
    """Periodic sub-box of side 2*half+1 centred on `center` (wrapping)."""
    idx = [np.arange(c - half, c + half + 1) % n for c, n in zip(center, field.shape)]
    return field[np.ix_(*idx)]


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = float(np.max(np.abs(ref)))
    return float(np.max(np.abs(x - ref))) / (den if den > 0 else 1.0)


def closed_form_heat3d(h, alpha, steps, shape):
    out = np.zeros(shape)
    for (kz, ky, kx), amp in zip(h.wavenumbers, h.amplitudes):
        lam = 1 - 4 * alpha * sum(math.sin(math.pi * kd / nd) ** 2 for kd, nd in zip((kz, ky, kx), shape))
        sz = np.sin(2 * np.pi * kz * np.arange(shape[0]) / shape[0])
        sy = np.sin(2 * np.pi * ky * np.arange(shape[1]) / shape[1])
        sx = np.sin(2 * np.pi * kx * np.arange(shape[2]) / shape[2])
        out += (amp * lam ** steps) * sz[:, None, None] * (sy[:, None] * sx[None, :])[None]
    return out
