"""GPU parity of the lid-driven cavity flow (stencil_cavity_*, the paper's
multi-field benchmark) against the numpy oracle (oracle/cavity.py).

Tolerances: FP64 <= 1e-12 normwise per field.  FP32: within twice the drift
of the oracle's own FP32 evaluation of the same expressions (the pressure
source divides velocity differences by dt, so FP32 loses digits there
whatever evaluates it), and never looser than 1e-3.
"""
import numpy as np
import pytest

from gpu_helpers import rel_err, require_cuda, torch
from oracle import cavity as cav
from paper_2512_19851_gb300.grid import Cavity

pytestmark = pytest.mark.gpu


def setup_module(_):
    require_cuda()


def run(P, shape, steps, dtype, u0=None, v0=None, p0=None, chunks=None):
    c = Cavity(shape[0], shape[1], P.dx, P.dy, P.dt, P.rho, P.nu, P.nit, P.lid, dtype=dtype)
    z = np.zeros(shape)
    c.set(z if u0 is None else u0, z if v0 is None else v0, z if p0 is None else p0)
    for n in chunks or [steps]:
        c.step(n)
    torch.cuda.synchronize()
    out = [t.double().cpu().numpy() for t in (c.u, c.v, c.p)]
    c.close()
    return out


def check(P, shape, steps, u0=None, v0=None, p0=None):
    z = np.zeros(shape)
    args = [z if a is None else a for a in (u0, v0, p0)]
    ref = cav.cavity_run(*args, P, steps)
    ref32 = cav.cavity_run(*args, P, steps, dtype=np.float32)
    got64 = run(P, shape, steps, torch.float64, *args)
    got32 = run(P, shape, steps, torch.float32, *args)
    for g, r in zip(got64, ref):
        assert rel_err(g, r) <= 1e-12
    for g, r, r32 in zip(got32, ref, ref32):
        drift = rel_err(r32, r)
        assert rel_err(g, r) <= max(2 * drift, 1e-3), (rel_err(g, r), drift)


def test_lid_driven_cavity_from_rest():
    """41 x 41 unit-density cavity on [0, 2]^2 from rest, nu = 0.1,
    dt = 0.001, 50 pressure iterations per step, 40 steps."""
    n = 41
    P = cav.CavityParams(dx=2 / (n - 1), dy=2 / (n - 1), dt=0.001, rho=1.0, nu=0.1, nit=50, lid=1.0)
    check(P, (n, n), 40)


def test_non_square_random_start_odd_iterations():
    """37 x 53 with dx != dy, rho != 1, 7 pressure iterations (the pressure
    ends in the other buffer), a random interior start."""
    rng = np.random.default_rng(71)
    shape = (37, 53)
    P = cav.CavityParams(dx=0.04, dy=0.05, dt=0.0005, rho=1.3, nu=0.05, nit=7, lid=0.8)
    u0, v0, p0 = (0.1 * rng.standard_normal(shape) for _ in range(3))
    check(P, shape, 12, u0, v0, p0)


def test_many_tiles():
    """97 x 130: interior blocks, blocks on every edge and ragged last blocks
    of the pressure kernel's 32 x 8 tiles."""
    rng = np.random.default_rng(73)
    shape = (97, 130)
    P = cav.CavityParams(dx=0.02, dy=0.025, dt=0.0002, rho=1.0, nu=0.05, nit=20, lid=1.0)
    u0, v0, p0 = (0.1 * rng.standard_normal(shape) for _ in range(3))
    check(P, shape, 6, u0, v0, p0)


def test_split_calls_equal_one_call_and_no_pressure_iterations():
    rng = np.random.default_rng(72)
    shape = (29, 34)
    P = cav.CavityParams(dx=0.05, dy=0.05, dt=0.001, nit=3)
    u0, v0, p0 = (0.1 * rng.standard_normal(shape) for _ in range(3))
    one = run(P, shape, 5, torch.float64, u0, v0, p0)
    split = run(P, shape, 5, torch.float64, u0, v0, p0, chunks=[2, 3])
    for a, b in zip(one, split):
        assert np.array_equal(a, b)
    P0 = cav.CavityParams(dx=0.05, dy=0.05, dt=0.001, nit=0)
    ref = cav.cavity_run(u0, v0, p0, P0, 4)
    for g, r in zip(run(P0, shape, 4, torch.float64, u0, v0, p0), ref):
        assert rel_err(g, r) <= 1e-12


def test_large_grid_ragged_tiles_and_partial_passes():
    """2050 x 2077 (ragged 128 x 32 tiles of the FP32 pressure passes, every
    edge), 13 pressure iterations per step (a pass of 8 and one of 5), a
    random start, 3 steps: FP64 and FP32 against the oracle."""
    rng = np.random.default_rng(74)
    shape = (2050, 2077)
    P = cav.CavityParams(dx=2 / 2076, dy=2 / 2049, dt=2e-5, rho=1.0, nu=0.1, nit=13, lid=1.0)
    u0, v0, p0 = (0.1 * rng.standard_normal(shape) for _ in range(3))
    check(P, shape, 3, u0, v0, p0)


def test_benchmark_scheme_at_2048_from_rest():
    """The benchmark's scheme at 2048^2 (50 pressure iterations per step,
    dt from the stability limit, from rest), 4 steps."""
    n = 2048
    dx = 2.0 / (n - 1)
    P = cav.CavityParams(dx=dx, dy=dx, dt=0.25 * min(dx, dx * dx / 0.4), rho=1.0, nu=0.1, nit=50, lid=1.0)
    check(P, (n, n), 4)


def test_fp32_split_calls_equal_one_call():
    """FP32 (pressure iterations in shared-memory passes): split calls give
    the bits of one call."""
    rng = np.random.default_rng(75)
    shape = (70, 300)
    P = cav.CavityParams(dx=0.05, dy=0.04, dt=0.0005, nit=11)
    u0, v0, p0 = (0.1 * rng.standard_normal(shape) for _ in range(3))
    one = run(P, shape, 5, torch.float32, u0, v0, p0)
    split = run(P, shape, 5, torch.float32, u0, v0, p0, chunks=[1, 4])
    for a, b in zip(one, split):
        assert np.array_equal(a, b)
