"""Device-resident snapshot and restore (the single-process form of the
paper's rescale checkpoint, Sec. IV): a run interrupted by a snapshot, the
destruction of its grid and buffers, and a restore into a new grid must
continue exactly as the uninterrupted run (bit for bit: the same kernels on
the same data), and the restarted run must match the CPU oracle's
uninterrupted run (FP64 <= 1e-12, FP32 diffusion <= 1e-5, FP32 wave <= 1e-3,
normwise against the FP64 oracle)."""
import gc

import numpy as np
import pytest

import oracle
from gpu_helpers import rel_err, require_cuda, torch
from paper_2512_19851_gb300 import inputs, stencils
from paper_2512_19851_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def setup_module(_):
    require_cuda()


def heat(shape, periodic, dtype=torch.float32):
    offs, w, _ = stencils.heat3d()
    return Grid(shape, offs, w, periodic=periodic, bc_value=0.25, dtype=dtype)


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-5), (torch.float64, 1e-12)])
@pytest.mark.parametrize("periodic", [True, False])
def test_heat_restart_equals_uninterrupted_run(periodic, dtype, tol):
    shape = (40, 52, 68)
    u0 = inputs.heat3d(shape=shape).u0
    offs, w, _ = stencils.heat3d()
    ref_oracle = oracle.sweep_const(u0, offs, w, periodic, 0.25, 23)
    g = heat(shape, periodic, dtype)
    g.set_field(u0)
    g.step(23)
    g.sync()
    ref = g.current().cpu().numpy().copy()
    g.close()

    g = heat(shape, periodic, dtype)
    g.set_field(u0)
    g.step(10)
    snap = g.snapshot()
    g.sync()
    g.close()
    del g
    gc.collect()
    torch.cuda.empty_cache()
    h = heat(shape, periodic, dtype)   # new handle, new buffers
    h.restore(snap)
    h.step(13)
    h.sync()
    got = h.current().cpu().numpy()
    assert np.array_equal(got, ref)
    assert rel_err(got, ref_oracle) <= tol, h.kernel
    h.close()


@pytest.mark.parametrize("dtype,tol", [(torch.float32, 1e-3), (torch.float64, 1e-12)])
def test_wave_restart_keeps_both_levels_and_the_step_counter(dtype, tol):
    """Leapfrog: the snapshot holds u^n and u^{n-1}; the step counter keeps
    the source on schedule after the restore."""
    n, steps, cut = 48, 37, 20
    wv = inputs.wave3d(n=n, steps=steps)
    offs, alpha, beta = stencils.wave25()
    z = np.zeros((n,) * 3)
    a8 = [float(x) for x in oracle.taylor_second_derivative_coeffs(4)]
    ora_now, ora_prev = oracle.wave25(z, z, wv.m, a8, wv.src, wv.amps, False, 0.0, steps)

    def make():
        g = Grid((n,) * 3, offs, alpha, beta, periodic=False, dtype=dtype, time_levels=2)
        g.set_coeff(wv.m)
        g.set_source(wv.src, wv.amps)
        return g

    g = make()
    g.set_levels(z, z)
    g.step(steps)
    g.sync()
    ref_now, ref_prev = g.current().cpu().numpy().copy(), g.previous().cpu().numpy().copy()
    g.close()

    g = make()
    g.set_levels(z, z)
    g.step(cut)
    snap = g.snapshot()
    assert snap[1] == cut
    g.sync()
    g.close()
    h = make()
    h.restore(snap)
    h.step(steps - cut)
    h.sync()
    now, prev = h.current().cpu().numpy(), h.previous().cpu().numpy()
    assert np.array_equal(now, ref_now)
    assert np.array_equal(prev, ref_prev)
    assert rel_err(now, ora_now) <= tol, h.kernel
    assert rel_err(prev, ora_prev) <= tol, h.kernel
    h.close()
