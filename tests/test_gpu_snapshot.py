"""Device-resident snapshot and restore (the single-process form of the
paper's rescale checkpoint, Sec. IV): a run interrupted by a snapshot, the
destruction of its grid and buffers, and a restore into a new grid must
continue exactly as the uninterrupted run (bit for bit: the same kernels on
the same data)."""
import gc

import numpy as np
import pytest

from gpu_helpers import require_cuda, torch
from paper_2512_19851_gb300 import inputs, stencils
from paper_2512_19851_gb300.grid import Grid

pytestmark = pytest.mark.gpu


def setup_module(_):
    require_cuda()


def heat(shape, periodic):
    offs, w, _ = stencils.heat3d()
    return Grid(shape, offs, w, periodic=periodic, bc_value=0.25, dtype=torch.float32)


@pytest.mark.parametrize("periodic", [True, False])
def test_heat_restart_equals_uninterrupted_run(periodic):
    shape = (40, 52, 68)
    u0 = inputs.heat3d(shape=shape).u0
    g = heat(shape, periodic)
    g.set_field(u0)
    g.step(23)
    g.sync()
    ref = g.current().cpu().numpy().copy()
    g.close()

    g = heat(shape, periodic)
    g.set_field(u0)
    g.step(10)
    snap = g.snapshot()
    g.sync()
    g.close()
    del g
    gc.collect()
    torch.cuda.empty_cache()
    h = heat(shape, periodic)          # new handle, new buffers
    h.restore(snap)
    h.step(13)
    h.sync()
    assert np.array_equal(h.current().cpu().numpy(), ref)
    h.close()


def test_wave_restart_keeps_both_levels_and_the_step_counter():
    """Leapfrog: the snapshot holds u^n and u^{n-1}; the step counter keeps
    the source on schedule after the restore."""
    n, steps, cut = 48, 37, 20
    wv = inputs.wave3d(n=n, steps=steps)
    offs, alpha, beta = stencils.wave25()

    def make():
        g = Grid((n,) * 3, offs, alpha, beta, periodic=False, dtype=torch.float32, time_levels=2)
        g.set_coeff(wv.m)
        g.set_source(wv.src, wv.amps)
        return g

    z = np.zeros((n,) * 3)
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
    assert np.array_equal(h.current().cpu().numpy(), ref_now)
    assert np.array_equal(h.previous().cpu().numpy(), ref_prev)
    h.close()
