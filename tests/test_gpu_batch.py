"""GPU parity of the batched 2D 3x3-box sweeps (uneven grids, per-grid
normalised weights, periodic).  Tolerances: FP32 <= 1e-5 normwise against
the FP64 oracle (diffusion-like: non-negative weights summing to 1, so the
map is max-norm contractive and rounding errors do not grow); FP64 plain
per-grid launches <= 1e-12."""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_err, require_cuda, torch
from paper_2512_19851_gb300 import abi, inputs
from paper_2512_19851_gb300.grid import Batch, Grid

pytestmark = pytest.mark.gpu

TOL32 = 1e-5
TOL64 = 1e-12


def setup_module(_):
    require_cuda()


def run_batch(b, steps, dtype=torch.float32, generic=False, tune=False, chunks=None):
    bt = Batch(b.shapes, inputs.OFFSETS_BOX9, b.weights, periodic=True, dtype=dtype, generic=generic)
    bt.set_fields(b.fields)
    if tune:
        bt.tune(steps)
    for c in (chunks or [steps]):
        bt.step(c)
    bt.sync()
    out = [bt.current(i).double().cpu().numpy() for i in range(len(b.fields))]
    bt.close()
    return out


def test_small_batch_matches_oracle():
    b = inputs.batch2d(ngrids=24, lo=5, hi=300)
    got = run_batch(b, 50)
    for i in range(24):
        ref = oracle.sweep_const(b.fields[i], inputs.OFFSETS_BOX9, b.weights[i], True, 0.0, 50)
        assert rel_err(got[i], ref) <= TOL32, (i, b.shapes[i])


def test_batch_equals_grids_run_alone_bitwise():
    b = inputs.batch2d(ngrids=12, lo=8, hi=400)
    got = run_batch(b, 23)
    for i in range(12):
        g = Grid(tuple(b.shapes[i]), inputs.OFFSETS_BOX9, b.weights[i], periodic=True, dtype=torch.float32)
        g.set_field(b.fields[i])
        g.step(23)
        g.sync()
        alone = g.current().double().cpu().numpy()
        g.close()
        assert np.array_equal(got[i], alone), (i, b.shapes[i])


def test_tuned_and_chunked_equal_default():
    b = inputs.batch2d(ngrids=16, lo=16, hi=700)
    a = run_batch(b, 50)
    t = run_batch(b, 50, tune=True)
    c = run_batch(b, 50, chunks=[7, 20, 23])
    for i in range(16):
        assert np.array_equal(a[i], t[i]) and np.array_equal(a[i], c[i])


def test_plain_fp64_launches_match_oracle():
    b = inputs.batch2d(ngrids=10, lo=16, hi=200)
    got = run_batch(b, 50, dtype=torch.float64, generic=True)
    for i in range(10):
        ref = oracle.sweep_const(b.fields[i], inputs.OFFSETS_BOX9, b.weights[i], True, 0.0, 50)
        assert rel_err(got[i], ref) <= TOL64


def test_full_batch_sampled_grids():
    """All 512 grids of the batched workload in one call; every 16th grid is
    checked point by point against the oracle, and every grid conserves its
    sum (periodic, weights sum to 1).  In FP32 the nine rounded weights sum
    to 1 within 9 * 2^-24, so 50 steps may scale a sum by up to 2.7e-5; the
    bound is 5e-5."""
    b = inputs.batch2d()
    bt = Batch(b.shapes, inputs.OFFSETS_BOX9, b.weights, periodic=True, dtype=torch.float32)
    bt.set_fields(b.fields)
    bt.tune(50)
    bt.step(50)
    bt.sync()
    for i in range(0, 512, 16):
        ref = oracle.sweep_const(b.fields[i], inputs.OFFSETS_BOX9, b.weights[i], True, 0.0, 50)
        assert rel_err(bt.current(i).double().cpu().numpy(), ref) <= TOL32, i
    for i in range(512):
        s0 = float(np.sum(b.fields[i]))
        s1 = float(bt.current(i).double().sum())
        assert abs(s1 - s0) <= 5e-5 * abs(s0), i
    bt.close()


def test_barrier_timeout_is_reported_and_context_survives():
    """Failure detection without a GPU fault: the persistent kernel's grid
    barrier is made to wait for one CTA more than launched; its bounded wait
    (50 ms) runs out, the status word reports ST_ERR_DEVICE_TIMEOUT, and the
    same handle then steps normally (one step was done before the barrier)."""
    b = inputs.batch2d(ngrids=6, lo=16, hi=120)
    bt = Batch(b.shapes, inputs.OFFSETS_BOX9, b.weights, periodic=True, dtype=torch.float32)
    bt.set_fields(b.fields)
    abi.stencil_batch_selftest_barrier(bt.h, 50_000_000)
    with pytest.raises(abi.StencilError) as e:
        bt.sync()
    assert e.value.code == abi.ST_ERR_DEVICE_TIMEOUT
    bt.step(4)
    bt.sync()
    for i in range(6):
        ref = oracle.sweep_const(b.fields[i], inputs.OFFSETS_BOX9, b.weights[i], True, 0.0, 5)
        assert rel_err(bt.current(i).double().cpu().numpy(), ref) <= TOL32
    bt.close()


def test_dirichlet_batch_matches_oracle():
    b = inputs.batch2d(ngrids=8, lo=10, hi=150)
    bt = Batch(b.shapes, inputs.OFFSETS_BOX9, b.weights, periodic=False, bc_value=0.25, dtype=torch.float32)
    bt.set_fields(b.fields)
    bt.step(13)
    bt.sync()
    for i in range(8):
        ref = oracle.sweep_const(b.fields[i], inputs.OFFSETS_BOX9, b.weights[i], False, 0.25, 13)
        assert rel_err(bt.current(i).double().cpu().numpy(), ref) <= TOL32
    bt.close()
