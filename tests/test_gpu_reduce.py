"""GPU parity of the FP32 interior reductions (sum, sum of squares, max |a - b|
in double precision) and of the loss residual, against the oracle's index-
order double sums of the same FP32 values.

The FP32 kernel stages work items through a shared-memory ring: runs of whole
padded rows of one plane when a row fits a stage (9216 floats for one field,
4608 per field for two), else segments of one interior row; the warps of a
block share out the rows of an item, or slices of a row when an item has
fewer rows than warps.  The shapes cover both kinds of item, ragged last
items (rows left over in a plane, a short last segment, rows whose length is
not a multiple of four), grids whose items are all whole (the kernel then
skips item positions), several items per block and fewer items than
blocks.

Tolerances: the GPU accumulates each block's values in a compensated float
pair (about 48 bits) and sums the block partials in double, so sums agree
with the oracle to a few units of 2^-44 relative to sum |x| (1e-12 is
asserted); the maximum is exact (equal bits).  The residual lambda = u - t is
rounded to FP32 once, as numpy's float32 subtraction is: equal bits."""
import numpy as np
import pytest

import oracle
from gpu_helpers import require_cuda, seven_point, torch

pytestmark = pytest.mark.gpu

SHAPES = [
    (7, 9),             # one item
    (129, 67),          # rows of 67 (not a multiple of 4), 16 rows per item
    (2050, 2077),       # 513 row items (1025 for two fields), ragged rows
    (5, 8200),          # one row per item; two fields: segments of 4608 and 3592
    (5, 9217),          # segments of 9216 and 1
    (4, 4610),          # two fields: segments of 4608 and 2
    (3, 16389),         # two or four segments per row, ragged last one
    (40, 52, 68),       # 3D, four items per plane
    (2, 3, 24583),      # 3D segments
    (96, 96, 96),       # 3D, 576 items, every item whole
    (64, 64),           # every row item whole
    (2, 18432),         # every segment whole (one field and two)
]


def setup_module(_):
    require_cuda()


def _grid(shape, r=1):
    from paper_2512_19851_gb300.grid import Grid
    if len(shape) == 3:
        offs, w = seven_point(0.1)
    else:
        offs, w = [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4
    if r == 2:
        far = [tuple(2 * c for c in o) for o in offs if any(o)]
        offs = list(offs) + far
        w = list(w) + [0.0] * len(far)
    return Grid(shape, offs, w, periodic=False, dtype=torch.float32)


def _check(got, ref, x):
    scale = np.sum(np.abs(x))
    assert abs(got[0] - ref[0]) <= 1e-12 * scale
    assert abs(got[1] - ref[1]) <= 1e-12 * ref[1]
    assert got[2] == ref[2]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("r", [1, 2])
def test_reduce_fp32_matches_oracle(shape, r):
    rng = np.random.default_rng(sum(shape) + r)
    a = (rng.standard_normal(shape) * 3.0).astype(np.float32)
    b = (rng.standard_normal(shape) + 0.5).astype(np.float32)
    g = _grid(shape, r)
    g.set_field(a, 0)
    g.set_field(b, 1)
    # nonzero ghosts: a kernel that summed a ghost or pad cell would show it
    for buf in g.bufs:
        full = buf.clone()
        buf.fill_(1e3)
        g.interior(buf).copy_(g.interior(full))
    one = g.reduce(g.bufs[0]).cpu().numpy()
    two = g.reduce(g.bufs[0], g.bufs[1]).cpu().numpy()
    g.close()
    _check(one, oracle.reduce(a), a.astype(np.float64))
    _check(two, oracle.reduce(a, b), a.astype(np.float64) - b.astype(np.float64))


@pytest.mark.parametrize("shape", [(129, 67), (5, 8200), (40, 52, 68), (2, 3, 24583)])
def test_residual_fp32_matches_oracle(shape):
    from paper_2512_19851_gb300 import abi
    rng = np.random.default_rng(len(shape) + shape[-1])
    u = rng.standard_normal(shape).astype(np.float32)
    t = rng.standard_normal(shape).astype(np.float32)
    g = _grid(shape)
    g.set_field(u, 0)
    g.set_field(t, 1)
    lam = torch.full_like(g.bufs[0], 7.0)
    loss = torch.zeros(3, dtype=torch.float64, device=g.device)
    s = torch.cuda.current_stream(g.device)
    abi.stencil_residual(g.h, g.bufs[0].data_ptr(), g.bufs[1].data_ptr(), lam.data_ptr(), loss.data_ptr(), s)
    torch.cuda.synchronize()
    got_lam = g.interior(lam).cpu().numpy()
    assert np.array_equal(got_lam.view(np.uint32), (u - t).view(np.uint32))
    ring = g.ring(lam).clone()
    ring[tuple(slice(g.radius, g.radius + n) for n in shape)] = 0
    assert float(ring.abs().max()) == 0.0  # every ghost cell set to 0
    ref = oracle.reduce(u, t)
    assert abs(float(loss[0]) - 0.5 * ref[1]) <= 1e-12 * 0.5 * ref[1]
    g.close()


def test_reduce_rejects_misaligned_buffers():
    from paper_2512_19851_gb300 import abi
    g = _grid((64, 64))
    out = torch.zeros(3, dtype=torch.float64, device=g.device)
    with pytest.raises(abi.StencilError):
        abi.stencil_reduce(g.h, g.bufs[0].data_ptr() + 4, 0, out.data_ptr(), torch.cuda.current_stream())
    with pytest.raises(abi.StencilError):
        abi.stencil_reduce_noalloc(g.h, g.bufs[0].data_ptr(), g.bufs[1].data_ptr() + 8, out.data_ptr(),
                                   torch.cuda.current_stream())
    g.close()


@pytest.mark.parametrize("shape,periodic", [((40, 52, 68), False), ((17, 23, 45), True), ((64, 64, 512), True),
                                            ((3, 64, 8), False), ((130, 33, 96), True)])
def test_step_reduce_fused_sweep_matches_oracle(shape, periodic):
    """stencil_step_reduce: the last sweep of an FP32 constant symmetric 3D
    star reduces the level it writes.  The field equals stencil_step's bit
    for bit; the sums agree with the oracle's double sums of the same FP32
    values within 1e-12 of sum |u| and the maximum exactly; nsteps = 0 reduces
    the current level; every result is the same on a repeated run."""
    from paper_2512_19851_gb300 import abi
    from paper_2512_19851_gb300.grid import Grid
    offs, w = seven_point(0.1)
    u0 = (np.random.default_rng(sum(shape)).random(shape) - 0.3).astype(np.float32)
    s = torch.cuda.current_stream()
    outs = []
    for rep in range(2):
        g = Grid(shape, offs, w, periodic=periodic, bc_value=0.5, dtype=torch.float32)
        g.set_field(u0)
        out = torch.zeros(3, dtype=torch.float64, device=g.device)
        abi.stencil_step_reduce(g.h, 7, out.data_ptr(), s)
        g.sync()
        got = g.current().cpu().numpy()
        outs.append(out.cpu().numpy())
        out0 = torch.zeros(3, dtype=torch.float64, device=g.device)
        abi.stencil_step_reduce(g.h, 0, out0.data_ptr(), s)
        g.sync()
        g.close()
        _check(out0.cpu().numpy(), oracle.reduce(got), got.astype(np.float64))
    assert np.array_equal(outs[0], outs[1])
    g = Grid(shape, offs, w, periodic=periodic, bc_value=0.5, dtype=torch.float32)
    g.set_field(u0)
    g.step(7)
    g.sync()
    ref_field = g.current().cpu().numpy()
    g.close()
    assert np.array_equal(got, ref_field)
    _check(outs[0], oracle.reduce(got), got.astype(np.float64))


def test_step_reduce_unfused_grids_equal_the_two_calls():
    """Grids without the fused sweep (FP64, per-cell weights) run stencil_step
    and stencil_reduce: the same bits as the two calls."""
    from paper_2512_19851_gb300 import abi
    from paper_2512_19851_gb300.grid import Grid
    offs, w = seven_point(0.1)
    shape = (20, 24, 36)
    u0 = np.random.default_rng(3).random(shape)
    s = torch.cuda.current_stream()
    res = []
    for fused_call in (True, False):
        g = Grid(shape, offs, w, periodic=True, dtype=torch.float64)
        g.set_field(u0)
        out = torch.zeros(3, dtype=torch.float64, device=g.device)
        if fused_call:
            abi.stencil_step_reduce(g.h, 5, out.data_ptr(), s)
        else:
            abi.stencil_step(g.h, 5, s)
            abi.stencil_reduce(g.h, g.bufs[g.current_slot()].data_ptr(), 0, out.data_ptr(), s)
        g.sync()
        res.append(out.cpu().numpy())
        g.close()
    assert np.array_equal(res[0], res[1])
