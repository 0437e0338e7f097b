"""GPU parity of sweeps whose Dirichlet ghost cells hold the caller's values
(ST_FLAG_CALLER_GHOSTS: per-face or varying boundary data, Example 1's
boundary ring with edges that differ), against the oracle's padded sweep.

Tolerances as elsewhere: FP64 <= 1e-12, FP32 <= 1e-5 normwise against the
FP64 oracle (weights summing to at most 1 in absolute value).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_err, require_cuda, torch
from paper_2512_19851_gb300 import abi, inputs
from paper_2512_19851_gb300.abi import StencilError
from paper_2512_19851_gb300.grid import Grid

pytestmark = pytest.mark.gpu

TOL = {torch.float64: 1e-12, torch.float32: 1e-5}
ASYM2 = ([(0, 0), (-2, 1), (1, -2), (0, 2), (2, 0), (-1, -1)], [0.3, 0.1, 0.25, -0.15, 0.2, 0.05])


def setup_module(_):
    require_cuda()


def run(padded, offsets, weights, steps, dtype, chunks=None, two_step=False):
    """Interior + ring on the GPU (both buffers get the same ring); returns
    the newest level's interior + ring, the other buffer's ring and the kernel."""
    r = max(abs(c) for o in offsets for c in o)
    shape = tuple(s - 2 * r for s in padded.shape)
    g = Grid(shape, offsets, weights, dtype=dtype, caller_ghosts=True, two_step=two_step)
    t = torch.as_tensor(padded, dtype=dtype, device=g.device)
    for b in g.bufs:
        g.ring(b).copy_(t)
    for n in chunks or [steps]:
        g.step(n)
    g.sync()
    cur = g.current_slot()
    out = g.ring(g.bufs[cur]).double().cpu().numpy()
    other = g.ring(g.bufs[1 - cur]).double().cpu().numpy()
    kern = g.kernel
    g.close()
    return out, other, kern


def ring_mask(shape, r):
    m = np.ones(shape, dtype=bool)
    m[tuple(slice(r, s - r) for s in shape)] = False
    return m


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape,stencil,r", [
    ((70, 45), (inputs.OFFSETS_5PT, [0.2] * 5), 1),
    ((37, 61), ASYM2, 2),
    ((20, 36, 52), (inputs.OFFSETS_7PT, [0.4] + [0.1] * 6), 1),
    ((9, 17, 131), (inputs.OFFSETS_7PT, [0.4] + [0.1] * 6), 1),
])
def test_random_ring_matches_oracle(dtype, shape, stencil, r):
    """Random interior and random ring values; 13 steps split 6 + 7 (both
    parities, graph and direct paths).  The ring is never written."""
    rng = np.random.default_rng(31)
    pad = rng.random(tuple(s + 2 * r for s in shape))
    offs, w = stencil
    ref = oracle.sweep_ghosts(pad, r, offs, w, 13)
    got, other, kern = run(pad, offs, w, 13, dtype, chunks=[6, 7])
    inner = tuple(slice(r, r + s) for s in shape)
    assert rel_err(got[inner], ref[inner]) <= TOL[dtype], kern
    m = ring_mask(pad.shape, r)
    want = pad.astype(np.float32).astype(np.float64) if dtype == torch.float32 else pad
    assert np.array_equal(got[m], want[m]) and np.array_equal(other[m], want[m]), kern


def test_hot_edge_laplace_converges_like_the_oracle():
    """The classic Dirichlet Laplace problem (one edge at 1, the others at
    0), Example 1's update, 500 iterations in FP64."""
    n = 64
    pad = np.zeros((n + 2, n + 2))
    pad[0, :] = 1.0
    offs, w = [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4
    ref = oracle.sweep_ghosts(pad, 1, offs, w, 500)
    got, _, kern = run(pad, offs, w, 500, torch.float64)
    assert rel_err(got, ref) <= 1e-12, kern


def test_two_step_flag_keeps_single_sweeps():
    """The two-step 3D pass substitutes the boundary value for ghost reads, so
    caller ghosts keep single sweeps even when two-step passes are asked for."""
    rng = np.random.default_rng(32)
    pad = rng.random((34, 66, 66))
    offs, w = inputs.OFFSETS_7PT, [0.4] + [0.1] * 6
    ref = oracle.sweep_ghosts(pad, 1, offs, w, 8)
    got, _, kern = run(pad, offs, w, 8, torch.float32, two_step=True)
    assert rel_err(got[1:-1, 1:-1, 1:-1], ref[1:-1, 1:-1, 1:-1]) <= 1e-5, kern


def test_caller_ghost_errors():
    with pytest.raises(StencilError) as e:
        abi.stencil_create(2, (8, 8), 0, inputs.OFFSETS_5PT, [0.2] * 5, None, abi.ST_PERIODIC, 0.0, abi.ST_F64, 1,
                           abi.ST_FLAG_CALLER_GHOSTS)
    assert e.value.code == abi.ST_ERR_ARG
    g = Grid((8, 9, 10), inputs.OFFSETS_7PT, [1.0] + [0.0] * 6, [-6.0] + [1.0] * 6, dtype=torch.float64,
             caller_ghosts=True)
    ws = torch.empty(1 << 20, dtype=torch.uint8, device=g.device)
    with pytest.raises(StencilError) as e:
        abi.stencil_step_ckpt(g.h, 2, 1, ws.data_ptr())
    assert e.value.code == abi.ST_ERR_UNSUPPORTED
    g.close()


# ---------------------------------------------------------------- zero-flux (Neumann) boundary
def run_neumann(u0, offsets, weights, dtype, chunks):
    g = Grid(u0.shape, offsets, weights, dtype=dtype, neumann=True)
    g.set_field(u0)
    for n in chunks:
        g.step(n)
    g.sync()
    out = g.current().double().cpu().numpy()
    kern = g.kernel
    g.close()
    return out, kern


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape,stencil", [
    ((70, 45), (inputs.OFFSETS_5PT, [0.2] * 5)),
    ((37, 61), ASYM2),
    ((20, 36, 52), (inputs.OFFSETS_7PT, [0.4] + [0.1] * 6)),
    ((9, 17, 131), (inputs.OFFSETS_7PT, [0.4] + [0.1] * 6)),
])
def test_neumann_matches_oracle(dtype, shape, stencil):
    """Mirror-image ghosts refreshed before every sweep; 21 steps split 8 + 13."""
    rng = np.random.default_rng(33)
    u0 = rng.random(shape)
    offs, w = stencil
    ref = oracle.sweep_neumann(u0, offs, w, 21)
    got, kern = run_neumann(u0, offs, w, dtype, [8, 13])
    assert rel_err(got, ref) <= TOL[dtype], kern


def test_neumann_conserves_heat_at_size():
    """Zero flux: 100 FP64 sweeps of the 7-point heat step on 128 x 192 x 256
    keep sum(u) to rounding, and a cosine mode decays by its eigenvalue."""
    shape, k, a = (128, 192, 256), (2, 3, 5), 0.1
    grids = np.meshgrid(*[np.arange(n) + 0.5 for n in shape], indexing="ij")
    u0 = 1.0 + np.prod([np.cos(np.pi * kk * gg / n) for kk, gg, n in zip(k, grids, shape)], axis=0)
    del grids
    lam = 1 - 4 * a * sum(np.sin(np.pi * kk / (2 * n)) ** 2 for kk, n in zip(k, shape))
    got, kern = run_neumann(u0, inputs.OFFSETS_7PT, [1 - 6 * a] + [a] * 6, torch.float64, [100])
    assert abs(got.sum() - u0.sum()) <= 1e-12 * u0.sum(), kern
    assert np.max(np.abs(got - (1.0 + lam ** 100 * (u0 - 1.0)))) <= 1e-12, kern


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("shape,stencil,steps,m", [
    ((37, 53), (inputs.OFFSETS_5PT, [0.2] * 5), 12, 5),
    ((23, 29), ASYM2, 9, 4),
    ((14, 17, 19), (inputs.OFFSETS_7PT, [0.4] + [0.1] * 6), 10, 3),
    ((9, 12, 70), (inputs.OFFSETS_7PT, [0.3, 0.1, 0.15, 0.12, 0.08, 0.13, 0.12]), 8, 8),
])
def test_neumann_adjoint_matches_oracle(dtype, shape, stencil, steps, m):
    """Checkpointed zero-flux run and its reverse pass (the transpose of the
    mirror-then-sweep step): the loss and dL/du0 against the oracle's
    scatter transpose; lambda_0 bitwise independent of the checkpoint
    interval (every transposed step is one launch of the same kernel and
    recomputed states equal the forward run's)."""
    from paper_2512_19851_gb300.grid import VarCoefProblem
    rng = np.random.default_rng(34)
    u0, t = rng.random(shape), rng.random(shape)
    offs, w = stencil
    loss_r, uT_r, lam_r = oracle.neumann_loss_gradient(u0, t, offs, w, steps)
    out = []
    for mm in (m, 1, steps):
        g = Grid(shape, offs, w, dtype=dtype, neumann=True)
        p = VarCoefProblem(g, steps, mm)
        uT = p.forward(u0).double().cpu().numpy()
        lam0, _, loss = p.backward_from(target=t)
        g.sync()
        out.append((uT, lam0.double().cpu().numpy(), float(loss.cpu()[0])))
        g.close()
    uT, lam0, loss = out[0]
    tol = TOL[dtype]
    assert rel_err(uT, uT_r) <= tol
    assert abs(loss - loss_r) <= tol * loss_r
    assert rel_err(lam0, lam_r) <= tol
    assert np.array_equal(lam0, out[1][1]) and np.array_equal(lam0, out[2][1])
