"""GPU parity of the per-cell 7-point diffusion, its transpose (adjoint) and
the coefficient gradient with checkpoint-every-m recomputation.

Tolerances: FP64 <= 1e-12 normwise against the FP64 oracle; FP32 forward
<= 1e-5 (diffusion); FP32 gradients <= 1e-3 normwise against the FP64
oracle.  The gradient bound follows from the arithmetic: dL/dkappa sums
lambda * (Laplacian of u_t) over 200 steps, and the FP32 Laplacian of a
smoothed field cancels most of its digits (|sum of neighbours - 6u| is ~1e-2
of |u|), so its relative rounding error is ~100x FP32 epsilon before the sum.
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_err, require_cuda, torch
from paper_2512_19851_gb300 import abi, inputs
from paper_2512_19851_gb300.grid import Grid, StencilFn, VarCoefProblem

pytestmark = pytest.mark.gpu

TOL64 = 1e-12
TOL32_FWD = 1e-5
TOL32_GRAD = 1e-3
# Different pairings of steps into fused passes: one extra rounding of the
# working precision per pair of gradient terms (2^-24 or 2^-53 relative to the
# pair), amplified by the cancellation between a point's terms over the run
# (|sum of terms| is at least ~1e-2 of sum |terms| on these fields).
PAIR32 = 1e-5
PAIR64 = 1e-13
# FP32 grids: a checkpoint segment's terms are summed in an FP32 partial
# gradient (up to m terms, each rounding 2^-24 relative to the running sum)
# before the FP64 accumulator, so runs with different segments agree to that
# grouping's rounding, amplified by the same cancellation.
SEG32 = 1e-4
ALPHA = [1.0] + [0.0] * 6
BETA = [-6.0] + [1.0] * 6


def setup_module(_):
    require_cuda()


def make(shape, dtype, periodic=False, bc=0.0, generic=False):
    return Grid(shape, inputs.OFFSETS_7PT, ALPHA, BETA, periodic=periodic, bc_value=bc, dtype=dtype,
                generic=generic)


def gpu_grad(v, steps, m, dtype, periodic=False, bc=0.0, generic=False):
    g = make(v.u0.shape, dtype, periodic, bc, generic)
    prob = VarCoefProblem(g, steps, m)
    uT = prob.forward(v.u0, v.kappa).double().cpu().numpy()
    lam0, gk, loss = prob.backward_from(target=v.target)
    g.sync()
    out = (uT, lam0.double().cpu().numpy(), gk.cpu().numpy(), float(loss.cpu()[0]), g.kernel)
    g.close()
    return out


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_forward_full_size(dtype):
    """256^3, 200 steps, Dirichlet 0: the benchmark's forward."""
    v = inputs.varcoef3d(n=256)
    ref = oracle.varcoef7_forward(v.u0, v.kappa, False, 0.0, 200)
    g = make(v.u0.shape, dtype)
    g.set_field(v.u0)
    g.set_coeff(v.kappa)
    g.step(200)
    g.sync()
    got = g.current().double().cpu().numpy()
    assert rel_err(got, ref) <= (TOL64 if dtype == torch.float64 else TOL32_FWD), g.kernel
    g.close()


@pytest.mark.parametrize("periodic,bc", [(False, 0.0), (False, 0.3), (True, 0.0)])
@pytest.mark.parametrize("generic", [False, True])
def test_gradient_fp64_matches_oracle(periodic, bc, generic):
    v = inputs.varcoef3d(shape=(30, 27, 45))
    steps, m = 40, 7
    loss_r, uT_r, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, periodic, bc, steps, m)
    uT, lam0, gk, loss, kern = gpu_grad(v, steps, m, torch.float64, periodic, bc, generic)
    assert rel_err(uT, uT_r) <= TOL64, kern
    assert abs(loss - loss_r) <= TOL64 * loss_r
    assert rel_err(lam0, lam_r) <= TOL64, kern
    assert rel_err(gk, gk_r) <= TOL64, kern


def test_gradient_fp32_matches_fp64_oracle():
    v = inputs.varcoef3d(n=64)
    steps, m = 200, 20
    loss_r, uT_r, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, steps, m)
    uT, lam0, gk, loss, kern = gpu_grad(v, steps, m, torch.float32)
    assert rel_err(uT, uT_r) <= TOL32_FWD, kern
    assert abs(loss - loss_r) <= TOL32_FWD * loss_r
    assert rel_err(lam0, lam_r) <= TOL32_GRAD, kern
    assert rel_err(gk, gk_r) <= TOL32_GRAD, kern


def test_gradient_full_size_fused_pass():
    """256^3 FP32 Dirichlet, the benchmark's grid: four steps with a
    checkpoint every 2, so the reverse pass runs the fused two-step kernel in
    the benchmark's launch configuration (10-row tiles, two halo sub-tasks,
    the flat (tile, plane) distribution) on a recomputed and on a kept
    segment; every point of lambda_0 and of the gradient against the FP64
    oracle."""
    v = inputs.varcoef3d(n=256)
    steps, m = 4, 2
    loss_r, uT_r, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, steps, m)
    uT, lam0, gk, loss, kern = gpu_grad(v, steps, m, torch.float32)
    assert rel_err(uT, uT_r) <= TOL32_FWD, kern
    assert abs(loss - loss_r) <= TOL32_FWD * loss_r
    assert rel_err(lam0, lam_r) <= TOL32_FWD, kern
    assert rel_err(gk, gk_r) <= TOL32_GRAD, kern


def test_gradient_full_size_two_segments():
    """256^3 FP32 Dirichlet with the benchmark's checkpoint interval: 40
    steps, a checkpoint every 20, so the reverse pass recomputes one segment
    and reads the other from the forward run, in the benchmark's launch
    configuration; every point of lambda_0 and of the gradient against the
    FP64 oracle (which recomputes its own segments)."""
    v = inputs.varcoef3d(n=256)
    steps, m = 40, 20
    loss_r, uT_r, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, steps, m)
    uT, lam0, gk, loss, kern = gpu_grad(v, steps, m, torch.float32)
    assert rel_err(uT, uT_r) <= TOL32_FWD, kern
    assert abs(loss - loss_r) <= TOL32_FWD * loss_r
    assert rel_err(lam0, lam_r) <= TOL32_FWD, kern
    assert rel_err(gk, gk_r) <= TOL32_GRAD, kern
    # the recomputed segment (two steps per pass) holds the same states as the
    # forward run's single sweeps: keeping every state gives the same lambda
    # bits; the gradient sums each segment's terms in FP32 before the FP64
    # accumulator, so it agrees to that grouping's rounding
    kept = gpu_grad(v, steps, steps, torch.float32)
    assert np.array_equal(lam0, kept[1])
    assert rel_err(gk, kept[2]) <= SEG32


@pytest.mark.parametrize("periodic,bc", [(False, 0.0), (False, 0.3), (True, 0.0)])
def test_gradient_fp32_ragged_matches_fp64_oracle(periodic, bc):
    """FP32 transpose on rows that end inside a 16-byte group (nx = 45), a
    ragged last y tile and segments of 5, 5 and 2 steps (two-step and
    one-step passes)."""
    v = inputs.varcoef3d(shape=(30, 27, 45))
    steps, m = 12, 5
    loss_r, uT_r, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, periodic, bc, steps, m)
    uT, lam0, gk, loss, kern = gpu_grad(v, steps, m, torch.float32, periodic, bc)
    assert rel_err(uT, uT_r) <= TOL32_FWD, kern
    assert rel_err(lam0, lam_r) <= TOL32_FWD, kern
    assert rel_err(gk, gk_r) <= TOL32_GRAD, kern


@pytest.mark.parametrize("periodic,bc", [(False, 0.0), (True, 0.0)])
def test_gradient_wide_rows_matches_oracle(periodic, bc):
    """Rows wider than one warp of x groups: FP32 rows of 150 points (38
    groups, the last one ragged) and FP64 rows of 70 points (35 groups), so a
    tile's halo rows take two 32-group sub-tasks per halo warp, the second
    partly filled.  FP32 m = 5 and m = 1 give the same lambda_0 bitwise and
    gradients within the segment-grouping tolerance."""
    steps, m = 10, 5
    v = inputs.varcoef3d(shape=(14, 22, 150))
    loss_r, uT_r, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, periodic, bc, steps, m)
    uT, lam0, gk, loss, kern = gpu_grad(v, steps, m, torch.float32, periodic, bc)
    assert rel_err(uT, uT_r) <= TOL32_FWD, kern
    assert rel_err(lam0, lam_r) <= TOL32_FWD, kern
    assert rel_err(gk, gk_r) <= TOL32_GRAD, kern
    other = gpu_grad(v, steps, 1, torch.float32, periodic, bc)
    assert np.array_equal(lam0, other[1])
    assert rel_err(other[2], gk) <= SEG32
    v = inputs.varcoef3d(shape=(14, 22, 70))
    loss_r, uT_r, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, periodic, bc, steps, m)
    uT, lam0, gk, loss, kern = gpu_grad(v, steps, m, torch.float64, periodic, bc)
    assert rel_err(uT, uT_r) <= TOL64, kern
    assert rel_err(lam0, lam_r) <= TOL64, kern
    assert rel_err(gk, gk_r) <= TOL64, kern


def test_checkpoint_interval_does_not_change_gradient_fp32():
    """FP32 grids: fused two-step passes round lambda exactly like single
    steps, so m = 1, 6 and 20 give bitwise equal lambda_0.  The gradient sums
    a checkpoint segment's terms in an FP32 partial field before adding it to
    the FP64 accumulator, so different m agree within SEG32."""
    v = inputs.varcoef3d(shape=(20, 26, 44))
    base = gpu_grad(v, 20, 20, torch.float32, True)
    other = gpu_grad(v, 20, 6, torch.float32, True)
    assert np.array_equal(base[1], other[1])
    assert rel_err(other[2], base[2]) <= SEG32
    other = gpu_grad(v, 20, 1, torch.float32, True)
    assert np.array_equal(base[1], other[1])
    assert rel_err(other[2], base[2]) <= SEG32


def test_checkpoint_interval_does_not_change_gradient():
    """Recomputation is deterministic: m = 1, 7, 10 and 20 give bitwise equal
    lambda_0; gradients are bitwise equal for m = 10 and 20 (the same pairs of
    steps) and within PAIR64 for m = 1 and 7."""
    v = inputs.varcoef3d(shape=(20, 24, 32))
    base = gpu_grad(v, 20, 20, torch.float64)
    other = gpu_grad(v, 20, 10, torch.float64)
    assert np.array_equal(base[1], other[1]) and np.array_equal(base[2], other[2])
    for m in (1, 7):
        other = gpu_grad(v, 20, m, torch.float64)
        assert np.array_equal(base[1], other[1])
        assert rel_err(other[2], base[2]) <= PAIR64


def test_dot_product_identity_gpu():
    """<S x, y> = <x, S^T y> with the GPU forward and the GPU transpose."""
    shape = (24, 20, 28)
    v = inputs.varcoef3d(shape=shape)
    rng = np.random.default_rng(4)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    g = make(shape, torch.float64)
    prob = VarCoefProblem(g, 15, 4)
    sx = prob.forward(x, v.kappa).cpu().numpy().copy()
    lam0, _, _ = prob.backward_from(lam_T=y)
    st = lam0.cpu().numpy()
    lhs, rhs = float(np.vdot(sx, y)), float(np.vdot(x, st))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + np.abs(sx).sum())
    g.close()


def test_finite_differences_32cube():
    """Central differences of the GPU loss (FP64, 32^3 instance of the adjoint
    workload, 200 steps) against the GPU gradient: 8 random directions and 16
    single coordinates of kappa, 4 directions of u0.  The loss is exactly
    quadratic in u0 and smooth in kappa, so with eps = 1e-5 the truncation
    error is far below the FP64 rounding of the loss (~1e-13 of ~1e3 over
    2 eps), which sets the absolute floor of 1e-7."""
    v = inputs.varcoef3d(n=32)
    steps, m = 200, 20
    _, g_u, g_k, _, _ = gpu_grad(v, steps, m, torch.float64)
    grid = make(v.u0.shape, torch.float64)
    prob = VarCoefProblem(grid, steps, m)
    tgt = torch.as_tensor(v.target, device=grid.device)

    def L(u0, kappa):
        uT = prob.forward(u0, kappa)
        return 0.5 * float(((uT - tgt) ** 2).sum())

    rng = np.random.default_rng(0)
    eps = 1e-5
    for i in range(8):
        d = rng.standard_normal(v.kappa.shape)
        d /= np.linalg.norm(d)
        fd = (L(v.u0, v.kappa + eps * d) - L(v.u0, v.kappa - eps * d)) / (2 * eps)
        assert abs(fd - float(np.sum(g_k * d))) <= 1e-6 * abs(fd) + 1e-7
    for i in range(4):
        d = rng.standard_normal(v.u0.shape)
        d /= np.linalg.norm(d)
        fd = (L(v.u0 + eps * d, v.kappa) - L(v.u0 - eps * d, v.kappa)) / (2 * eps)
        assert abs(fd - float(np.sum(g_u * d))) <= 1e-6 * abs(fd) + 1e-7
    for j in range(16):
        p = tuple(int(c) for c in rng.integers(0, 32, size=3))
        e = np.zeros(v.kappa.shape)
        e[p] = 1.0
        fd = (L(v.u0, v.kappa + eps * e) - L(v.u0, v.kappa - eps * e)) / (2 * eps)
        assert abs(fd - g_k[p]) <= 1e-6 * abs(fd) + 1e-7
    grid.close()


def test_autograd_function():
    shape = (16, 18, 20)
    v = inputs.varcoef3d(shape=shape)
    steps, m = 12, 5
    loss_r, _, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, steps, m)
    g = make(shape, torch.float64)
    prob = VarCoefProblem(g, steps, m)
    u0 = torch.tensor(v.u0, device="cuda", requires_grad=True)
    kappa = torch.tensor(v.kappa, device="cuda", requires_grad=True)
    uT = StencilFn.apply(u0, kappa, prob)
    loss = 0.5 * ((uT - torch.as_tensor(v.target, device="cuda")) ** 2).sum()
    loss.backward()
    assert abs(float(loss.detach()) - loss_r) <= 1e-12 * loss_r
    assert rel_err(u0.grad.cpu().numpy(), lam_r) <= TOL64
    assert rel_err(kappa.grad.cpu().numpy(), gk_r) <= TOL64
    g.close()


def test_autograd_function_fp32_grid_takes_float64_tensors():
    """An FP32 grid fed float64 tensors: the gradients come back in the
    inputs' dtypes, close to the FP64 oracle."""
    shape = (12, 14, 40)
    v = inputs.varcoef3d(shape=shape)
    steps, m = 8, 3
    _, _, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, steps, m)
    g = make(shape, torch.float32)
    prob = VarCoefProblem(g, steps, m)
    u0 = torch.tensor(v.u0, device="cuda", requires_grad=True)
    kappa = torch.tensor(v.kappa, device="cuda", requires_grad=True)
    uT = StencilFn.apply(u0, kappa, prob)
    (0.5 * ((uT - torch.as_tensor(v.target, device="cuda")) ** 2).sum()).backward()
    assert u0.grad.dtype == torch.float64 and kappa.grad.dtype == torch.float64
    assert rel_err(u0.grad.cpu().numpy(), lam_r) <= TOL32_FWD
    assert rel_err(kappa.grad.cpu().numpy(), gk_r) <= TOL32_GRAD
    g.close()


def test_adjoint_argument_errors():
    g = make((8, 8, 8), torch.float32)
    prob = VarCoefProblem(g, 4, 2)
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_adjoint(g.h, 4, 2, prob.ws.data_ptr(), prob.lam.data_ptr(), prob.lam.data_ptr(), 0)
    assert e.value.code == abi.ST_ERR_ALIAS
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_step_ckpt(g.h, 4, 0, prob.ws.data_ptr())
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_bind(g.h, abi.ST_SLOT_B, g.bufs[0].data_ptr())
    assert e.value.code == abi.ST_ERR_ALIAS
    g.close()


def test_autograd_second_application_invalidates_first():
    """One problem applied twice before backward: the first node's backward
    raises (its checkpoints were overwritten) instead of returning the
    gradient of the second trajectory; the second node's backward is right.
    set_coeff on the grid also invalidates a recorded run.  The returned
    gradients are copies: a later reverse pass does not change them."""
    shape = (10, 12, 16)
    v = inputs.varcoef3d(shape=shape)
    steps, m = 6, 3
    _, _, lam_r, gk_r = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, steps, m)
    g = make(shape, torch.float64)
    prob = VarCoefProblem(g, steps, m)
    tgt = torch.as_tensor(v.target, device="cuda")
    u0a = torch.tensor(v.u0 * 0.5, device="cuda", requires_grad=True)
    ka = torch.tensor(v.kappa, device="cuda", requires_grad=True)
    la = 0.5 * ((StencilFn.apply(u0a, ka, prob) - tgt) ** 2).sum()
    u0 = torch.tensor(v.u0, device="cuda", requires_grad=True)
    kappa = torch.tensor(v.kappa, device="cuda", requires_grad=True)
    lb = 0.5 * ((StencilFn.apply(u0, kappa, prob) - tgt) ** 2).sum()
    with pytest.raises(RuntimeError):
        la.backward()
    lb.backward()
    assert rel_err(u0.grad.cpu().numpy(), lam_r) <= TOL64
    assert rel_err(kappa.grad.cpu().numpy(), gk_r) <= TOL64
    keep = kappa.grad.clone()
    prob.backward_from(lam_T=np.zeros(shape))  # zeroes and rewrites prob.gk
    torch.cuda.synchronize()
    assert torch.equal(kappa.grad, keep)
    u0c = torch.tensor(v.u0, device="cuda", requires_grad=True)
    kc = torch.tensor(v.kappa, device="cuda", requires_grad=True)
    lc = 0.5 * ((StencilFn.apply(u0c, kc, prob) - tgt) ** 2).sum()
    g.set_coeff(v.kappa)
    with pytest.raises(RuntimeError):
        lc.backward()
    g.close()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_kept_second_to_last_segment_and_repeated_reverse(dtype):
    """The forward run keeps the second-to-last segment's states in the
    recomputation levels, and the first reverse pass reads them; a second
    reverse pass on the same record recomputes that segment (the first one
    overwrote the levels).  All three reverse passes give the same bits, and
    those of a run that keeps every state (one segment; the same pairing of
    steps, since every segment has an even length) for lambda_0 and the FP64
    gradient; the FP32 gradient, summed per segment in FP32, within SEG32."""
    v = inputs.varcoef3d(shape=(18, 22, 40))
    steps, m = 24, 6
    g = make(v.u0.shape, dtype)
    prob = VarCoefProblem(g, steps, m)
    prob.forward(v.u0, v.kappa)
    first = [t.double().cpu().numpy() for t in prob.backward_from(target=v.target)[:2]]
    second = [t.double().cpu().numpy() for t in prob.backward_from(target=v.target)[:2]]
    other = VarCoefProblem(g, steps, m)   # a second record: the handle now remembers its workspace
    other.forward(v.u0, v.kappa)
    third = [t.double().cpu().numpy() for t in prob.backward_from(target=v.target)[:2]]
    g.close()
    _, lam_all, gk_all, _, _ = gpu_grad(v, steps, steps, dtype)
    for got in (first, second, third):
        assert np.array_equal(got[0], lam_all)
        if dtype == torch.float64:
            assert np.array_equal(got[1], gk_all)
        else:  # FP32 partial sums per segment before the FP64 accumulator
            assert rel_err(got[1], gk_all) <= SEG32
    assert np.array_equal(first[1], second[1]) and np.array_equal(first[1], third[1])
