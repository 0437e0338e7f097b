"""GPU parity of the conservative (face-averaged) per-cell diffusion
(stencil_create_conservative), its transpose and the coefficient gradient,
against the numpy oracle (oracle/conservative.py).

Tolerances as for the affine per-cell operator: FP64 <= 1e-12 normwise;
FP32 forward and lambda <= 1e-5, FP32 gradient <= 1e-3 (the gradient sums
products of differences of a smoothed field, which cancel most digits).
"""
import numpy as np
import pytest

import oracle
from gpu_helpers import rel_err, require_cuda, torch
from paper_2512_19851_gb300 import inputs
from paper_2512_19851_gb300.grid import Grid, VarCoefProblem

pytestmark = pytest.mark.gpu


def setup_module(_):
    require_cuda()


def make(shape, dtype, periodic, bc):
    return Grid(shape, None, None, periodic=periodic, bc_value=bc, dtype=dtype, conservative=True)


def fields(shape, seed):
    rng = np.random.default_rng(seed)
    u0 = rng.random(shape)
    kappa = np.clip(0.05 * np.exp(0.5 * rng.standard_normal(shape)), 0.0, 0.16)
    return u0, kappa, rng.random(shape)


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("shape,periodic,bc", [((30, 27, 45), False, 0.3), ((30, 27, 45), True, 0.0),
                                                ((24, 20, 32), False, 0.3), ((24, 20, 32), True, 0.0),
                                                ((64, 50), False, 0.7), ((33, 70), True, 0.0), ((40, 64), True, 0.0)])
def test_forward_matches_oracle(dtype, tol, shape, periodic, bc):
    """Rows of 45 points take the one-point-per-thread kernels, rows of 32 and
    64 the 16-byte-group kernels (50 and 70 the group kernels in FP64 only)."""
    u0, kappa, _ = fields(shape, 51)
    g = make(shape, dtype, periodic, bc)
    g.set_field(u0)
    g.set_coeff(kappa)
    g.step(17)
    g.step(23)
    g.sync()
    ref = oracle.cons_forward(u0, kappa, periodic, bc, 40)
    assert rel_err(g.current().double().cpu().numpy(), ref) <= tol, g.kernel
    g.close()


def test_periodic_sum_conserved_at_size():
    """Any coefficient field: 100 FP64 sweeps on 128 x 96 x 80 keep sum(u)."""
    shape = (128, 96, 80)
    u0, kappa, _ = fields(shape, 52)
    g = make(shape, torch.float64, True, 0.0)
    g.set_field(u0)
    g.set_coeff(kappa)
    g.step(100)
    g.sync()
    got = g.current().cpu().numpy()
    assert abs(got.sum() - u0.sum()) <= 1e-12 * u0.sum()
    g.close()


def gpu_grad(shape, dtype, periodic, bc, steps, m, seed=53):
    u0, kappa, tgt = fields(shape, seed)
    g = make(shape, dtype, periodic, bc)
    prob = VarCoefProblem(g, steps, m)
    uT = prob.forward(u0, kappa).double().cpu().numpy()
    lam0, gk, loss = prob.backward_from(target=tgt)
    g.sync()
    out = uT, lam0.double().cpu().numpy(), gk.cpu().numpy(), float(loss.cpu()[0])
    g.close()
    return out, oracle.cons_loss_gradient(u0, kappa, tgt, periodic, bc, steps)


@pytest.mark.parametrize("periodic,bc", [(False, 0.3), (True, 0.0)])
@pytest.mark.parametrize("shape", [(20, 18, 22), (20, 18, 23)])
def test_gradient_fp64_matches_oracle(periodic, bc, shape):
    (uT, lam0, gk, loss), (loss_r, uT_r, lam_r, gk_r) = gpu_grad(shape, torch.float64, periodic, bc, 30, 7)
    assert rel_err(uT, uT_r) <= 1e-12
    assert abs(loss - loss_r) <= 1e-12 * loss_r
    assert rel_err(lam0, lam_r) <= 1e-12
    assert rel_err(gk, gk_r) <= 1e-12


@pytest.mark.parametrize("shape,periodic", [((40, 36, 44), False), ((40, 36, 44), True), ((40, 36, 45), False)])
def test_gradient_fp32_matches_fp64_oracle(shape, periodic):
    (uT, lam0, gk, loss), (loss_r, uT_r, lam_r, gk_r) = gpu_grad(shape, torch.float32, periodic, 0.0, 60, 20)
    assert rel_err(uT, uT_r) <= 1e-5
    assert rel_err(lam0, lam_r) <= 1e-5
    assert rel_err(gk, gk_r) <= 1e-3


def test_gradient_2d_and_checkpoint_interval():
    """2D, and m = 1, 6 and 25 give bitwise equal results (single-step
    transposes: the same expressions in the same order whatever m is)."""
    outs = [gpu_grad((48, 37), torch.float64, False, 0.2, 25, m)[0] for m in (25, 6, 1)]
    for o in outs[1:]:
        assert np.array_equal(o[1], outs[0][1]) and np.array_equal(o[2], outs[0][2])
    (uT, lam0, gk, loss), (loss_r, uT_r, lam_r, gk_r) = gpu_grad((48, 37), torch.float64, False, 0.2, 25, 6)
    assert rel_err(lam0, lam_r) <= 1e-12 and rel_err(gk, gk_r) <= 1e-12


@pytest.mark.parametrize("dtype,tol", [(torch.float64, 1e-13), (torch.float32, 1e-5)])
def test_gradient_3d_checkpoint_interval(dtype, tol):
    """3D (transposed steps as the forward sweep on lambda, the coefficient
    gradient in one pass per few steps): m = 30, 7 and 1 give bitwise equal
    lambda_0 (the same sweeps whatever m is); the gradient adds up to five
    steps' terms in the grid's precision before the FP64 accumulator, so
    different m agree to that grouping's rounding: a few units of the
    working precision relative to the terms, amplified by the cancellation
    between a point's terms over the run (the bound the varcoef adjoint's
    pairing test uses)."""
    outs = [gpu_grad((20, 18, 23), dtype, False, 0.2, 30, m)[0] for m in (30, 7, 1)]
    for o in outs[1:]:
        assert np.array_equal(o[1], outs[0][1])
        assert rel_err(o[2], outs[0][2]) <= tol
