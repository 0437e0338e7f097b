"""GPU parity of programs written in the slice-assignment frontend (the
paper's Example 1 and variants), executed by the library's kernels through
the C ABI, against the golden fixture (exact rationals) and the oracle.

Tolerances: Example 1's values are dyadic rationals with at most 22
significant bits at every partial sum, so FP64 and FP32 must match the exact
fixture bit for bit; elsewhere FP64 <= 1e-12 and FP32 <= 1e-5 normwise
against the FP64 oracle (diffusion with non-negative weights summing to 1).
"""
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from gpu_helpers import rel_err, require_cuda
from paper_2512_19851_gb300.frontend import Program, UnsupportedExpression

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "example1_laplace_8x6_10it.txt")
OFF4 = [(-1, 0), (1, 0), (0, -1), (0, 1)]


def setup_module(_):
    require_cuda()


def example1(p, shape, iters, dtype, ring=1.0, u0=None):
    u1 = p.create_array(shape, dtype)
    u2 = p.create_array(shape, dtype)
    if u0 is not None:
        u1[1:-1, 1:-1] = u0
    u1[0, :] = u1[-1, :] = u1[:, 0] = u1[:, -1] = ring
    u2[0, :] = u2[-1, :] = u2[:, 0] = u2[:, -1] = ring
    for _ in range(iters):
        u2[1:-1, 1:-1] = 0.25 * (u1[:-2, 1:-1] + u1[2:, 1:-1] + u1[1:-1, :-2] + u1[1:-1, 2:])
        u1, u2 = u2, u1
    return u1, u2


def golden():
    rows = [ln.split() for ln in open(GOLDEN) if not ln.startswith("#")]
    return np.array([[float(Fraction(v)) for v in r] for r in rows])


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_example1_matches_exact_fixture(dtype):
    """Example 1 scaled to an 8 x 6 interior, 10 iterations: bit for bit."""
    p = Program()
    u1, u2 = example1(p, (10, 8), 10, dtype)
    p.sync()
    got = u1.get()
    assert np.array_equal(got[1:-1, 1:-1].astype(np.float64), golden())
    assert np.all(got[0, :] == 1) and np.all(got[:, -1] == 1)
    # the other array holds iteration 9
    ref9 = oracle.sweep_const(np.zeros((8, 6)), OFF4, [0.25] * 4, False, 1.0, 9)
    assert np.array_equal(u2.get()[1:-1, 1:-1].astype(np.float64), ref9)
    p.close()


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
@pytest.mark.parametrize("iters", [37, 40])
def test_example1_ragged_against_oracle(dtype, tol, iters):
    """A random interior on a 300 x 203 array (ragged rows and tiles), odd
    and even iteration counts: both arrays against the oracle."""
    rng = np.random.default_rng(11)
    u0 = rng.random((298, 201))
    p = Program()
    u1, u2 = example1(p, (300, 203), iters, dtype, ring=0.75, u0=u0)
    p.sync()
    refn = oracle.sweep_const(u0, OFF4, [0.25] * 4, False, 0.75, iters)
    refm = oracle.sweep_const(u0, OFF4, [0.25] * 4, False, 0.75, iters - 1)
    a, b = u1.get(), u2.get()
    assert rel_err(a[1:-1, 1:-1].astype(np.float64), refn) <= tol
    assert rel_err(b[1:-1, 1:-1].astype(np.float64), refm) <= tol
    assert np.all(a[0] == np.asarray(0.75, dtype)) and np.all(b[:, 0] == np.asarray(0.75, dtype))
    p.close()


def test_depth_limited_flushes_equal_one_run():
    """A DAG flushed every 5 levels gives the same result as one flush."""
    rng = np.random.default_rng(12)
    u0 = rng.random((62, 45))
    outs = []
    for depth in (1 << 16, 5):
        p = Program(max_depth=depth)
        u1, _ = example1(p, (64, 47), 23, np.float64, ring=0.0, u0=u0)
        outs.append(u1.get())
        p.close()
    assert np.array_equal(outs[0], outs[1])
    ref = oracle.sweep_const(u0, OFF4, [0.25] * 4, False, 0.0, 23)
    assert rel_err(outs[0][1:-1, 1:-1], ref) <= 1e-12


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_fused_fields_run_as_one_batch(dtype, tol):
    """Two fields updated in each iteration fuse (Sec. III-B node fusion) and
    run as one batched launch per call; each field against the oracle."""
    rng = np.random.default_rng(13)
    v0, w0 = rng.random((128, 95)), rng.random((128, 95))
    p = Program()
    v1, v2 = p.create_array((130, 97), dtype), p.create_array((130, 97), dtype)
    w1, w2 = p.create_array((130, 97), dtype), p.create_array((130, 97), dtype)
    v1[1:-1, 1:-1] = v0
    w1[1:-1, 1:-1] = w0
    iters = 11
    for _ in range(iters):
        v2[1:-1, 1:-1] = 0.5 * (v1[:-2, 1:-1] + v1[2:, 1:-1])
        w2[1:-1, 1:-1] = 0.125 * (w1[:-2, :-2] + w1[2:, 2:]) + 0.25 * (w1[1:-1, :-2] + w1[1:-1, 2:]) \
            + 0.25 * w1[1:-1, 1:-1]
        v1, v2 = v2, v1
        w1, w2 = w2, w1
    assert p.plan() == [("fill", 0), ("fill", 1), ("run", [2, 3], iters)]
    p.sync()
    refv = oracle.sweep_const(v0, [(-1, 0), (1, 0)], [0.5, 0.5], False, 0.0, iters)
    refw = oracle.sweep_const(w0, [(-1, -1), (1, 1), (0, -1), (0, 1), (0, 0)],
                              [0.125, 0.125, 0.25, 0.25, 0.25], False, 0.0, iters)
    assert rel_err(v1.get()[1:-1, 1:-1].astype(np.float64), refv) <= tol
    assert rel_err(w1.get()[1:-1, 1:-1].astype(np.float64), refw) <= tol
    refw1 = oracle.sweep_const(w0, [(-1, -1), (1, 1), (0, -1), (0, 1), (0, 0)],
                               [0.125, 0.125, 0.25, 0.25, 0.25], False, 0.0, iters - 1)
    assert rel_err(w2.get()[1:-1, 1:-1].astype(np.float64), refw1) <= tol
    p.close()


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_3d_heat_program(dtype, tol):
    """A 3D seven-point heat program (the library's 3D star kernel)."""
    rng = np.random.default_rng(14)
    u0 = rng.random((32, 38, 50))
    i = slice(1, -1)
    p = Program()
    a, b = p.create_array((34, 40, 52), dtype), p.create_array((34, 40, 52), dtype)
    a[i, i, i] = u0
    a[0], a[-1], a[:, 0], a[:, -1], a[:, :, 0], a[:, :, -1] = (0.5,) * 6
    b[0], b[-1], b[:, 0], b[:, -1], b[:, :, 0], b[:, :, -1] = (0.5,) * 6
    for _ in range(7):
        b[i, i, i] = 0.4 * a[i, i, i] + 0.1 * (a[:-2, i, i] + a[2:, i, i] + a[i, :-2, i] + a[i, 2:, i]
                                               + a[i, i, :-2] + a[i, i, 2:])
        a, b = b, a
    p.sync()
    offs = [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    ref = oracle.sweep_const(u0, offs, [0.4] + [0.1] * 6, False, 0.5, 7)
    assert rel_err(a.get()[i, i, i].astype(np.float64), ref) <= tol
    p.close()


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_edges_with_different_values(dtype, tol):
    """Example 1 with a hot top edge (1) and the other edges at 0 in one
    array, and another ring in the other: the rings go to the library as
    caller-owned ghost cells; each sweep reads its input array's ring."""
    p = Program()
    u1, u2 = p.create_array((50, 41), dtype), p.create_array((50, 41), dtype)
    u1[0, :] = 1.0
    u2[0, :] = 1.0
    u2[:, -1] = 0.5                      # differs from u1's ring
    for _ in range(31):
        u2[1:-1, 1:-1] = 0.25 * (u1[:-2, 1:-1] + u1[2:, 1:-1] + u1[1:-1, :-2] + u1[1:-1, 2:])
        u1, u2 = u2, u1
    p.sync()
    # reference: steps alternate between the two rings, one step at a time
    r1 = np.zeros((50, 41))
    r1[0, :] = 1.0
    r2 = r1.copy()
    r2[:, -1] = 0.5
    a, b = r1, r2
    for _ in range(31):
        out = oracle.sweep_ghosts(a, 1, OFF4, [0.25] * 4, 1)
        b = b.copy()
        b[1:-1, 1:-1] = out[1:-1, 1:-1]
        a, b = b, a
    assert rel_err(u1.get().astype(np.float64), a) <= tol
    assert rel_err(u2.get().astype(np.float64), b) <= tol
    p.close()


def test_errors_surface_at_sync():
    p = Program()
    a, b = p.create_array((8, 8)), p.create_array((8, 8))
    b[1:-1, 1:-1] = a[1:-1, 1:-1]
    p.sync()
    b[2, 2] = 1.0                        # host-side write after a device sweep
    with pytest.raises(UnsupportedExpression, match="after a sweep"):
        p.sync()
    p.close()


@pytest.mark.parametrize("dtype,tol", [(np.float64, 1e-12), (np.float32, 1e-5)])
def test_example1_at_the_benchmark_size(dtype, tol):
    """Example 1 as the benchmark runs it: 16384^2 arrays, ring 1, interior
    0, 1000 iterations, through the frontend.  Information moves one cell per
    iteration, so after 1000 iterations (a) every point farther than 1000
    cells from the ring is still exactly 0, and (b) the points of a corner
    window of W cells that lie more than 1000 cells from the window's inner
    edges equal the oracle run on that W x W window with the same ring (what
    the oracle assumes beyond the inner edges cannot reach them).  FP32 is
    held to the 1e-5 of the other diffusion runs although the four-point
    average, being contractive, only guarantees about 1000 x 3 x 2^-24 =
    1.8e-4 after 1000 steps; the measured error is 1.5e-7 (FP64: 0)."""
    n, iters, w = 16384, 1000, 1080
    p = Program()
    u1, u2 = example1(p, (n, n), iters, dtype)
    p.sync()
    got = u1.view                              # device view of the newest level, 16384^2
    inner = got[1 + iters + 1:n - 1 - iters - 1, 1 + iters + 1:n - 1 - iters - 1]
    assert int((inner != 0).sum().item()) == 0
    ref = oracle.sweep_const(np.zeros((w, w)), OFF4, [0.25] * 4, False, 1.0, iters)
    k = w - iters - 1                          # exact part of the window
    corners = {
        "top-left": got[1:1 + k, 1:1 + k],
        "bottom-right": got[n - 1 - k:n - 1, n - 1 - k:n - 1],
    }
    want = {"top-left": ref[:k, :k], "bottom-right": ref[w - k:, w - k:]}
    for name, g in corners.items():
        e = rel_err(g.double().cpu().numpy(), want[name])
        print(f"{dtype.__name__} {name} window: normwise error {e:.3g}")
        assert e <= tol, name
    p.close()
