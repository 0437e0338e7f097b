"""Pins of the CPU oracle to facts fixed by the mathematics, not by itself.

Each oracle routine is checked against at least one of: a closed form (the
decay factor of a discrete Fourier/sine mode, the leapfrog recurrence of a
plane wave), an invariant (constant fields, sum conservation, the maximum
principle, the discrete leapfrog energy), an exact golden fixture (Example 1
of Sec. III-A in rational arithmetic), brute force through an explicitly
assembled operator matrix on tiny grids, and for the adjoint the dot-product
identity and central finite differences.  The cases are picked so that a
dropped term, a wrong sign, a wrong index or a transposed operand fails one.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle.taylor import taylor_second_derivative_coeffs
from paper_2512_19851_gb300 import inputs

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------- helpers
def assemble(shape, offsets, weights, periodic, bc_value):
    """Dense matrix A and vector b with u_{t+1} = A u_t + b, built point by
    point from the neighbour list (brute force, tiny grids only)."""
    shape = tuple(shape)
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    b = np.zeros(n)
    for p in np.ndindex(*shape):
        ip = np.ravel_multi_index(p, shape)
        for o, w in zip(offsets, weights):
            q = [pi + oi for pi, oi in zip(p, o)]
            if periodic:
                q = [qi % si for qi, si in zip(q, shape)]
            elif any(qi < 0 or qi >= si for qi, si in zip(q, shape)):
                b[ip] += w * bc_value
                continue
            A[ip, np.ravel_multi_index(tuple(q), shape)] += w
    return A, b


def assemble_varcoef7(kappa, periodic, bc_value):
    shape = kappa.shape
    offs = [(0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)]
    n = kappa.size
    A = np.zeros((n, n))
    b = np.zeros(n)
    for p in np.ndindex(*shape):
        ip = np.ravel_multi_index(p, shape)
        k = kappa[p]
        A[ip, ip] += 1.0 - 6.0 * k
        for o in offs:
            q = [pi + oi for pi, oi in zip(p, o)]
            if periodic:
                q = [qi % si for qi, si in zip(q, shape)]
            elif any(qi < 0 or qi >= si for qi, si in zip(q, shape)):
                b[ip] += k * bc_value
                continue
            A[ip, np.ravel_multi_index(tuple(q), shape)] += k
    return A, b


def five_point(a):
    return inputs.OFFSETS_5PT, [1 - 4 * a, a, a, a, a]


def seven_point(a):
    return inputs.OFFSETS_7PT, [1 - 6 * a] + [a] * 6


# ---------------------------------------------------------------- golden
def test_example1_golden_exact():
    """Example 1 (Sec. III-A): boundary 1, weight 1/4, 10 iterations.  All
    values are dyadic, so double precision must match the exact fixture."""
    rows = []
    with open(os.path.join(HERE, "golden", "example1_laplace_8x6_10it.txt")) as f:
        for line in f:
            if line.startswith("#"):
                continue
            rows.append([float(Fraction(t)) for t in line.split()])
    gold = np.array(rows)
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    got = oracle.sweep_const(np.zeros(gold.shape), offs, [0.25] * 4, False, 1.0, 10)
    assert np.array_equal(got, gold)


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("shape,k,a,steps", [((9, 13), (2, 3), 0.2, 17), ((16, 11), (1, 2), 0.2, 100),
                                             ((7, 7), (1, 3), 0.1, 20)])
def test_dirichlet_sine_mode_decay(shape, k, a, steps):
    """A Dirichlet sine mode sin(pi k (i+1)/(n+1)) decays by
    1 - 4a (sin^2(pi ky/(2(ny+1))) + sin^2(pi kx/(2(nx+1)))) per step."""
    ny, nx = shape
    ky, kx = k
    my = np.sin(np.pi * ky * np.arange(1, ny + 1) / (ny + 1))
    mx = np.sin(np.pi * kx * np.arange(1, nx + 1) / (nx + 1))
    u0 = my[:, None] * mx[None, :]
    lam = 1 - 4 * a * (math.sin(math.pi * ky / (2 * (ny + 1))) ** 2 +
                       math.sin(math.pi * kx / (2 * (nx + 1))) ** 2)
    offs, w = five_point(a)
    got = oracle.sweep_const(u0, offs, w, False, 0.0, steps)
    assert oracle.normwise_error(got, lam ** steps * u0) < 1e-13


def test_periodic_2d_fourier_decay():
    """Periodic 2D: the eigenvalue of a Fourier mode is the one quoted in the
    workload description, 1 - 4a(sin^2(pi kx/N) + sin^2(pi ky/N))."""
    n, a, steps = 24, 0.2, 30
    kx, ky = 1, 2
    i = np.arange(n)
    u0 = np.cos(2 * np.pi * ky * i / n)[:, None] * np.sin(2 * np.pi * kx * i / n)[None, :]
    lam = 1 - 4 * a * (math.sin(math.pi * kx / n) ** 2 + math.sin(math.pi * ky / n) ** 2)
    offs, w = five_point(a)
    got = oracle.sweep_const(u0, offs, w, True, 0.0, steps)
    assert oracle.normwise_error(got, lam ** steps * u0) < 1e-13


def test_periodic_3d_sine_modes_closed_form():
    """heat3d recipe without noise: sum of product-of-sines modes, each
    decaying by 1 - 4 alpha sum_d sin^2(pi k_d / N_d)."""
    shape = (12, 10, 16)
    alpha, steps = 0.1, 25
    h = inputs.heat3d(shape=shape, noise=False)
    expect = np.zeros(shape)
    for (kz, ky, kx), amp in zip(h.wavenumbers, h.amplitudes):
        lam = 1 - 4 * alpha * sum(math.sin(math.pi * kd / nd) ** 2
                                  for kd, nd in zip((kz, ky, kx), shape))
        mode = (np.sin(2 * np.pi * kz * np.arange(shape[0]) / shape[0])[:, None, None] *
                np.sin(2 * np.pi * ky * np.arange(shape[1]) / shape[1])[None, :, None] *
                np.sin(2 * np.pi * kx * np.arange(shape[2]) / shape[2])[None, None, :])
        expect += amp * lam ** steps * mode
    offs, w = seven_point(alpha)
    got = oracle.sweep_const(h.u0, offs, w, True, 0.0, steps)
    assert oracle.normwise_error(got, expect) < 1e-12


# ---------------------------------------------------------------- invariants
def test_constant_field_invariant():
    """Paper's boundary value 1 with a constant interior of 1 stays 1 under
    weights 1/4 (exact), and a periodic constant stays under 7-point."""
    u = np.ones((10, 7))
    got = oracle.sweep_const(u, [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4, False, 1.0, 50)
    assert np.array_equal(got, u)
    v = np.full((6, 5, 7), 3.5)
    offs, w = seven_point(0.125)
    assert np.array_equal(oracle.sweep_const(v, offs, w, True, 0.0, 9), v)


def test_periodic_sum_conserved():
    u0 = inputs.heat3d(shape=(8, 9, 10)).u0
    offs, w = seven_point(0.1)
    s0 = math.fsum(u0.ravel())
    got = oracle.sweep_const(u0, offs, w, True, 0.0, 30)
    assert abs(math.fsum(got.ravel()) - s0) < 1e-12 * np.abs(u0).sum()


def test_max_principle():
    u0 = inputs.heat2d(shape=(20, 17))
    offs, w = five_point(0.2)
    lo, hi = u0.min(), u0.max()
    u = u0
    for _ in range(10):
        u = oracle.sweep_const(u, offs, w, False, 0.0, 3)
        assert u.min() >= min(lo, 0.0) - 1e-15 and u.max() <= hi + 1e-15
    # mass leaks out through a zero Dirichlet boundary
    assert u.sum() < u0.sum()


def test_linearity_periodic():
    shape = (6, 7, 5)
    rng = np.random.default_rng(11)
    x, y = rng.standard_normal(shape), rng.standard_normal(shape)
    offs, w = seven_point(0.1)
    lhs = oracle.sweep_const(2.5 * x - 0.75 * y, offs, w, True, 0.0, 6)
    rhs = 2.5 * oracle.sweep_const(x, offs, w, True, 0.0, 6) - 0.75 * oracle.sweep_const(y, offs, w, True, 0.0, 6)
    assert oracle.normwise_error(lhs, rhs) < 1e-13


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("periodic", [False, True])
@pytest.mark.parametrize("shape", [(6, 7), (4, 5, 3)])
def test_sweep_vs_assembled_matrix(shape, periodic):
    """Asymmetric offsets (radius 2) and unequal weights: the oracle equals
    u_S = A(...(A u_0 + b)...) + b with A, b assembled point by point."""
    rng = np.random.default_rng(7)
    nd = len(shape)
    offs = [tuple(int(v) for v in rng.integers(-2, 3, size=nd)) for _ in range(6)]
    offs[0] = (0,) * nd
    w = list(rng.standard_normal(6) * 0.3)
    u0 = rng.standard_normal(shape)
    steps = 5
    A, b = assemble(shape, offs, w, periodic, 0.7)
    v = u0.ravel().copy()
    for _ in range(steps):
        v = A @ v + b
    got = oracle.sweep_const(u0, offs, w, periodic, 0.7, steps)
    assert oracle.normwise_error(got.ravel(), v) < 1e-13


@pytest.mark.parametrize("periodic", [False, True])
def test_varcoef7_vs_assembled_matrix(periodic):
    shape = (4, 3, 5)
    rng = np.random.default_rng(3)
    kappa = rng.uniform(0.0, 0.16, size=shape)
    u0 = rng.random(shape)
    A, b = assemble_varcoef7(kappa, periodic, 0.3)
    v = u0.ravel().copy()
    for _ in range(7):
        v = A @ v + b
    got = oracle.varcoef7_forward(u0, kappa, periodic, 0.3, 7)
    assert oracle.normwise_error(got.ravel(), v) < 1e-13


# ---------------------------------------------------------------- adjoint
@pytest.mark.parametrize("periodic", [False, True])
def test_adjoint_equals_matrix_transpose(periodic):
    """lambda_0 = (A_S ... A_1)^T lambda_S with the assembled matrices, and
    the dot-product identity <S x, y> = <x, S^T y>."""
    shape = (3, 4, 5)
    rng = np.random.default_rng(5)
    kappa = rng.uniform(0.0, 0.16, size=shape)
    A, _ = assemble_varcoef7(kappa, periodic, 0.0)
    steps = 6
    x = rng.standard_normal(shape)
    y = rng.standard_normal(shape)
    _, states = oracle.varcoef7_forward(x, kappa, periodic, 0.0, steps, store_states=True)
    lam0, _ = oracle.varcoef7_adjoint(states[:steps], kappa, y, periodic, 0.0)
    M = np.linalg.matrix_power(A, steps)
    assert oracle.normwise_error(lam0.ravel(), M.T @ y.ravel()) < 1e-13
    sx = states[steps]
    lhs = float(np.dot(sx.ravel(), y.ravel()))
    rhs = float(np.dot(x.ravel(), lam0.ravel()))
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1.0)


def test_adjoint_symmetric_special_case():
    """Constant kappa with a periodic boundary gives a symmetric operator:
    one transpose step equals one forward step."""
    shape = (6, 5, 4)
    kappa = np.full(shape, 0.11)
    y = np.random.default_rng(9).standard_normal(shape)
    _, states = oracle.varcoef7_forward(np.zeros(shape), kappa, True, 0.0, 1, store_states=True)
    lam, _ = oracle.varcoef7_adjoint(states[:1], kappa, y, True, 0.0)
    fwd = oracle.varcoef7_forward(y, kappa, True, 0.0, 1)
    assert oracle.normwise_error(lam, fwd) < 1e-15


def test_gradient_central_differences():
    """Loss 0.5||u_S - target||^2: gradients w.r.t. u_0 and kappa against
    central differences (double precision, 8 random directions + coordinates)."""
    shape = (5, 4, 6)
    v = inputs.varcoef3d(shape=shape)
    steps, bc = 12, 0.25
    loss, _, g_u0, g_k = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, bc, steps, 4)

    def L(u0, kappa):
        uT = oracle.varcoef7_forward(u0, kappa, False, bc, steps)
        return 0.5 * float(np.sum((uT - v.target) ** 2))

    assert abs(L(v.u0, v.kappa) - loss) < 1e-12 * loss
    rng = np.random.default_rng(1)
    eps = 1e-6
    for i in range(8):
        du = rng.standard_normal(shape)
        du /= np.linalg.norm(du)
        dk = rng.standard_normal(shape)
        dk /= np.linalg.norm(dk)
        fd_u = (L(v.u0 + eps * du, v.kappa) - L(v.u0 - eps * du, v.kappa)) / (2 * eps)
        fd_k = (L(v.u0, v.kappa + eps * dk) - L(v.u0, v.kappa - eps * dk)) / (2 * eps)
        assert abs(fd_u - np.sum(g_u0 * du)) < 1e-7 * (abs(fd_u) + 1e-3)
        assert abs(fd_k - np.sum(g_k * dk)) < 1e-7 * (abs(fd_k) + 1e-3)
    for j in range(16):
        p = tuple(int(c) for c in rng.integers(0, shape))
        e = np.zeros(shape)
        e[p] = 1.0
        fd_k = (L(v.u0, v.kappa + eps * e) - L(v.u0, v.kappa - eps * e)) / (2 * eps)
        assert abs(fd_k - g_k[p]) < 1e-7 * (abs(fd_k) + 1e-3)


def test_checkpointing_bitwise_equal_store_all():
    shape = (6, 5, 7)
    v = inputs.varcoef3d(shape=shape)
    a = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, 20, 20)
    for m in (1, 3, 7):
        b = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, False, 0.0, 20, m)
        assert a[0] == b[0]
        assert np.array_equal(a[2], b[2]) and np.array_equal(a[3], b[3])


def test_adjoint_threads_bitwise():
    shape = (9, 6, 5)
    v = inputs.varcoef3d(shape=shape)
    for periodic in (False, True):
        r1 = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, periodic, 0.0, 8, 3, threads=1)
        r4 = oracle.varcoef7_gradient(v.u0, v.kappa, v.target, periodic, 0.0, 8, 3, threads=4)
        assert np.array_equal(r1[2], r4[2]) and np.array_equal(r1[3], r4[3])


# ---------------------------------------------------------------- wave / leapfrog
def test_taylor_coefficients():
    """The solved coefficients satisfy the moment conditions (checked here by
    direct summation) and the symbol a_0 + 2 sum a_j cos(j t) matches -t^2 to
    8th order."""
    a = taylor_second_derivative_coeffs(4)
    for q in range(0, 5):
        mom = (a[0] if q == 0 else 0) + 2 * sum(a[j] * Fraction(j) ** (2 * q) for j in range(1, 5))
        assert mom == (2 if q == 1 else 0)
    af = [float(x) for x in a]
    for t in (0.05, 0.1, 0.2):
        sym = af[0] + 2 * sum(af[j] * math.cos(j * t) for j in range(1, 5))
        assert abs(sym + t * t) < 0.1 * t ** 10
    assert abs(af[0] + 205 / 72) < 1e-15 and abs(af[4] + 1 / 560) < 1e-18


def _lap8(u, a, periodic):
    """Radius-4 star Laplacian by array shifts (zero ghosts or wrap)."""
    out = 3 * a[0] * u
    for ax in range(3):
        for j in range(1, 5):
            if periodic:
                out = out + a[j] * (np.roll(u, -j, axis=ax) + np.roll(u, j, axis=ax))
            else:
                pad = [(0, 0)] * 3
                pad[ax] = (4, 4)
                up = np.pad(u, pad)
                sl_p = [slice(None)] * 3
                sl_m = [slice(None)] * 3
                sl_p[ax] = slice(4 + j, 4 + j + u.shape[ax])
                sl_m[ax] = slice(4 - j, 4 - j + u.shape[ax])
                out = out + a[j] * (up[tuple(sl_p)] + up[tuple(sl_m)])
    return out


def test_wave_plane_wave_recurrence():
    """Periodic, constant m: a cosine mode obeys the scalar recurrence
    g_{n+1} = (2 + m sigma) g_n - g_{n-1}, sigma = sum_d sym(theta_d)."""
    shape = (16, 12, 20)
    a = [float(x) for x in taylor_second_derivative_coeffs(4)]
    k = (2, 1, 3)
    th = [2 * math.pi * kd / nd for kd, nd in zip(k, shape)]
    mode = (np.cos(th[0] * np.arange(shape[0]))[:, None, None] *
            np.cos(th[1] * np.arange(shape[1]))[None, :, None] *
            np.cos(th[2] * np.arange(shape[2]))[None, None, :])
    sigma = sum(a[0] + 2 * sum(a[j] * math.cos(j * t) for j in range(1, 5)) for t in th)
    mval = 0.09
    g_nm1, g_n = 0.8, 1.0
    steps = 57
    un, unm1 = oracle.wave25(g_n * mode, g_nm1 * mode, np.full(shape, mval), a, None, None,
                             True, 0.0, steps)
    for _ in range(steps):
        g_nm1, g_n = g_n, (2 + mval * sigma) * g_n - g_nm1
    assert oracle.normwise_error(un, g_n * mode) < 1e-12
    assert oracle.normwise_error(unm1, g_nm1 * mode) < 1e-12


def test_wave_source_injection():
    shape = (11, 11, 11)
    a = [float(x) for x in taylor_second_derivative_coeffs(4)]
    m = np.full(shape, 0.05)
    src = (5, 5, 5)
    s = [0.7, -0.2]
    z = np.zeros(shape)
    u1, u0 = oracle.wave25(z, z, m, a, src, s, False, 0.0, 1)
    e = np.zeros(shape)
    e[src] = 0.7
    assert np.array_equal(u1, e) and np.array_equal(u0, z)
    u2, u1b = oracle.wave25(z, z, m, a, src, s, False, 0.0, 2)
    expect = 2 * e + m * _lap8(e, a, False)
    expect[src] += -0.2
    assert np.array_equal(u1b, e)
    assert oracle.normwise_error(u2, expect) < 1e-15


def test_wave_energy_conserved():
    """Dirichlet-zero, layered m, no source: the discrete leapfrog energy
    E = (u1-u0)^T M^-1 (u1-u0) - u1^T L u0 is constant."""
    shape = (12, 9, 10)
    a = [float(x) for x in taylor_second_derivative_coeffs(4)]
    rng = np.random.default_rng(2)
    m = np.repeat(rng.uniform(0.02, 0.15, size=shape[0]), shape[1] * shape[2]).reshape(shape)
    u_nm1 = rng.standard_normal(shape)
    u_n = u_nm1 + 0.1 * rng.standard_normal(shape)

    def energy(u1, u0):
        d = u1 - u0
        return float(np.sum(d * d / m) - np.sum(u1 * _lap8(u0, a, False)))

    e0 = energy(u_n, u_nm1)
    cur, old = u_n, u_nm1
    for _ in range(6):
        cur, old = oracle.wave25(cur, old, m, a, None, None, False, 0.0, 5)
        assert abs(energy(cur, old) - e0) < 1e-11 * abs(e0)


def test_wave_matches_shift_formula_dirichlet():
    """Variable m, Dirichlet: the oracle's gather equals the update written
    with array shifts on a zero-padded copy (independent indexing)."""
    shape = (7, 9, 8)
    a = [float(x) for x in taylor_second_derivative_coeffs(4)]
    rng = np.random.default_rng(4)
    m = rng.uniform(0.01, 0.15, size=shape)
    un, unm1 = rng.standard_normal(shape), rng.standard_normal(shape)
    got, prev = oracle.wave25(un, unm1, m, a, (3, 4, 2), [0.5], False, 0.0, 1)
    expect = 2 * un - unm1 + m * _lap8(un, a, False)
    expect[3, 4, 2] += 0.5
    assert np.array_equal(prev, un)
    assert oracle.normwise_error(got, expect) < 1e-14


# ---------------------------------------------------------------- reductions / threads / fp32
def test_reduce_matches_fsum():
    rng = np.random.default_rng(8)
    a = rng.standard_normal(10007)
    b = rng.standard_normal(10007)
    s, q, mx = oracle.reduce(a, b)
    d = a - b
    # recursive summation error bound |s - exact| <= (n-1) u sum|d_i|
    u = 2.0 ** -53
    assert abs(s - math.fsum(d)) <= (d.size - 1) * u * math.fsum(np.abs(d))
    assert abs(q - math.fsum(d * d)) <= d.size * u * math.fsum(d * d)
    assert mx == float(np.max(np.abs(d)))
    assert oracle.reduce(np.array([3.0, -4.0]))[1] == 25.0


def test_threads_bitwise_identical():
    u0 = inputs.heat3d(shape=(10, 12, 9)).u0
    offs, w = seven_point(0.1)
    r1 = oracle.sweep_const(u0, offs, w, True, 0.0, 7, threads=1)
    r4 = oracle.sweep_const(u0, offs, w, True, 0.0, 7, threads=4)
    assert np.array_equal(r1, r4)


def test_single_precision_build_same_definition():
    """The float build evaluates the same definition: close to the double
    result at float accuracy, but not bitwise equal."""
    u0 = inputs.heat2d(shape=(33, 40))
    offs, w = five_point(0.2)
    r64 = oracle.sweep_const(u0, offs, w, False, 0.0, 50)
    r32 = oracle.sweep_const(u0, offs, w, False, 0.0, 50, dtype=np.float32)
    err = oracle.normwise_error(r32, r64)
    assert r32.dtype == np.float32
    assert 1e-9 < err < 1e-5


# ---------------------------------------------------------------- arbitrary Dirichlet rings
def _padded(interior, r, ring):
    """Pad `interior` by r cells per side and fill the ring from ring(index)."""
    shape = tuple(s + 2 * r for s in interior.shape)
    u = np.empty(shape)
    for p in np.ndindex(*shape):
        u[p] = ring(p)
    u[tuple(slice(r, r + s) for s in interior.shape)] = interior
    return u


@pytest.mark.parametrize("shape,offsets,weights,r", [
    ((9, 7), [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4, 1),
    ((5, 6, 7), inputs.OFFSETS_7PT, [0.4] + [0.1] * 6, 1),
    ((8, 9), [(0, 0), (-2, 1), (1, -2), (0, 2), (2, 0)], [0.3, 0.1, 0.25, -0.15, 0.2], 2),
])
def test_ghost_sweep_uniform_ring_equals_constant_boundary(shape, offsets, weights, r):
    """A ring holding one value is the constant Dirichlet boundary of the C
    oracle: two independent implementations, the same operation order."""
    rng = np.random.default_rng(21)
    u0 = rng.random(shape)
    got = oracle.sweep_ghosts(_padded(u0, r, lambda p: 0.7), r, offsets, weights, 9)
    ref = oracle.sweep_const(u0, offsets, weights, False, 0.7, 9)
    assert np.array_equal(got[tuple(slice(r, r + s) for s in shape)], ref)
    ring = np.ones(got.shape, dtype=bool)
    ring[tuple(slice(r, r + s) for s in shape)] = False
    assert np.all(got[ring] == 0.7)


@pytest.mark.parametrize("shape,offsets,weights", [
    ((9, 7), [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4),
    ((6, 5, 7), inputs.OFFSETS_7PT[1:], [1 / 6] * 6),
])
def test_ghost_sweep_linear_ring_is_a_fixed_point(shape, offsets, weights):
    """A linear function is discretely harmonic: with its values on the ring
    and in the interior, the neighbour average leaves it unchanged."""
    coef = np.array([0.3, -1.1, 0.7][:len(shape)])
    f = lambda p: 2.0 + float(np.dot(coef, p))  # noqa: E731
    u = _padded(np.zeros(shape), 1, f)
    u[tuple(slice(1, 1 + s) for s in shape)] = np.array([f(tuple(i + 1 for i in p)) for p in np.ndindex(*shape)]
                                                       ).reshape(shape)
    got = oracle.sweep_ghosts(u, 1, offsets, weights, 25)
    assert np.max(np.abs(got - u)) <= 1e-13


def test_ghost_sweep_converges_to_the_discrete_dirichlet_solution():
    """Jacobi from a zero interior with a linear ring converges to the
    linear function (the unique discrete harmonic extension of the ring);
    the error contracts by the spectral radius (cos(pi/11) + cos(pi/9)) / 2
    per step, < 1e-10 after 600 steps on a 10 x 8 interior."""
    f = lambda p: 1.0 + 0.5 * p[0] - 0.25 * p[1]  # noqa: E731
    u = _padded(np.zeros((10, 8)), 1, f)
    got = oracle.sweep_ghosts(u, 1, [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4, 600)
    want = np.array([[f((y, x)) for x in range(10)] for y in range(12)])
    assert np.max(np.abs(got - want)) <= 1e-10


def test_ghost_sweep_vs_assembled_operator():
    """Brute force on a tiny grid with random ring values: u_{t+1} = A u_t + b
    with b the weighted ring values each point reaches, assembled point by
    point from the neighbour list."""
    rng = np.random.default_rng(22)
    shape, r = (4, 5), 2
    offsets = [(0, 0), (-2, 1), (1, -2), (0, 2), (2, 0), (-1, -1)]
    weights = [0.3, 0.1, 0.25, -0.15, 0.2, 0.05]
    u = rng.random((shape[0] + 2 * r, shape[1] + 2 * r))
    n = shape[0] * shape[1]
    A = np.zeros((n, n))
    b = np.zeros(n)
    for p in np.ndindex(*shape):
        ip = np.ravel_multi_index(p, shape)
        for o, w in zip(offsets, weights):
            q = (p[0] + o[0], p[1] + o[1])
            if 0 <= q[0] < shape[0] and 0 <= q[1] < shape[1]:
                A[ip, np.ravel_multi_index(q, shape)] += w
            else:
                b[ip] += w * u[q[0] + r, q[1] + r]
    x = u[r:-r, r:-r].reshape(-1)
    for _ in range(3):
        x = A @ x + b
    got = oracle.sweep_ghosts(u, r, offsets, weights, 3)
    assert np.max(np.abs(got[r:-r, r:-r].reshape(-1) - x)) <= 1e-14
    assert np.array_equal(got[:r], u[:r]) and np.array_equal(got[:, -r:], u[:, -r:])


# ---------------------------------------------------------------- zero-flux (Neumann) boundary
def _mirror(i, n):
    return -1 - i if i < 0 else (2 * n - 1 - i if i >= n else i)


@pytest.mark.parametrize("shape,k,a,steps", [((12, 9), (3, 2), 0.2, 15), ((7, 10), (0, 4), 0.15, 30)])
def test_neumann_cosine_mode_decay(shape, k, a, steps):
    """cos(pi k (i + 1/2) / n) per axis is an eigenvector of the 5-point
    operator with mirror-image ghosts; eigenvalue
    1 - 4a (sin^2(pi ky / (2 ny)) + sin^2(pi kx / (2 nx)))."""
    ny, nx = shape
    y = (np.arange(ny) + 0.5)[:, None]
    x = (np.arange(nx) + 0.5)[None, :]
    u0 = np.cos(np.pi * k[0] * y / ny) * np.cos(np.pi * k[1] * x / nx)
    lam = 1 - 4 * a * (np.sin(np.pi * k[0] / (2 * ny)) ** 2 + np.sin(np.pi * k[1] / (2 * nx)) ** 2)
    got = oracle.sweep_neumann(u0, inputs.OFFSETS_5PT, [1 - 4 * a] + [a] * 4, steps)
    assert np.max(np.abs(got - lam ** steps * u0)) <= 1e-13


def test_neumann_3d_cosine_mode_decay():
    shape, k, a, steps = (6, 9, 11), (1, 3, 5), 0.1, 12
    grids = np.meshgrid(*[np.arange(n) + 0.5 for n in shape], indexing="ij")
    u0 = np.prod([np.cos(np.pi * kk * g / n) for kk, g, n in zip(k, grids, shape)], axis=0)
    lam = 1 - 4 * a * sum(np.sin(np.pi * kk / (2 * n)) ** 2 for kk, n in zip(k, shape))
    got = oracle.sweep_neumann(u0, inputs.OFFSETS_7PT, [1 - 6 * a] + [a] * 6, steps)
    assert np.max(np.abs(got - lam ** steps * u0)) <= 1e-13


def test_neumann_conserves_the_sum_and_constants():
    """Zero flux through the boundary: symmetric weights summing to 1 keep
    sum(u); a constant field stays constant."""
    rng = np.random.default_rng(23)
    u0 = rng.random((9, 14, 11))
    got = oracle.sweep_neumann(u0, inputs.OFFSETS_7PT, [0.4] + [0.1] * 6, 40)
    assert abs(got.sum() - u0.sum()) <= 1e-12 * u0.sum()
    c = oracle.sweep_neumann(np.full((5, 8), 0.3), inputs.OFFSETS_5PT, [0.2] * 5, 25)
    assert np.max(np.abs(c - 0.3)) <= 1e-15


def test_neumann_vs_assembled_operator():
    """Brute force with asymmetric radius-2 offsets: the matrix assembled
    point by point with mirrored neighbour indices."""
    rng = np.random.default_rng(24)
    shape = (5, 6)
    offsets = [(0, 0), (-2, 1), (1, -2), (0, 2), (2, 0), (-1, -1)]
    weights = [0.3, 0.1, 0.25, -0.15, 0.2, 0.05]
    n = shape[0] * shape[1]
    A = np.zeros((n, n))
    for p in np.ndindex(*shape):
        ip = np.ravel_multi_index(p, shape)
        for o, w in zip(offsets, weights):
            q = (_mirror(p[0] + o[0], shape[0]), _mirror(p[1] + o[1], shape[1]))
            A[ip, np.ravel_multi_index(q, shape)] += w
    u0 = rng.random(shape)
    x = u0.reshape(-1)
    for _ in range(4):
        x = A @ x
    got = oracle.sweep_neumann(u0, offsets, weights, 4)
    assert np.max(np.abs(got.reshape(-1) - x)) <= 1e-14


def _neumann_matrix(shape, offsets, weights):
    n = int(np.prod(shape))
    A = np.zeros((n, n))
    for p in np.ndindex(*shape):
        ip = np.ravel_multi_index(p, shape)
        for o, w in zip(offsets, weights):
            q = tuple(_mirror(p[a] + o[a], shape[a]) for a in range(len(shape)))
            A[ip, np.ravel_multi_index(q, shape)] += w
    return A


@pytest.mark.parametrize("shape,offsets,weights", [
    ((5, 6), [(0, 0), (-2, 1), (1, -2), (0, 2), (2, 0), (-1, -1)], [0.3, 0.1, 0.25, -0.15, 0.2, 0.05]),
    ((4, 3, 5), [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)],
     [0.4, 0.05, 0.15, 0.1, 0.1, 0.12, 0.08]),
])
def test_neumann_transpose_is_the_assembled_transpose(shape, offsets, weights):
    """The zero-flux transpose equals A^T of the matrix assembled with
    mirrored indices (asymmetric offsets and weights, so A^T != A), and the
    dot-product identity <S x, y> = <x, S^T y> holds."""
    A = _neumann_matrix(shape, offsets, weights)
    rng = np.random.default_rng(25)
    y = rng.random(shape)
    got = oracle.neumann_transpose(y, offsets, weights)
    assert np.max(np.abs(got.reshape(-1) - A.T @ y.reshape(-1))) <= 1e-14
    x = rng.random(shape)
    sx = oracle.sweep_neumann(x, offsets, weights, 1)
    assert abs(np.sum(sx * y) - np.sum(x * got)) <= 1e-13 * abs(np.sum(sx * y))


def test_neumann_loss_gradient_finite_differences():
    """dL/du0 of L = 0.5 ||S^n u0 - t||^2 by central differences along random
    directions and single coordinates (the loss is quadratic, so central
    differences are exact up to rounding)."""
    rng = np.random.default_rng(26)
    shape = (6, 7, 5)
    offsets, weights = inputs.OFFSETS_7PT, [0.3, 0.1, 0.15, 0.12, 0.08, 0.13, 0.12]
    u0, t = rng.random(shape), rng.random(shape)
    _, _, g = oracle.neumann_loss_gradient(u0, t, offsets, weights, 9)
    L = lambda u: oracle.neumann_loss_gradient(u, t, offsets, weights, 9)[0]  # noqa: E731
    eps = 1e-4
    for _ in range(4):
        d = rng.standard_normal(shape)
        d /= np.linalg.norm(d)
        fd = (L(u0 + eps * d) - L(u0 - eps * d)) / (2 * eps)
        assert abs(fd - np.sum(g * d)) <= 1e-8 * abs(fd) + 1e-12
    for p in ((0, 0, 0), (5, 6, 4), (2, 3, 1)):
        e = np.zeros(shape)
        e[p] = 1.0
        fd = (L(u0 + eps * e) - L(u0 - eps * e)) / (2 * eps)
        assert abs(fd - g[p]) <= 1e-8 * abs(fd) + 1e-12


# ---------------------------------------------------------------- conservative face-averaged operator
def _cons_matrix(shape, kappa, periodic):
    """S assembled column by column from the oracle's step (boundary value 0,
    so the constant part vanishes)."""
    n = int(np.prod(shape))
    S = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        S[:, j] = oracle.cons_step(e.reshape(shape), kappa, periodic, 0.0).reshape(-1)
    return S


def _cons_rows(shape, kappa, periodic):
    """The same matrix written out row by row from the face rule (brute force)."""
    n = int(np.prod(shape))
    S = np.zeros((n, n))
    for p in np.ndindex(*shape):
        ip = np.ravel_multi_index(p, shape)
        S[ip, ip] += 1.0
        for ax in range(len(shape)):
            for s in (-1, 1):
                q = list(p)
                q[ax] += s
                if periodic:
                    q[ax] %= shape[ax]
                inside = 0 <= q[ax] < shape[ax]
                w = (kappa[p] + kappa[tuple(q)]) / 2 if inside else kappa[p]
                S[ip, ip] -= w
                if inside:
                    S[ip, np.ravel_multi_index(tuple(q), shape)] += w
    return S


@pytest.mark.parametrize("periodic", [False, True])
def test_cons_constant_kappa_is_the_heat_step(periodic):
    """kappa = c everywhere: the 7-point heat step (1 - 6c) u + c sum(neighbours)."""
    rng = np.random.default_rng(41)
    u0 = rng.random((7, 6, 9))
    got = oracle.cons_forward(u0, np.full(u0.shape, 0.11), periodic, 0.4, 12)
    ref = oracle.sweep_const(u0, inputs.OFFSETS_7PT, [1 - 6 * 0.11] + [0.11] * 6, periodic, 0.4, 12)
    assert np.max(np.abs(got - ref)) <= 1e-13


@pytest.mark.parametrize("periodic", [False, True])
def test_cons_matrix_is_symmetric_and_matches_the_face_rule(periodic):
    rng = np.random.default_rng(42)
    shape = (3, 4, 5)
    kappa = rng.uniform(0.0, 0.16, shape)
    S = _cons_matrix(shape, kappa, periodic)
    assert np.max(np.abs(S - _cons_rows(shape, kappa, periodic))) <= 1e-15
    assert np.max(np.abs(S - S.T)) <= 1e-15


def test_cons_periodic_conserves_the_sum_for_any_kappa():
    rng = np.random.default_rng(43)
    u0 = rng.random((10, 12, 8))
    kappa = np.clip(0.05 * np.exp(0.5 * rng.standard_normal(u0.shape)), 0, 0.16)
    got = oracle.cons_forward(u0, kappa, True, 0.0, 50)
    assert abs(got.sum() - u0.sum()) <= 1e-12 * u0.sum()
    c = oracle.cons_forward(np.full((5, 6), 0.7), kappa[0, :5, :6], False, 0.7, 20)
    assert np.max(np.abs(c - 0.7)) <= 1e-15


@pytest.mark.parametrize("periodic", [False, True])
def test_cons_transpose_equals_the_matrix_transpose(periodic):
    rng = np.random.default_rng(44)
    shape = (4, 3, 5)
    kappa = rng.uniform(0.0, 0.16, shape)
    lam = rng.standard_normal(shape)
    S = _cons_matrix(shape, kappa, periodic)
    got = oracle.cons_transpose(lam, kappa, periodic)
    assert np.max(np.abs(got.reshape(-1) - S.T @ lam.reshape(-1))) <= 1e-14


@pytest.mark.parametrize("periodic,bc", [(False, 0.3), (True, 0.0)])
def test_cons_gradient_central_differences(periodic, bc):
    """dL/du0 and dL/dkappa against central differences of the loss along
    random directions and single coordinates (FP64, 5 x 4 x 6, 6 steps)."""
    rng = np.random.default_rng(45)
    shape, steps = (5, 4, 6), 6
    u0 = rng.random(shape)
    kappa = rng.uniform(0.02, 0.15, shape)
    tgt = rng.random(shape)
    loss, _, du0, dk = oracle.cons_loss_gradient(u0, kappa, tgt, periodic, bc, steps)

    def L(u, k):
        return 0.5 * float(np.sum((oracle.cons_forward(u, k, periodic, bc, steps) - tgt) ** 2))

    for _ in range(4):
        d = rng.standard_normal(shape)
        eps = 1e-6
        fd_u = (L(u0 + eps * d, kappa) - L(u0 - eps * d, kappa)) / (2 * eps)
        fd_k = (L(u0, kappa + eps * d) - L(u0, kappa - eps * d)) / (2 * eps)
        assert abs(fd_u - np.sum(du0 * d)) <= 1e-7 * max(1.0, abs(fd_u))
        assert abs(fd_k - np.sum(dk * d)) <= 1e-7 * max(1.0, abs(fd_k))
    for idx in [(0, 0, 0), (4, 3, 5), (2, 1, 3), (0, 2, 5)]:
        e = np.zeros(shape)
        e[idx] = 1.0
        fd = (L(u0, kappa + 1e-6 * e) - L(u0, kappa - 1e-6 * e)) / 2e-6
        assert abs(fd - dk[idx]) <= 1e-7 * max(1.0, abs(fd))


# ---------------------------------------------------------------- lid-driven cavity flow
from oracle import cavity as cav  # noqa: E402

CAVP = cav.CavityParams(dx=0.05, dy=0.04, dt=0.001, rho=1.3, nu=0.1, nit=5, lid=1.0)


def _cavity_loops(u0, v0, p0, P, nsteps):
    """The same scheme written point by point with Python loops (brute force,
    tiny grids only)."""
    u, v, p = [np.array(a, dtype=np.float64) for a in (u0, v0, p0)]
    ny, nx = u.shape
    dx, dy, dt, rho, nu = P.dx, P.dy, P.dt, P.rho, P.nu
    for _ in range(nsteps):
        b = np.zeros_like(u)
        for j in range(1, ny - 1):
            for i in range(1, nx - 1):
                ux = (u[j, i + 1] - u[j, i - 1]) / (2 * dx)
                uy = (u[j + 1, i] - u[j - 1, i]) / (2 * dy)
                vx = (v[j, i + 1] - v[j, i - 1]) / (2 * dx)
                vy = (v[j + 1, i] - v[j - 1, i]) / (2 * dy)
                b[j, i] = rho * ((ux + vy) / dt - ux * ux - 2 * uy * vx - vy * vy)
        for _ in range(P.nit):
            pn = p.copy()
            for j in range(1, ny - 1):
                for i in range(1, nx - 1):
                    p[j, i] = ((pn[j, i + 1] + pn[j, i - 1]) * dy * dy + (pn[j + 1, i] + pn[j - 1, i]) * dx * dx
                               - b[j, i] * dx * dx * dy * dy) / (2 * (dx * dx + dy * dy))
            for j in range(ny):
                p[j, nx - 1] = p[j, nx - 2]
            for i in range(nx):
                p[0, i] = p[1, i]
            for j in range(ny):
                p[j, 0] = p[j, 1]
            for i in range(nx):
                p[ny - 1, i] = 0.0
        un, vn = u.copy(), v.copy()
        for j in range(1, ny - 1):
            for i in range(1, nx - 1):
                c, w, s = un[j, i], un[j, i - 1], un[j - 1, i]
                u[j, i] = (c - c * dt / dx * (c - w) - vn[j, i] * dt / dy * (c - s)
                           - dt / (2 * rho * dx) * (p[j, i + 1] - p[j, i - 1])
                           + nu * (dt / dx ** 2 * (un[j, i + 1] - 2 * c + w) + dt / dy ** 2 * (un[j + 1, i] - 2 * c + s)))
                c, w, s = vn[j, i], vn[j, i - 1], vn[j - 1, i]
                v[j, i] = (c - un[j, i] * dt / dx * (c - w) - c * dt / dy * (c - s)
                           - dt / (2 * rho * dy) * (p[j + 1, i] - p[j - 1, i])
                           + nu * (dt / dx ** 2 * (vn[j, i + 1] - 2 * c + w) + dt / dy ** 2 * (vn[j + 1, i] - 2 * c + s)))
        u[0, :] = u[:, 0] = u[:, -1] = 0.0
        u[-1, :] = P.lid
        v[0, :] = v[-1, :] = v[:, 0] = v[:, -1] = 0.0
    return u, v, p


def test_cavity_vectorised_equals_point_loops():
    rng = np.random.default_rng(61)
    shape = (7, 9)
    u0, v0, p0 = (0.2 * rng.standard_normal(shape) for _ in range(3))
    got = cav.cavity_run(u0, v0, p0, CAVP, 3)
    ref = _cavity_loops(u0, v0, p0, CAVP, 3)
    for g, r in zip(got, ref):
        assert np.max(np.abs(g - r)) <= 1e-12 * max(1.0, np.max(np.abs(r)))


def test_cavity_rest_state_stays_at_rest():
    z = np.zeros((11, 13))
    P = cav.CavityParams(dx=0.1, dy=0.1, dt=0.001, lid=0.0, nit=20)
    for a in cav.cavity_run(z, z, z, P, 5):
        assert np.all(a == 0.0)


def test_cavity_pressure_source_of_linear_fields():
    """u = a x + c y, v = d x + e y: central differences are exact, so
    b = rho ((a + e) / dt - a^2 - 2 c d - e^2) at every interior point."""
    a, c, d, e = 0.7, -0.3, 0.4, 1.1
    y, x = np.meshgrid(np.arange(8) * CAVP.dy, np.arange(10) * CAVP.dx, indexing="ij")
    b = cav.pressure_source(a * x + c * y, d * x + e * y, CAVP)
    want = CAVP.rho * ((a + e) / CAVP.dt - a * a - 2 * c * d - e * e)
    assert np.max(np.abs(b[1:-1, 1:-1] - want)) <= 1e-9 * abs(want)
    assert np.all(b[0] == 0) and np.all(b[:, -1] == 0)


def test_cavity_pressure_iteration_solves_the_discrete_poisson_problem():
    """At the fixed point of the Jacobi iteration, the five-point Laplacian of
    p (spacings dx != dy) equals b at every interior point, and the boundary
    rule holds."""
    rng = np.random.default_rng(62)
    shape = (9, 7)
    b = np.zeros(shape)
    b[1:-1, 1:-1] = rng.standard_normal((7, 5))
    p = cav.pressure_iterations(np.zeros(shape), b, CAVP, nit=6000)
    lap = ((p[1:-1, 2:] - 2 * p[1:-1, 1:-1] + p[1:-1, :-2]) / CAVP.dx ** 2
           + (p[2:, 1:-1] - 2 * p[1:-1, 1:-1] + p[:-2, 1:-1]) / CAVP.dy ** 2)
    assert np.max(np.abs(lap - b[1:-1, 1:-1])) <= 1e-8 * np.max(np.abs(b))
    assert np.all(p[-1] == 0) and np.array_equal(p[1:-1, 0], p[1:-1, 1]) and np.array_equal(p[0, 1:-1], p[1, 1:-1])


def test_cavity_velocity_update_of_simple_fields():
    """Uniform u = U, v = V with p = g x + h y: advection and diffusion vanish
    and the pressure gradient is exact, so u' = U - dt g / rho and
    v' = V - dt h / rho inside.  u = a x with v = 0 and p = 0: the backward
    difference of a linear field is exact, so u' = u - dt a u inside."""
    y, x = np.meshgrid(np.arange(8) * CAVP.dy, np.arange(10) * CAVP.dx, indexing="ij")
    U, V, g, h = 0.3, -0.2, 2.0, -1.5
    u2, v2 = cav.velocity_update(np.full(x.shape, U), np.full(x.shape, V), g * x + h * y, CAVP)
    assert np.max(np.abs(u2[1:-1, 1:-1] - (U - CAVP.dt * g / CAVP.rho))) <= 1e-14
    assert np.max(np.abs(v2[1:-1, 1:-1] - (V - CAVP.dt * h / CAVP.rho))) <= 1e-14
    assert np.all(u2[-1] == CAVP.lid) and np.all(u2[0] == 0) and np.all(v2[:, 0] == 0)
    a = 0.8
    u2, v2 = cav.velocity_update(a * x, np.zeros(x.shape), np.zeros(x.shape), CAVP)
    assert np.max(np.abs(u2[1:-1, 1:-1] - (a * x - CAVP.dt * a * a * x)[1:-1, 1:-1])) <= 1e-14
    assert np.all(v2 == 0)


def test_sweep_const_into_equals_sweep_const():
    """The resident-array wrapper used for timing runs the same C loop: bit
    for bit the result of sweep_const, for even and odd step counts."""
    rng = np.random.default_rng(41)
    u0 = rng.random((6, 7, 9))
    w = [0.4] + [0.1] * 6
    for n in (1, 2, 5):
        ref = oracle.sweep_const(u0, inputs.OFFSETS_7PT, w, True, 0.0, n)
        u = u0.copy()
        oracle.sweep_const_into(u, np.empty_like(u), inputs.OFFSETS_7PT, w, True, 0.0, n)
        assert np.array_equal(u, ref)
