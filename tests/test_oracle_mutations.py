"""Planted mistakes in the CPU oracle must be caught by its pins.

Each mutant is a copy of oracle/stencil_oracle.c with one plausible slip (a
dropped term, a wrong sign, a wrong index or axis, a transposed operand),
compiled to a temporary library and swapped in for the double-precision
oracle while a few pins from test_oracle_pins.py run.  At least one of them
must fail.  Nothing here touches a GPU.
"""
import contextlib
import ctypes
import os
import subprocess
import sys
import tempfile
import types

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "stencil_oracle.c")

MUTANTS = {
    "sweep drops the last neighbour": (
        "for (int k = 0; k < npts; ++k) {\n                        REAL v",
        "for (int k = 0; k < npts - 1; ++k) {\n                        REAL v",
        ["matrix", "golden", "decay"]),
    "Dirichlet ghost ignores bc_value": (
        "        return bc_value;", "        return (REAL)0;", ["matrix", "golden"]),
    "sweep mixes up the z and x offsets": (
        "orc_read(src, nz, ny, nx, z + off[3 * k], y + off[3 * k + 1],\n                                          x + off[3 * k + 2]",
        "orc_read(src, nz, ny, nx, z + off[3 * k + 2], y + off[3 * k + 1],\n                                          x + off[3 * k]",
        ["matrix"]),
    "periodic wrap off by one": (
        "    while (i < 0) i += n;", "    while (i < 0) i += n - 1;", ["matrix", "fourier", "conserve"]),
    "variable diffusion centre weight 1 - 5 kappa": (
        "dst[p] = ((REAL)1 - (REAL)6 * k) * src[p] + k * nb;",
        "dst[p] = ((REAL)1 - (REAL)5 * k) * src[p] + k * nb;", ["varmatrix"]),
    "variable diffusion drops the z+1 neighbour": (
        "nb = nb + orc_read(src, nz, ny, nx, z + 1, y, x, periodic, bc);\n                    REAL k",
        "REAL k", ["varmatrix"]),
    "adjoint uses the receiver's kappa (transposed operand)": (
        "lout[q] = lout[q] + k * lp;", "lout[q] = lout[q] + kappa[q] * lp;", ["transpose", "fd"]),
    "gradient term has the wrong sign": (
        "gk[p] = gk[p] + lp * (nb - (REAL)6 * ut[p]);", "gk[p] = gk[p] + lp * (nb + (REAL)6 * ut[p]);", ["fd"]),
    "adjoint centre weight 1 - 6 kappa dropped to 1": (
        "lout[p] = lout[p] + ((REAL)1 - (REAL)6 * k) * lp;", "lout[p] = lout[p] + lp;", ["transpose", "fd"]),
    "leapfrog drops u^{n-1}": (
        "REAL v = (REAL)2 * c - old[p] + m[p] * lap;", "REAL v = (REAL)2 * c + m[p] * lap;",
        ["planewave", "energy", "shift"]),
    "wave star reads z - j + 1": (
        "orc_read(cur, nz, ny, nx, z - j, y, x, periodic, bc));",
        "orc_read(cur, nz, ny, nx, z - j + 1, y, x, periodic, bc));", ["planewave", "shift"]),
    "wave source added to the wrong step": (
        "if (p == src) v = v + (REAL)s[st];", "if (p == src) v = v + (REAL)s[st + 1];", ["source"]),
    "reduction sums |d| instead of d^2": (
        "q = q + d * d;", "q = q + (d < 0 ? -d : d);", ["reduce"]),
}

PINS = {
    "matrix": lambda: [pins.test_sweep_vs_assembled_matrix(s, p) for s in [(6, 7), (4, 5, 3)] for p in (False, True)],
    "golden": pins.test_example1_golden_exact,
    "decay": lambda: pins.test_dirichlet_sine_mode_decay((9, 13), (2, 3), 0.2, 17),
    "fourier": pins.test_periodic_2d_fourier_decay,
    "conserve": pins.test_periodic_sum_conserved,
    "varmatrix": lambda: [pins.test_varcoef7_vs_assembled_matrix(p) for p in (False, True)],
    "transpose": lambda: [pins.test_adjoint_equals_matrix_transpose(p) for p in (False, True)],
    "fd": pins.test_gradient_central_differences,
    "planewave": pins.test_wave_plane_wave_recurrence,
    "energy": pins.test_wave_energy_conserved,
    "shift": pins.test_wave_matches_shift_formula_dirichlet,
    "source": pins.test_wave_source_injection,
    "reduce": pins.test_reduce_matches_fsum,
}


@contextlib.contextmanager
def mutant_oracle(old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "mut.c")
        so = os.path.join(d, "mut.so")
        open(c, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                               "-DREAL=double", "-DORC_SUFFIX=_f64", c, "-o", so])
        oracle.build()
        saved = oracle._loaded.get(np.float64)
        oracle._loaded[np.float64] = ctypes.CDLL(so)
        try:
            yield
        finally:
            if saved is None:
                oracle._loaded.pop(np.float64, None)
            else:
                oracle._loaded[np.float64] = saved


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    old, new, which = MUTANTS[name]
    caught = []
    with mutant_oracle(old, new):
        for key in which:
            try:
                PINS[key]()
            except Exception as e:  # an assertion, or a numerical blow-up
                caught.append((key, type(e).__name__))
    assert caught, f"no pin caught the planted mistake: {name}"


def test_unmutated_oracle_passes_the_same_pins():
    for key, fn in PINS.items():
        fn()


# ------------------------------------------------ the numpy ghost-ring and Neumann sweeps
GHOST_SRC = os.path.join(os.path.dirname(oracle.__file__), "ghosts.py")

GHOST_MUTANTS = {
    "ghost sweep drops the last neighbour": ("for o, wk in zip(offs, w):", "for o, wk in zip(offs[:-1], w[:-1]):"),
    "ghost sweep reads the offset with the wrong sign": ("slice(r + c, r + c + m)", "slice(r - c, r - c + m)"),
    "ghost sweep transposes the offset axes": ("for c, m in zip(o, n))", "for c, m in zip(o[::-1], n))"),
    "ghost sweep never swaps the arrays": ("u, tmp = tmp, u", "tmp = tmp"),
    "ghost sweep reads the output array": ("tmp[inner] = _sweep_once(u,", "tmp[inner] = _sweep_once(tmp,"),
    "Neumann mirror skips the edge cell (reflect)": ('mode="symmetric"', 'mode="reflect"'),
    "Neumann ghosts wrap around (periodic)": ('mode="symmetric"', 'mode="wrap"'),
    "Neumann ghosts held at zero (Dirichlet)": ('mode="symmetric"', 'mode="constant"'),
    "Neumann transpose gathers instead of scattering": (
        "np.add.at(out, tgt, dtype(wk) * lam)", "out += dtype(wk) * lam[tgt]"),
    "Neumann transpose reflects without the edge cell": (
        "np.where(i < 0, -1 - i,", "np.where(i < 0, -i,"),
    "Neumann transpose loses repeated targets": (
        "np.add.at(out, tgt, dtype(wk) * lam)", "out[tgt] += dtype(wk) * lam"),
}

GHOST_PINS = [
    lambda: [pins.test_ghost_sweep_uniform_ring_equals_constant_boundary(*a) for a in [
        ((9, 7), [(-1, 0), (1, 0), (0, -1), (0, 1)], [0.25] * 4, 1),
        ((8, 9), [(0, 0), (-2, 1), (1, -2), (0, 2), (2, 0)], [0.3, 0.1, 0.25, -0.15, 0.2], 2)]],
    pins.test_ghost_sweep_converges_to_the_discrete_dirichlet_solution,
    pins.test_ghost_sweep_vs_assembled_operator,
    lambda: pins.test_neumann_cosine_mode_decay((12, 9), (3, 2), 0.2, 15),
    pins.test_neumann_conserves_the_sum_and_constants,
    pins.test_neumann_vs_assembled_operator,
    lambda: [pins.test_neumann_transpose_is_the_assembled_transpose(*a) for a in [
        ((5, 6), [(0, 0), (-2, 1), (1, -2), (0, 2), (2, 0), (-1, -1)], [0.3, 0.1, 0.25, -0.15, 0.2, 0.05]),
        ((4, 3, 5), [(0, 0, 0), (-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)],
         [0.4, 0.05, 0.15, 0.1, 0.1, 0.12, 0.08])]],
    pins.test_neumann_loss_gradient_finite_differences,
]


@pytest.mark.parametrize("name", sorted(GHOST_MUTANTS))
def test_ghost_pins_catch_planted_mistake(name, monkeypatch):
    old, new = GHOST_MUTANTS[name]
    src = open(GHOST_SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    ns = {}
    exec(compile(src.replace(old, new), "ghosts_mutant", "exec"), ns)
    monkeypatch.setattr(oracle, "sweep_ghosts", ns["sweep_ghosts"])
    monkeypatch.setattr(oracle, "sweep_neumann", ns["sweep_neumann"])
    monkeypatch.setattr(oracle, "neumann_transpose", ns["neumann_transpose"])
    monkeypatch.setattr(oracle, "neumann_loss_gradient", ns["neumann_loss_gradient"])
    caught = []
    for fn in GHOST_PINS:
        try:
            fn()
        except Exception as e:
            caught.append(type(e).__name__)
    assert caught, f"no pin caught the planted mistake: {name}"


def test_unmutated_ghost_sweep_passes_the_same_pins():
    for fn in GHOST_PINS:
        fn()


# ------------------------------------------------ the conservative operator
CONS_SRC = os.path.join(os.path.dirname(oracle.__file__), "conservative.py")

CONS_MUTANTS = {
    "face coefficient is kappa[p] alone": ("w = (kappa + _shift(kp, o, u.shape)) / 2\n        acc",
                                           "w = kappa + 0 * _shift(kp, o, u.shape)\n        acc"),
    "ghost faces padded with zero kappa": ('return np.pad(a, 1, mode="edge")', 'return np.pad(a, 1, mode="constant")'),
    "transpose forgets the diagonal": ("out -= w * lam", "out -= 0 * w * lam"),
    "gradient sends nothing to the neighbour": ("_scatter_add(g, np.where(inner, 0.5 * t, 0.0), o, periodic)",
                                                "pass"),
    "gradient ghost face weighted one half": ("g += np.where(inner, 0.5 * t, t)", "g += 0.5 * t"),
}

CONS_PINS = [
    lambda: [pins.test_cons_constant_kappa_is_the_heat_step(p) for p in (False, True)],
    lambda: [pins.test_cons_matrix_is_symmetric_and_matches_the_face_rule(p) for p in (False, True)],
    pins.test_cons_periodic_conserves_the_sum_for_any_kappa,
    lambda: [pins.test_cons_transpose_equals_the_matrix_transpose(p) for p in (False, True)],
    lambda: [pins.test_cons_gradient_central_differences(p, b) for p, b in ((False, 0.3), (True, 0.0))],
]


@pytest.mark.parametrize("name", sorted(CONS_MUTANTS))
def test_conservative_pins_catch_planted_mistake(name, monkeypatch):
    old, new = CONS_MUTANTS[name]
    src = open(CONS_SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    ns = {}
    exec(compile(src.replace(old, new), "conservative_mutant", "exec"), ns)
    for fn in ("cons_step", "cons_forward", "cons_transpose", "cons_loss_gradient"):
        monkeypatch.setattr(oracle, fn, ns[fn])
    caught = []
    for pin in CONS_PINS:
        try:
            pin()
        except Exception as e:
            caught.append(type(e).__name__)
    assert caught, f"no pin caught the planted mistake: {name}"


def test_unmutated_conservative_oracle_passes_the_same_pins():
    for pin in CONS_PINS:
        pin()


# ------------------------------------------------ the cavity flow
CAV_SRC = os.path.join(os.path.dirname(oracle.__file__), "cavity.py")

CAV_MUTANTS = {
    "pressure iteration swaps dx and dy": ("((pe + pw) * dy2 + (pnn + ps) * dx2", "((pe + pw) * dx2 + (pnn + ps) * dy2"),
    "pressure source drops the factor 2 of the cross term": ("- 2 * uy * vx", "- uy * vx"),
    "pressure source takes uy along x": ("uy = (un - us) / (2 * P.dy)", "uy = (ue - uw) / (2 * P.dy)"),
    "velocity pressure gradient with the wrong sign": ("- P.dt / (2 * P.rho * P.dx) * (pe - pw)",
                                                       "+ P.dt / (2 * P.rho * P.dx) * (pe - pw)"),
    "v advected by v along x": ("(vc - uc * cx * (vc - vw)", "(vc - vc * cx * (vc - vw)"),
    "boundary rule: bottom row copies itself": ("p[0, :] = p[1, :]", "p[0, :] = p[0, :]"),
}


@pytest.mark.parametrize("name", sorted(CAV_MUTANTS))
def test_cavity_pins_catch_planted_mistake(name, monkeypatch):
    old, new = CAV_MUTANTS[name]
    src = open(CAV_SRC).read()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    mod = types.ModuleType("cavity_mutant")
    monkeypatch.setitem(sys.modules, "cavity_mutant", mod)   # dataclasses look their module up
    exec(compile(src.replace(old, new), "cavity_mutant", "exec"), mod.__dict__)
    ns = mod.__dict__
    for fn in ("pressure_source", "pressure_iterations", "velocity_update", "cavity_run", "pressure_boundary"):
        monkeypatch.setattr(pins.cav, fn, ns[fn])
    caught = []
    for pin in (pins.test_cavity_vectorised_equals_point_loops, pins.test_cavity_pressure_source_of_linear_fields,
                pins.test_cavity_pressure_iteration_solves_the_discrete_poisson_problem,
                pins.test_cavity_velocity_update_of_simple_fields):
        try:
            pin()
        except Exception as e:
            caught.append(type(e).__name__)
    assert caught, f"no pin caught the planted mistake: {name}"

