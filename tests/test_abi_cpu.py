"""The C-ABI library builds, loads and exports every entry point declared in
include/stencil.h; host-side validation and layout work without a GPU (no
compute call is made here)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

from paper_2512_19851_gb300 import abi, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "stencil.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:st_status|const char\s*\*)\s*(\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("stencil_create", "stencil_step", "stencil_adjoint", "stencil_batch_create",
                 "stencil_batch_step", "stencil_last_error"):
        assert must in names
    assert set(names) == set(abi.SIGNATURES), "binding and header disagree"


def test_library_exports_every_symbol():
    path = build.build()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    lib = ctypes.CDLL(path)
    for n in declared_functions():
        assert getattr(lib, n) is not None


def test_version_and_empty_error():
    assert "sm_103a" in abi.stencil_version()
    assert isinstance(abi.stencil_last_error(), str)


def _create(**kw):
    args = dict(ndim=3, dims=(8, 9, 10), radius=0, offsets=[(0, 0, 0), (0, 0, 1), (0, 0, -1)],
                alpha=[0.5, 0.25, 0.25], beta=None, bc=abi.ST_DIRICHLET, bc_value=0.0, dtype=abi.ST_F32,
                time_levels=1, flags=0)
    args.update(kw)
    return abi.stencil_create(**args)


def test_layout_rules():
    for dtype, es in ((abi.ST_F32, 4), (abi.ST_F64, 8)):
        for r in (1, 2, 4):
            h = _create(dtype=dtype, radius=r, dims=(5, 7, 13))
            pd, org, n = abi.stencil_layout(h, 3)
            assert org[0] == r and org[1] == r
            assert org[2] >= r and (org[2] * es) % 16 == 0
            assert (pd[2] * es) % 16 == 0 and pd[2] >= org[2] + 13 + r
            assert pd[0] == 5 + 2 * r and pd[1] == 7 + 2 * r
            assert n == pd[0] * pd[1] * pd[2]
            abi.stencil_destroy(h)
    h = abi.stencil_create(2, (6, 11), 0, [(0, 0), (1, 0), (-1, 0)], [1, 0, 0], dtype=abi.ST_F64)
    pd, org, n = abi.stencil_layout(h, 2)
    assert pd[0] == 8 and org == (1, 2) and n == pd[0] * pd[1]
    abi.stencil_destroy(h)


def test_radius_is_derived_from_offsets():
    h = _create(offsets=[(0, 0, 0), (0, 3, 0), (-2, 0, 0)], alpha=[1, 0, 0])
    assert abi.stencil_info(h)[0] == 3
    abi.stencil_destroy(h)
    h = _create(radius=5)
    assert abi.stencil_info(h)[0] == 5
    abi.stencil_destroy(h)


@pytest.mark.parametrize("kw,code", [
    (dict(ndim=4), abi.ST_ERR_ARG),
    (dict(dims=(0, 4, 4)), abi.ST_ERR_ARG),
    (dict(radius=1, offsets=[(0, 0, 2)], alpha=[1.0]), abi.ST_ERR_ARG),
    (dict(offsets=[(0, 0, 9)], alpha=[1.0]), abi.ST_ERR_ARG),
    (dict(bc=abi.ST_PERIODIC, dims=(8, 9, 2), offsets=[(0, 0, 2)], alpha=[1.0]), abi.ST_ERR_ARG),
    (dict(dtype=7), abi.ST_ERR_ARG),
    (dict(time_levels=3), abi.ST_ERR_ARG),
    (dict(flags=16), abi.ST_ERR_ARG),
    (dict(bc=abi.ST_PERIODIC, flags=abi.ST_FLAG_CALLER_GHOSTS), abi.ST_ERR_ARG),
    (dict(alpha=[float("nan"), 0.25, 0.25]), abi.ST_ERR_ARG),
])
def test_create_rejects_bad_arguments(kw, code):
    with pytest.raises(abi.StencilError) as e:
        _create(**kw)
    assert e.value.code == code
    assert abi.stencil_last_error()


def test_calls_before_bind_are_state_errors():
    h = _create()
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_step(h, 1)
    assert e.value.code == abi.ST_ERR_STATE
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_step(h, -1)
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_bind(h, 3, 256)
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_bind(h, 0, 257)  # misaligned
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_set_current(h, 2)
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_set_source(h, (1, 1, 1), [1.0])   # one time level: no source
    assert e.value.code == abi.ST_ERR_UNSUPPORTED
    assert abi.stencil_current(h) == 0
    abi.stencil_destroy(h)


def test_adjoint_workspace_size():
    h = _create(dims=(16, 16, 16))
    _, _, n = abi.stencil_layout(h, 3)
    per = (n * 4 + 255) // 256 * 256
    # checkpoints + one segment's recomputation buffer + the kept last segment
    assert abi.stencil_adjoint_workspace(h, 200, 20) == per * (10 + 19 + 19)
    assert abi.stencil_adjoint_workspace(h, 7, 3) == per * (3 + 2 + 2)
    # one segment: the checkpoint and the kept levels, no recomputation buffer
    assert abi.stencil_adjoint_workspace(h, 200, 200) == per * (1 + 199)
    with pytest.raises(abi.StencilError):
        abi.stencil_adjoint_workspace(h, 10, 0)
    abi.stencil_destroy(h)


def test_batch_create_validation_and_layout():
    dims = np.array([[64, 80], [3, 100], [37, 41]])
    w = np.full((3, 9), 1.0 / 9)
    from paper_2512_19851_gb300 import inputs
    h = abi.stencil_batch_create(dims, inputs.OFFSETS_BOX9, w, abi.ST_PERIODIC, 0.0, abi.ST_F32)
    for i, (ny, nx) in enumerate(dims):
        pd, org, n = abi.stencil_batch_layout(h, i)
        assert pd[0] == ny + 2 and org == (1, 4) and pd[1] * 4 % 16 == 0 and n == pd[0] * pd[1]
    with pytest.raises(abi.StencilError):
        abi.stencil_batch_layout(h, 3)
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_batch_step(h, 1)
    assert e.value.code == abi.ST_ERR_STATE
    abi.stencil_batch_destroy(h)
    with pytest.raises(abi.StencilError):
        abi.stencil_batch_create([[1, 10]], inputs.OFFSETS_BOX9, np.ones((1, 9)), abi.ST_PERIODIC, 0.0, abi.ST_F32)


def test_caller_ghosts_choose_kernels_that_read_ghost_cells():
    """A 2D FP32 grid leaves the persistent tile kernel (which substitutes the
    boundary value) for the one-thread-per-point kernel when its ghosts are
    the caller's; 3D keeps the star kernel."""
    h = abi.stencil_create(2, (64, 64), 0, [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)], [0.2] * 5, dtype=abi.ST_F32)
    assert abi.stencil_info(h)[2] == "tile2d_persistent"
    abi.stencil_destroy(h)
    h = abi.stencil_create(2, (64, 64), 0, [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)], [0.2] * 5, dtype=abi.ST_F32,
                           flags=abi.ST_FLAG_CALLER_GHOSTS)
    assert abi.stencil_info(h)[2] == "generic_point"
    abi.stencil_destroy(h)
    h = _create(offsets=[(0, 0, 0), (0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)],
                alpha=[0.4] + [0.1] * 6, flags=abi.ST_FLAG_CALLER_GHOSTS)
    assert abi.stencil_info(h)[2].startswith("star3d")
    abi.stencil_destroy(h)


def test_snapshot_needs_bound_buffers():
    h = _create()
    assert abi.stencil_snapshot_bytes(h) == abi.stencil_layout(h, 3)[2] * 4
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_snapshot(h, 16)
    assert e.value.code == abi.ST_ERR_STATE
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_restore(h, 16, -1)
    assert e.value.code == abi.ST_ERR_ARG
    abi.stencil_destroy(h)
    h = _create(time_levels=2)
    assert abi.stencil_snapshot_bytes(h) == 2 * abi.stencil_layout(h, 3)[2] * 4
    abi.stencil_destroy(h)


def test_neumann_arguments():
    star = [(0, 0, 0), (0, 0, 1), (0, 0, -1), (0, 1, 0), (0, -1, 0), (1, 0, 0), (-1, 0, 0)]
    h = _create(bc=abi.ST_NEUMANN, offsets=star, alpha=[0.4] + [0.1] * 6)
    assert abi.stencil_info(h)[2].startswith("star3d")
    with pytest.raises(abi.StencilError) as e:  # the checkpointed run exists; unbound buffers are the error
        abi.stencil_step_ckpt(h, 2, 1, 16)
    assert e.value.code == abi.ST_ERR_STATE
    abi.stencil_destroy(h)
    with pytest.raises(abi.StencilError) as e:       # mirror image outside the interior
        _create(bc=abi.ST_NEUMANN, dims=(8, 1, 10), offsets=[(0, 0, 0), (0, 2, 0)], alpha=[0.5, 0.5])
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        _create(bc=abi.ST_NEUMANN, time_levels=2)
    assert e.value.code == abi.ST_ERR_UNSUPPORTED
    h = abi.stencil_create(2, (64, 64), 0, [(0, 0), (1, 0), (-1, 0), (0, 1), (0, -1)], [0.2] * 5,
                           bc=abi.ST_NEUMANN, dtype=abi.ST_F32)
    assert abi.stencil_info(h)[2] == "generic_point"
    abi.stencil_destroy(h)


def test_conservative_create():
    h = abi.stencil_create_conservative(3, (8, 9, 10), abi.ST_PERIODIC, 0.0, abi.ST_F64)
    r, n, name = abi.stencil_info(h)
    assert (r, n, name) == (1, 7, "cons_face_avg_bulk")  # 3D: the staged pipeline
    abi.stencil_destroy(h)
    h = abi.stencil_create_conservative(2, (8, 9), abi.ST_DIRICHLET, 0.5, abi.ST_F32)
    assert abi.stencil_info(h)[1:] == (5, "cons_face_avg_point")  # 2D: a thread per column
    abi.stencil_destroy(h)
    for kw in (dict(ndim=4, dims=(2, 2, 2, 2)), dict(bc=abi.ST_NEUMANN), dict(flags=1)):
        args = dict(ndim=3, dims=(8, 9, 10), bc=abi.ST_DIRICHLET, bc_value=0.0, dtype=abi.ST_F64, flags=0)
        args.update(kw)
        with pytest.raises(abi.StencilError) as e:
            abi.stencil_create_conservative(**args)
        assert e.value.code == abi.ST_ERR_ARG


def test_cavity_arguments():
    for kw in (dict(ny=2), dict(nx=2), dict(dx=0.0), dict(dt=-1.0), dict(rho=0.0), dict(nu=-0.1), dict(nit=-1),
               dict(dtype=5)):
        args = dict(ny=41, nx=41, dx=0.05, dy=0.05, dt=0.001, rho=1.0, nu=0.1, nit=50, lid=1.0, dtype=abi.ST_F64)
        args.update(kw)
        with pytest.raises(abi.StencilError) as e:
            abi.stencil_cavity_create(**args)
        assert e.value.code == abi.ST_ERR_ARG
    h = abi.stencil_cavity_create(41, 41, 0.05, 0.05, 0.001)
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_cavity_step(h, 1)
    assert e.value.code == abi.ST_ERR_STATE
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_cavity_bind(h, 0, 16, 32)
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:          # u and v overlap (checked before any allocation)
        abi.stencil_cavity_bind(h, 1 << 20, (1 << 20) + 8, 1 << 24)
    assert e.value.code == abi.ST_ERR_ALIAS
    abi.stencil_cavity_destroy(h)


def test_tile_passes_flag_selects_the_fp64_tile_option():
    """ST_FLAG_TILE_PASSES starts FP64 2D grids within the 3x3 neighbourhood
    on the tile passes; other grids ignore it."""
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]
    def name(dims, dtype, flags, bc=abi.ST_DIRICHLET, offsets=offs):
        off = np.asarray(offsets, dtype=np.int32).reshape(-1)
        h = abi.stencil_create(len(dims), dims, 0, off, [0.2] * (len(off) // len(dims)), None, bc, 0.0, dtype, 1,
                               flags)
        n = abi.stencil_info(h)[2]
        abi.stencil_destroy(h)
        return n
    assert name((64, 80), abi.ST_F64, 0) == "generic_point"
    assert name((64, 80), abi.ST_F64, abi.ST_FLAG_TILE_PASSES) == "tile2d_passes"
    assert name((64, 80), abi.ST_F64, abi.ST_FLAG_TILE_PASSES, abi.ST_PERIODIC) == "tile2d_passes"
    assert name((64, 80), abi.ST_F32, abi.ST_FLAG_TILE_PASSES) == "tile2d_persistent"
    # outside the 3x3 neighbourhood, caller ghosts, zero flux, generic: the per-point kernel
    wide = [(0, 0), (-2, 0), (2, 0), (0, -2), (0, 2)]
    assert name((64, 80), abi.ST_F64, abi.ST_FLAG_TILE_PASSES, offsets=wide) == "generic_point"
    assert name((64, 80), abi.ST_F64, abi.ST_FLAG_TILE_PASSES | abi.ST_FLAG_CALLER_GHOSTS) == "generic_point"
    assert name((64, 80), abi.ST_F64, abi.ST_FLAG_TILE_PASSES, abi.ST_NEUMANN) == "generic_point"
    assert name((64, 80), abi.ST_F64, abi.ST_FLAG_TILE_PASSES | abi.ST_FLAG_GENERIC) == "generic_point"



def test_tb2d_configuration_override(monkeypatch):
    """ST_TB2D_CFG = "TX,TY,k" starts an FP64 2D grid within the 3x3
    neighbourhood on the k-step static-tile kernel with that configuration;
    malformed or oversized values, other grids and ST_FLAG_TILE_PASSES leave
    the usual choice."""
    offs = [(0, 0), (-1, 0), (1, 0), (0, -1), (0, 1)]

    def made(dims, dtype, flags=0, bc=abi.ST_DIRICHLET, offsets=offs):
        off = np.asarray(offsets, dtype=np.int32).reshape(-1)
        h = abi.stencil_create(len(dims), dims, 0, off, [0.2] * (len(off) // len(dims)), None, bc, 0.0, dtype, 1,
                               flags)
        n = abi.stencil_info(h)[2]
        cfg = list(abi.stencil_tune_config(h))
        abi.stencil_destroy(h)
        return n, cfg

    monkeypatch.setenv("ST_TB2D_CFG", "16,14,3")
    assert made((64, 80), abi.ST_F64) == ("tb2d_passes", [16, 14, 512, 3])
    assert made((64, 80), abi.ST_F64, bc=abi.ST_PERIODIC)[0] == "tb2d_passes"
    assert made((64, 80), abi.ST_F64, abi.ST_FLAG_TILE_PASSES)[0] == "tile2d_passes"
    assert made((64, 80), abi.ST_F32)[0] == "tile2d_persistent"
    assert made((64, 80), abi.ST_F64, bc=abi.ST_NEUMANN)[0] == "generic_point"
    assert made((64, 80), abi.ST_F64, offsets=[(0, 0), (-2, 0), (2, 0), (0, -2), (0, 2)])[0] == "generic_point"
    assert made((8, 9, 10), abi.ST_F64, offsets=[(0, 0, 0), (0, 0, 1), (0, 0, -1)])[0] != "tb2d_passes"
    for bad in ("16,14", "0,14,3", "16,14,0", "x,y,z", "1000,1000,8"):
        monkeypatch.setenv("ST_TB2D_CFG", bad)
        assert made((64, 80), abi.ST_F64)[0] == "generic_point", bad
    monkeypatch.delenv("ST_TB2D_CFG")
    assert made((64, 80), abi.ST_F64) == ("generic_point", [0, 0, 0, 0])


def test_run_host_many_arguments():
    """Argument and state checks of the pipelined host form run before any
    device work: a NULL handle, a negative step count or a NULL host pointer
    is ST_ERR_ARG, an unbound grid ST_ERR_STATE, and the binding rejects
    lists of different lengths."""
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_run_host_many(None, 1, [], [])
    assert e.value.code == abi.ST_ERR_ARG
    h = _create()
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_run_host_many(h, -1, [], [])
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_run_host_many(h, 1, [0], [0])
    assert e.value.code == abi.ST_ERR_ARG
    with pytest.raises(abi.StencilError) as e:
        abi.stencil_run_host_many(h, 1, [], [])
    assert e.value.code == abi.ST_ERR_STATE
    with pytest.raises(ValueError):
        abi.stencil_run_host_many(h, 1, [64], [])
    abi.stencil_destroy(h)
