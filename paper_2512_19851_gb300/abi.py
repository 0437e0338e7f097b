"""ctypes binding of libstencil.so (include/stencil.h), same names as the C ABI.

Argument marshalling only: every computation happens in the CUDA library.
Device buffers are passed as integer addresses (``tensor.data_ptr()``),
streams as ``torch.cuda.Stream.cuda_stream`` (0 = legacy default stream).
A negative status raises :class:`StencilError` with the library's message.
If the library cannot be loaded (not built, no CUDA toolchain) every call
fails loudly; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ST_OK = 0
ST_ERR_ARG = -1
ST_ERR_ALIAS = -2
ST_ERR_UNSUPPORTED = -3
ST_ERR_CUDA = -4
ST_ERR_DEVICE_TIMEOUT = -5
ST_ERR_BOUNDS = -6
ST_ERR_OOM = -7
ST_ERR_STATE = -8
ST_F32, ST_F64 = 0, 1
ST_DIRICHLET, ST_PERIODIC, ST_NEUMANN = 0, 1, 2
ST_FLAG_GENERIC = 1
ST_FLAG_TWO_STEP = 2
ST_FLAG_CALLER_GHOSTS = 4
ST_FLAG_TILE_PASSES = 8
ST_SLOT_A, ST_SLOT_B, ST_SLOT_COEFF = 0, 1, 2
ST_MAX_POINTS = 64
ST_MAX_RADIUS = 8

STATUS_NAMES = {0: "ST_OK", -1: "ST_ERR_ARG", -2: "ST_ERR_ALIAS", -3: "ST_ERR_UNSUPPORTED", -4: "ST_ERR_CUDA",
                -5: "ST_ERR_DEVICE_TIMEOUT", -6: "ST_ERR_BOUNDS", -7: "ST_ERR_OOM", -8: "ST_ERR_STATE"}

# every entry point of include/stencil.h with its ctypes signature
_I, _I64, _D, _VP, _CP, _U32 = ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_void_p, ctypes.c_char_p, ctypes.c_uint32
_PI, _PI64, _PD, _PVP = (ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int64),
                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_void_p))
_PSZ = ctypes.POINTER(ctypes.c_size_t)
_PI32 = ctypes.POINTER(ctypes.c_int32)
SIGNATURES = {
    "stencil_version": (_CP, []),
    "stencil_last_error": (_CP, []),
    "stencil_create": (_I, [_PVP, _I, _PI64, _I, _I, _PI32, _PD, _PD, _I, _D, _I, _I, _U32]),
    "stencil_create_conservative": (_I, [_PVP, _I, _PI64, _I, _D, _I, _U32]),
    "stencil_destroy": (_I, [_VP]),
    "stencil_layout": (_I, [_VP, _PI64, _PI64, _PI64]),
    "stencil_info": (_I, [_VP, _PI, _PI, ctypes.POINTER(_CP)]),
    "stencil_bind": (_I, [_VP, _I, _VP]),
    "stencil_mark_dirty": (_I, [_VP, _I]),
    "stencil_current": (_I, [_VP, _PI]),
    "stencil_set_current": (_I, [_VP, _I]),
    "stencil_set_source": (_I, [_VP, _PI64, _PD, _I64]),
    "stencil_set_step_index": (_I, [_VP, _I64]),
    "stencil_get_step_index": (_I, [_VP, _PI64]),
    "stencil_snapshot_bytes": (_I, [_VP, _PSZ]),
    "stencil_snapshot": (_I, [_VP, _VP, _PI64, _VP]),
    "stencil_restore": (_I, [_VP, _VP, _I64, _VP]),
    "stencil_step": (_I, [_VP, _I, _VP]),
    "stencil_step_reduce": (_I, [_VP, _I, _VP, _VP]),
    "stencil_tune": (_I, [_VP, _I, _VP]),
    "stencil_tune_config": (_I, [_VP, _PI]),
    "stencil_run_host": (_I, [_VP, _I, _VP, _VP, _VP]),
    "stencil_run_host_many": (_I, [_VP, _I, _I, _VP, _VP, _VP]),
    "stencil_sync": (_I, [_VP]),
    "stencil_reduce": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "stencil_residual": (_I, [_VP, _VP, _VP, _VP, _VP, _VP]),
    "stencil_reduce_noalloc": (_I, [_VP, _VP, _VP, _VP, _VP]),
    "stencil_adjoint_workspace": (_I, [_VP, _I, _I, _PSZ]),
    "stencil_step_ckpt": (_I, [_VP, _I, _I, _VP, _VP]),
    "stencil_adjoint": (_I, [_VP, _I, _I, _VP, _VP, _VP, _VP, _VP]),
    "stencil_cavity_create": (_I, [_PVP, _I64, _I64, _D, _D, _D, _D, _D, _I, _D, _I]),
    "stencil_cavity_destroy": (_I, [_VP]),
    "stencil_cavity_bind": (_I, [_VP, _VP, _VP, _VP]),
    "stencil_cavity_step": (_I, [_VP, _I, _VP]),
    "stencil_batch_create": (_I, [_PVP, _I, _PI64, _I, _PI32, _PD, _I, _D, _I, _U32]),
    "stencil_batch_destroy": (_I, [_VP]),
    "stencil_batch_layout": (_I, [_VP, _I, _PI64, _PI64, _PI64]),
    "stencil_batch_bind": (_I, [_VP, _PVP, _PVP]),
    "stencil_batch_tune": (_I, [_VP, _I, _VP]),
    "stencil_batch_config": (_I, [_VP, _PI]),
    "stencil_batch_step": (_I, [_VP, _I, _VP]),
    "stencil_batch_current": (_I, [_VP, _PI]),
    "stencil_batch_sync": (_I, [_VP]),
    "stencil_batch_selftest_barrier": (_I, [_VP, ctypes.c_uint64, _VP]),
}

_lib = None


class StencilError(RuntimeError):
    def __init__(self, code: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def lib() -> ctypes.CDLL:
    """Load (building first if absent) libstencil.so."""
    global _lib
    if _lib is None:
        path = _build.LIB if os.path.exists(_build.LIB) else _build.build()
        cdll = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(cdll, name)
            fn.restype = res
            fn.argtypes = args
        _lib = cdll
    return _lib


def _check(code: int, where: str) -> None:
    if code != ST_OK:
        raise StencilError(code, where, stencil_last_error())


def _arr(values, ctype):
    a = (ctype * len(values))(*values)
    return a


def _stream(stream) -> int:
    if stream is None:
        return 0
    return int(getattr(stream, "cuda_stream", stream))


def stencil_version() -> str:
    return lib().stencil_version().decode()


def stencil_last_error() -> str:
    return lib().stencil_last_error().decode()


def stencil_create(ndim, dims, radius, offsets, alpha, beta=None, bc=ST_DIRICHLET, bc_value=0.0, dtype=ST_F64,
                   time_levels=1, flags=0):
    """Returns an opaque handle (int)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1))
    npts = len(alpha)
    h = ctypes.c_void_p()
    a = _arr([float(v) for v in alpha], ctypes.c_double)
    b = None if beta is None else _arr([float(v) for v in beta], ctypes.c_double)
    d = _arr([int(v) for v in dims], ctypes.c_int64)
    o = _arr([int(v) for v in off], ctypes.c_int32)
    _check(lib().stencil_create(ctypes.byref(h), int(ndim), d, int(radius), int(npts), o, a, b, int(bc),
                                float(bc_value), int(dtype), int(time_levels), int(flags)), "stencil_create")
    return h.value


def stencil_create_conservative(ndim, dims, bc=ST_DIRICHLET, bc_value=0.0, dtype=ST_F64, flags=0):
    """Handle of the conservative face-averaged per-cell diffusion (opaque int)."""
    h = ctypes.c_void_p()
    d = _arr([int(v) for v in dims], ctypes.c_int64)
    _check(lib().stencil_create_conservative(ctypes.byref(h), int(ndim), d, int(bc), float(bc_value), int(dtype),
                                             int(flags)), "stencil_create_conservative")
    return h.value


def stencil_destroy(h) -> None:
    _check(lib().stencil_destroy(h), "stencil_destroy")


def stencil_layout(h, ndim):
    pd = (ctypes.c_int64 * ndim)()
    org = (ctypes.c_int64 * ndim)()
    n = ctypes.c_int64()
    _check(lib().stencil_layout(h, pd, org, ctypes.byref(n)), "stencil_layout")
    return tuple(pd), tuple(org), n.value


def stencil_info(h):
    r, n, name = ctypes.c_int(), ctypes.c_int(), ctypes.c_char_p()
    _check(lib().stencil_info(h, ctypes.byref(r), ctypes.byref(n), ctypes.byref(name)), "stencil_info")
    return r.value, n.value, name.value.decode()


def stencil_bind(h, slot, ptr) -> None:
    _check(lib().stencil_bind(h, int(slot), ctypes.c_void_p(int(ptr))), "stencil_bind")


def stencil_mark_dirty(h, slot) -> None:
    _check(lib().stencil_mark_dirty(h, int(slot)), "stencil_mark_dirty")


def stencil_current(h) -> int:
    s = ctypes.c_int()
    _check(lib().stencil_current(h, ctypes.byref(s)), "stencil_current")
    return s.value


def stencil_set_current(h, slot) -> None:
    _check(lib().stencil_set_current(h, int(slot)), "stencil_set_current")


def stencil_set_source(h, index, amplitudes) -> None:
    amps = np.ascontiguousarray(amplitudes, dtype=np.float64)
    idx = _arr([int(v) for v in index], ctypes.c_int64) if index is not None else None
    _check(lib().stencil_set_source(h, idx, amps.ctypes.data_as(_PD) if amps.size else None, int(amps.size)),
           "stencil_set_source")


def stencil_set_step_index(h, t) -> None:
    _check(lib().stencil_set_step_index(h, int(t)), "stencil_set_step_index")


def stencil_get_step_index(h) -> int:
    t = ctypes.c_int64()
    _check(lib().stencil_get_step_index(h, ctypes.byref(t)), "stencil_get_step_index")
    return t.value


def stencil_snapshot_bytes(h) -> int:
    n = ctypes.c_size_t()
    _check(lib().stencil_snapshot_bytes(h, ctypes.byref(n)), "stencil_snapshot_bytes")
    return n.value


def stencil_snapshot(h, dst_ptr, stream=None) -> int:
    """Enqueue the snapshot copies into dst_ptr; returns the step counter."""
    t = ctypes.c_int64()
    _check(lib().stencil_snapshot(h, ctypes.c_void_p(int(dst_ptr)), ctypes.byref(t),
                                  ctypes.c_void_p(_stream(stream))), "stencil_snapshot")
    return t.value


def stencil_restore(h, src_ptr, step, stream=None) -> None:
    _check(lib().stencil_restore(h, ctypes.c_void_p(int(src_ptr)), int(step), ctypes.c_void_p(_stream(stream))),
           "stencil_restore")


def stencil_step(h, nsteps, stream=None) -> None:
    _check(lib().stencil_step(h, int(nsteps), ctypes.c_void_p(_stream(stream))), "stencil_step")


def stencil_tune(h, nsteps, stream=None) -> None:
    _check(lib().stencil_tune(h, int(nsteps), ctypes.c_void_p(_stream(stream))), "stencil_tune")


def stencil_tune_config(h):
    cfg = (ctypes.c_int * 4)()
    _check(lib().stencil_tune_config(h, cfg), "stencil_tune_config")
    return tuple(cfg)


def stencil_step_reduce(h, nsteps, out_ptr, stream=None) -> None:
    """nsteps sweeps, then (sum, sum of squares, max |u|) of the newest level
    into the 3 doubles at out_ptr (device)."""
    _check(lib().stencil_step_reduce(h, int(nsteps), ctypes.c_void_p(int(out_ptr)), ctypes.c_void_p(_stream(stream))),
           "stencil_step_reduce")


def stencil_run_host(h, nsteps, host_u0_ptr, host_uT_ptr, stream=None) -> None:
    _check(lib().stencil_run_host(h, int(nsteps), ctypes.c_void_p(int(host_u0_ptr)),
                                  ctypes.c_void_p(int(host_uT_ptr)), ctypes.c_void_p(_stream(stream))),
           "stencil_run_host")


def stencil_run_host_many(h, nsteps, host_in_ptrs, host_out_ptrs, stream=None) -> None:
    """Jobs i = 0..n-1: host_in_ptrs[i] -> nsteps -> host_out_ptrs[i], host
    copies overlapping the sweeps (pinned buffers)."""
    n = len(host_in_ptrs)
    if len(host_out_ptrs) != n:
        raise ValueError("stencil_run_host_many: as many output as input pointers")
    ins = (ctypes.c_void_p * max(n, 1))(*[int(p) for p in host_in_ptrs])
    outs = (ctypes.c_void_p * max(n, 1))(*[int(p) for p in host_out_ptrs])
    _check(lib().stencil_run_host_many(h, int(nsteps), n, ctypes.cast(ins, ctypes.c_void_p),
                                       ctypes.cast(outs, ctypes.c_void_p), ctypes.c_void_p(_stream(stream))),
           "stencil_run_host_many")


def stencil_sync(h) -> None:
    _check(lib().stencil_sync(h), "stencil_sync")


def stencil_reduce(h, a_ptr, b_ptr, out_ptr, stream=None) -> None:
    _check(lib().stencil_reduce(h, ctypes.c_void_p(int(a_ptr)), ctypes.c_void_p(int(b_ptr) if b_ptr else None),
                                ctypes.c_void_p(int(out_ptr)), ctypes.c_void_p(_stream(stream))), "stencil_reduce")


def stencil_reduce_noalloc(h, a_ptr, b_ptr, out_ptr, stream=None) -> None:
    """stencil_reduce without device allocation (partials in a static device array)."""
    _check(lib().stencil_reduce_noalloc(h, ctypes.c_void_p(int(a_ptr)),
                                        ctypes.c_void_p(int(b_ptr) if b_ptr else None),
                                        ctypes.c_void_p(int(out_ptr)), ctypes.c_void_p(_stream(stream))),
           "stencil_reduce_noalloc")


def stencil_residual(h, u_ptr, target_ptr, lam_ptr, loss_ptr, stream=None) -> None:
    _check(lib().stencil_residual(h, ctypes.c_void_p(int(u_ptr)), ctypes.c_void_p(int(target_ptr)),
                                  ctypes.c_void_p(int(lam_ptr)), ctypes.c_void_p(int(loss_ptr)),
                                  ctypes.c_void_p(_stream(stream))), "stencil_residual")


def stencil_adjoint_workspace(h, nsteps, ckpt_every) -> int:
    n = ctypes.c_size_t()
    _check(lib().stencil_adjoint_workspace(h, int(nsteps), int(ckpt_every), ctypes.byref(n)),
           "stencil_adjoint_workspace")
    return n.value


def stencil_step_ckpt(h, nsteps, ckpt_every, ws_ptr, stream=None) -> None:
    _check(lib().stencil_step_ckpt(h, int(nsteps), int(ckpt_every), ctypes.c_void_p(int(ws_ptr)),
                                   ctypes.c_void_p(_stream(stream))), "stencil_step_ckpt")


def stencil_adjoint(h, nsteps, ckpt_every, ws_ptr, lam_ptr, lam_tmp_ptr, grad_ptr, stream=None) -> None:
    _check(lib().stencil_adjoint(h, int(nsteps), int(ckpt_every), ctypes.c_void_p(int(ws_ptr)),
                                 ctypes.c_void_p(int(lam_ptr)), ctypes.c_void_p(int(lam_tmp_ptr)),
                                 ctypes.c_void_p(int(grad_ptr)) if grad_ptr else None,
                                 ctypes.c_void_p(_stream(stream))), "stencil_adjoint")


def stencil_batch_create(dims, offsets, weights, bc=ST_PERIODIC, bc_value=0.0, dtype=ST_F32, flags=0):
    dims = np.ascontiguousarray(np.asarray(dims, dtype=np.int64).reshape(-1, 2))
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 2))
    w = np.ascontiguousarray(np.asarray(weights, dtype=np.float64).reshape(dims.shape[0], off.shape[0]))
    h = ctypes.c_void_p()
    _check(lib().stencil_batch_create(ctypes.byref(h), int(dims.shape[0]), dims.ctypes.data_as(_PI64),
                                      int(off.shape[0]), off.ctypes.data_as(_PI32), w.ctypes.data_as(_PD),
                                      int(bc), float(bc_value), int(dtype), int(flags)), "stencil_batch_create")
    return h.value


def stencil_batch_destroy(h) -> None:
    _check(lib().stencil_batch_destroy(h), "stencil_batch_destroy")


def stencil_batch_layout(h, g):
    pd = (ctypes.c_int64 * 2)()
    org = (ctypes.c_int64 * 2)()
    n = ctypes.c_int64()
    _check(lib().stencil_batch_layout(h, int(g), pd, org, ctypes.byref(n)), "stencil_batch_layout")
    return tuple(pd), tuple(org), n.value


def stencil_batch_bind(h, ptrs_a, ptrs_b) -> None:
    pa = (ctypes.c_void_p * len(ptrs_a))(*[int(p) for p in ptrs_a])
    pb = (ctypes.c_void_p * len(ptrs_b))(*[int(p) for p in ptrs_b])
    _check(lib().stencil_batch_bind(h, pa, pb), "stencil_batch_bind")


def stencil_batch_tune(h, nsteps, stream=None) -> None:
    _check(lib().stencil_batch_tune(h, int(nsteps), ctypes.c_void_p(_stream(stream))), "stencil_batch_tune")


def stencil_batch_config(h):
    cfg = (ctypes.c_int * 4)()
    _check(lib().stencil_batch_config(h, cfg), "stencil_batch_config")
    return tuple(cfg)


def stencil_batch_step(h, nsteps, stream=None) -> None:
    _check(lib().stencil_batch_step(h, int(nsteps), ctypes.c_void_p(_stream(stream))), "stencil_batch_step")


def stencil_batch_current(h) -> int:
    s = ctypes.c_int()
    _check(lib().stencil_batch_current(h, ctypes.byref(s)), "stencil_batch_current")
    return s.value


def stencil_batch_sync(h) -> None:
    _check(lib().stencil_batch_sync(h), "stencil_batch_sync")


def stencil_batch_selftest_barrier(h, timeout_ns, stream=None) -> None:
    _check(lib().stencil_batch_selftest_barrier(h, int(timeout_ns), ctypes.c_void_p(_stream(stream))),
           "stencil_batch_selftest_barrier")


def stencil_cavity_create(ny, nx, dx, dy, dt, rho=1.0, nu=0.1, nit=50, lid=1.0, dtype=ST_F64):
    h = ctypes.c_void_p()
    _check(lib().stencil_cavity_create(ctypes.byref(h), int(ny), int(nx), float(dx), float(dy), float(dt), float(rho),
                                       float(nu), int(nit), float(lid), int(dtype)), "stencil_cavity_create")
    return h.value


def stencil_cavity_destroy(h) -> None:
    _check(lib().stencil_cavity_destroy(h), "stencil_cavity_destroy")


def stencil_cavity_bind(h, u_ptr, v_ptr, p_ptr) -> None:
    _check(lib().stencil_cavity_bind(h, ctypes.c_void_p(int(u_ptr)), ctypes.c_void_p(int(v_ptr)),
                                     ctypes.c_void_p(int(p_ptr))), "stencil_cavity_bind")


def stencil_cavity_step(h, nsteps, stream=None) -> None:
    _check(lib().stencil_cavity_step(h, int(nsteps), ctypes.c_void_p(_stream(stream))), "stencil_cavity_step")
