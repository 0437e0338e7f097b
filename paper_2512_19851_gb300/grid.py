"""Torch-facing helpers over the C ABI: padded buffers allocated by PyTorch,
bound to a handle, and a torch.autograd.Function whose backward is the
library's checkpointed adjoint.  PyTorch provides device memory, streams and
copies of input data into the interior views; the sweeps, the adjoint, the
residual and the reductions run in libstencil's kernels.
"""
from __future__ import annotations

import numpy as np
import torch

from . import abi
from .abi import ST_DIRICHLET, ST_F32, ST_F64, ST_FLAG_GENERIC, ST_PERIODIC, ST_SLOT_A, ST_SLOT_B, ST_SLOT_COEFF

_ST_DTYPE = {torch.float32: ST_F32, torch.float64: ST_F64}


def _before_torch_copies(stream, device):
    """torch writes a call's input copies on its current stream: when the
    library works on another `stream`, the current stream first waits for
    that stream's earlier work on the same buffers."""
    cur = torch.cuda.current_stream(device)
    if stream is not None and stream != cur:
        cur.wait_stream(stream)


def _after_torch_copies(stream, device):
    """The stream library work goes to: `stream`, or torch's current stream.
    A different stream first waits for the copies torch made on its current
    stream."""
    cur = torch.cuda.current_stream(device)
    if stream is None:
        return cur
    if stream != cur:
        stream.wait_stream(cur)
    return stream


def _as_tensor(x, dtype, device):
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=dtype)
    return torch.as_tensor(np.ascontiguousarray(x), dtype=dtype, device=device)


class Grid:
    """A grid handle with its two time-level buffers (and coefficient field)."""

    def __init__(self, shape, offsets, alpha, beta=None, periodic=False, bc_value=0.0, dtype=torch.float64,
                 time_levels=1, radius=0, generic=False, device=None, two_step=False, caller_ghosts=False,
                 neumann=False, conservative=False, tile_passes=False):
        """conservative=True: the face-averaged per-cell diffusion of
        stencil_create_conservative (offsets, alpha and beta are ignored)."""
        self.shape = tuple(int(s) for s in shape)
        self.ndim = len(self.shape)
        self.dtype = dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.periodic = bool(periodic)
        bc = ST_PERIODIC if periodic else (abi.ST_NEUMANN if neumann else ST_DIRICHLET)
        if conservative:
            self.h = abi.stencil_create_conservative(self.ndim, self.shape, bc, bc_value, _ST_DTYPE[dtype])
            beta = True
        else:
            self.h = abi.stencil_create(self.ndim, self.shape, radius, offsets, alpha, beta,
                                        bc, bc_value, _ST_DTYPE[dtype],
                                        time_levels, (ST_FLAG_GENERIC if generic else 0) |
                                        (abi.ST_FLAG_TWO_STEP if two_step else 0) |
                                        (abi.ST_FLAG_CALLER_GHOSTS if caller_ghosts else 0) |
                                        (abi.ST_FLAG_TILE_PASSES if tile_passes else 0))
        self.padded, self.origin, self.elems = abi.stencil_layout(self.h, self.ndim)
        self.radius, self.npts, self.kernel = abi.stencil_info(self.h)
        self.bufs = [torch.zeros(self.padded, dtype=dtype, device=self.device) for _ in range(2)]
        abi.stencil_bind(self.h, ST_SLOT_A, self.bufs[0].data_ptr())
        abi.stencil_bind(self.h, ST_SLOT_B, self.bufs[1].data_ptr())
        self.coeff = None
        # bumped by every set_coeff: a recorded adjoint is valid only for the
        # coefficient field its forward run used
        self.coeff_generation = 0
        if beta is not None:
            self.coeff = torch.zeros(self.padded, dtype=dtype, device=self.device)
            abi.stencil_bind(self.h, ST_SLOT_COEFF, self.coeff.data_ptr())

    # -- views -------------------------------------------------------------
    def interior(self, t: torch.Tensor) -> torch.Tensor:
        return t[tuple(slice(o, o + s) for o, s in zip(self.origin, self.shape))]

    def ring(self, t: torch.Tensor) -> torch.Tensor:
        """View of a buffer's interior plus its ghost ring (radius r on every
        side), the region ST_FLAG_CALLER_GHOSTS leaves to the caller."""
        r = self.radius
        return t[tuple(slice(o - r, o + s + r) for o, s in zip(self.origin, self.shape))]

    def new_field(self, dtype=None) -> torch.Tensor:
        return torch.zeros(self.padded, dtype=dtype or self.dtype, device=self.device)

    def current_slot(self) -> int:
        return abi.stencil_current(self.h)

    def current(self) -> torch.Tensor:
        """Interior view of the newest time level."""
        return self.interior(self.bufs[self.current_slot()])

    def previous(self) -> torch.Tensor:
        return self.interior(self.bufs[1 - self.current_slot()])

    # -- data --------------------------------------------------------------
    def set_field(self, u, slot=None) -> None:
        s = self.current_slot() if slot is None else slot
        self.interior(self.bufs[s]).copy_(_as_tensor(u, self.dtype, self.device))
        abi.stencil_mark_dirty(self.h, s)

    def set_levels(self, u_now, u_prev) -> None:
        """Leapfrog: newest level u_now in slot A, u_prev in slot B."""
        abi.stencil_set_current(self.h, ST_SLOT_A)
        self.set_field(u_now, ST_SLOT_A)
        self.set_field(u_prev, ST_SLOT_B)

    def set_coeff(self, kappa) -> None:
        self.interior(self.coeff).copy_(_as_tensor(kappa, self.dtype, self.device))
        abi.stencil_mark_dirty(self.h, ST_SLOT_COEFF)
        self.coeff_generation += 1

    def set_source(self, index, amplitudes) -> None:
        abi.stencil_set_source(self.h, index, amplitudes)

    def set_step_index(self, t) -> None:
        abi.stencil_set_step_index(self.h, t)

    # -- snapshot / restore -------------------------------------------------
    def snapshot(self, stream=None):
        """Park the state in a new device buffer (device-to-device copies):
        returns (buffer, step counter).  The buffer belongs to the caller and
        may outlive this grid."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        buf = torch.empty(abi.stencil_snapshot_bytes(self.h), dtype=torch.uint8, device=self.device)
        step = abi.stencil_snapshot(self.h, buf.data_ptr(), s)
        return buf, step

    def restore(self, snap, stream=None) -> None:
        buf, step = snap
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        abi.stencil_restore(self.h, buf.data_ptr(), step, s)

    # -- work --------------------------------------------------------------
    def step(self, nsteps: int, stream=None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        abi.stencil_step(self.h, nsteps, s)

    def sync(self) -> None:
        abi.stencil_sync(self.h)

    def tune(self, nsteps: int, stream=None) -> tuple:
        """Autotune for nsteps-step calls (2D tile kernel); returns the configuration."""
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        abi.stencil_tune(self.h, nsteps, s)
        self.kernel = abi.stencil_info(self.h)[2]  # the tuner may change the kernel family
        return abi.stencil_tune_config(self.h)

    def reduce(self, a: torch.Tensor, b: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """(sum, sum of squares, max abs) of a - b over the interior, float64 on device."""
        out = torch.empty(3, dtype=torch.float64, device=self.device)
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        abi.stencil_reduce(self.h, a.data_ptr(), b.data_ptr() if b is not None else 0, out.data_ptr(), s)
        return out

    def close(self) -> None:
        if getattr(self, "h", None):
            abi.stencil_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent 2D grids, one padded buffer pair per grid."""

    def __init__(self, shapes, offsets, weights, periodic=True, bc_value=0.0, dtype=torch.float32, generic=False,
                 device=None):
        self.shapes = [tuple(int(v) for v in s) for s in np.asarray(shapes).reshape(-1, 2)]
        self.dtype = dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.h = abi.stencil_batch_create(self.shapes, offsets, weights, ST_PERIODIC if periodic else ST_DIRICHLET,
                                          bc_value, _ST_DTYPE[dtype], ST_FLAG_GENERIC if generic else 0)
        self.layouts = [abi.stencil_batch_layout(self.h, i) for i in range(len(self.shapes))]
        # one arena per time level; each grid starts on a 256-byte boundary
        es = torch.tensor([], dtype=dtype).element_size()
        align = 256 // es
        offs, total = [], 0
        for pd, _, n in self.layouts:
            offs.append(total)
            total += (n + align - 1) // align * align
        self.arena = [torch.zeros(total, dtype=dtype, device=self.device) for _ in range(2)]
        self.offsets = offs
        self.views = [[self.arena[s][o:o + n].view(pd) for o, (pd, _, n) in zip(offs, self.layouts)] for s in range(2)]
        abi.stencil_batch_bind(self.h, [v.data_ptr() for v in self.views[0]], [v.data_ptr() for v in self.views[1]])

    def interior(self, slot: int, i: int) -> torch.Tensor:
        pd, org, _ = self.layouts[i]
        ny, nx = self.shapes[i]
        return self.views[slot][i][org[0]:org[0] + ny, org[1]:org[1] + nx]

    def set_fields(self, fields) -> None:
        cur = abi.stencil_batch_current(self.h)
        for i, f in enumerate(fields):
            self.interior(cur, i).copy_(_as_tensor(f, self.dtype, self.device))

    def current(self, i: int) -> torch.Tensor:
        return self.interior(abi.stencil_batch_current(self.h), i)

    def tune(self, nsteps: int, stream=None) -> tuple:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        abi.stencil_batch_tune(self.h, nsteps, s)
        return abi.stencil_batch_config(self.h)

    def step(self, nsteps: int, stream=None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        abi.stencil_batch_step(self.h, nsteps, s)

    def sync(self) -> None:
        abi.stencil_batch_sync(self.h)

    def close(self) -> None:
        if getattr(self, "h", None):
            abi.stencil_batch_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


class Cavity:
    """Lid-driven cavity flow on (ny, nx) arrays u, v, p (boundary included),
    borrowed by the library's stencil_cavity_* handle."""

    def __init__(self, ny, nx, dx, dy, dt, rho=1.0, nu=0.1, nit=50, lid=1.0, dtype=torch.float64, device=None):
        self.shape = (int(ny), int(nx))
        self.dtype = dtype
        self.device = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.h = abi.stencil_cavity_create(ny, nx, dx, dy, dt, rho, nu, nit, lid, _ST_DTYPE[dtype])
        self.u, self.v, self.p = (torch.zeros(self.shape, dtype=dtype, device=self.device) for _ in range(3))
        abi.stencil_cavity_bind(self.h, self.u.data_ptr(), self.v.data_ptr(), self.p.data_ptr())

    def set(self, u, v, p) -> None:
        for t, x in ((self.u, u), (self.v, v), (self.p, p)):
            t.copy_(_as_tensor(x, self.dtype, self.device))

    def step(self, nsteps: int, stream=None) -> None:
        s = stream if stream is not None else torch.cuda.current_stream(self.device)
        abi.stencil_cavity_step(self.h, nsteps, s)

    def close(self) -> None:
        if getattr(self, "h", None):
            abi.stencil_cavity_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


# ---------------------------------------------------------------------------
# Differentiation
# ---------------------------------------------------------------------------
class VarCoefProblem:
    """u_{t+1} = sum_k (alpha_k + beta_k kappa) u_t[p + o_k] run for nsteps with
    checkpoints every ckpt_every steps; gradient of 0.5||u_T - target||^2.

    The forward run also keeps the inner levels of its last segment, so the
    reverse pass recomputes every segment but that one: ckpt_every = nsteps
    keeps every level (nsteps fields of workspace, nothing recomputed, the
    fastest reverse pass), small ckpt_every trades recomputation for memory.
    """

    def __init__(self, grid: Grid, nsteps: int, ckpt_every: int):
        self.grid, self.nsteps, self.m = grid, int(nsteps), int(ckpt_every)
        nbytes = abi.stencil_adjoint_workspace(grid.h, self.nsteps, self.m)
        self.ws = torch.empty(max(nbytes, 16), dtype=torch.uint8, device=grid.device)
        self.lam = grid.new_field()
        self.lam_tmp = grid.new_field()
        self.gk = grid.new_field(torch.float64)
        self.loss = torch.zeros(1, dtype=torch.float64, device=grid.device)
        # One workspace records one forward run: `generation` counts the runs,
        # and `recorded` is (run, coefficient generation of the grid) of the
        # run the workspace now holds.
        self.generation = 0
        self.recorded = None

    def forward(self, u0, kappa=None, stream=None):
        g = self.grid
        _before_torch_copies(stream, g.device)
        abi.stencil_set_current(g.h, ST_SLOT_A)
        g.set_field(u0, ST_SLOT_A)
        if kappa is not None:
            g.set_coeff(kappa)
        s = _after_torch_copies(stream, g.device)
        abi.stencil_step_ckpt(g.h, self.nsteps, self.m, self.ws.data_ptr(), s)
        self.generation += 1
        self.recorded = (self.generation, g.coeff_generation)
        return g.current()

    def record_valid(self, record) -> bool:
        """True while the workspace and the bound coefficients still belong to
        the forward run identified by `record` (a value of `recorded`)."""
        return record is not None and record == self.recorded and record[1] == self.grid.coeff_generation

    def backward_from(self, lam_T=None, target=None, stream=None):
        """Reverse pass.  Either lam_T (dL/du_T) or target (then the library
        forms lambda_T = u_T - target and the loss) must be given."""
        g = self.grid
        _before_torch_copies(stream, g.device)
        if target is not None:
            tgt = g.new_field()
            g.interior(tgt).copy_(_as_tensor(target, g.dtype, g.device))
            s = _after_torch_copies(stream, g.device)
            cur = g.bufs[g.current_slot()]
            abi.stencil_residual(g.h, cur.data_ptr(), tgt.data_ptr(), self.lam.data_ptr(), self.loss.data_ptr(), s)
            if s != torch.cuda.current_stream(g.device):
                tgt.record_stream(s)  # freed here, still read by the residual on s
        else:
            self.lam.zero_()
            g.interior(self.lam).copy_(_as_tensor(lam_T, g.dtype, g.device))
        self.gk.zero_()
        s = _after_torch_copies(stream, g.device)
        abi.stencil_adjoint(g.h, self.nsteps, self.m, self.ws.data_ptr(), self.lam.data_ptr(),
                            self.lam_tmp.data_ptr(), self.gk.data_ptr() if g.coeff is not None else 0, s)
        return g.interior(self.lam), g.interior(self.gk), self.loss


class StencilFn(torch.autograd.Function):
    """u_T = S_kappa^n u_0 as a differentiable torch op.

    forward(u0, kappa, problem) -> u_T ; backward returns (dL/du0, dL/dkappa)
    computed by the library's transpose sweep with checkpoint recomputation.

    The checkpoints live in the problem's one workspace and the coefficients
    in its grid, so a problem records one forward run at a time: applying it
    again, or calling set_coeff on its grid, before the backward of an earlier
    application makes that backward raise RuntimeError instead of returning
    the gradient of another trajectory (use one problem per live graph node).
    The gradients returned are copies, never views of the problem's buffers.
    """

    @staticmethod
    def forward(ctx, u0, kappa, problem: VarCoefProblem):
        ctx.problem = problem
        ctx.u0_dtype = u0.dtype
        ctx.kappa_dtype = kappa.dtype
        out = problem.forward(u0, kappa)
        ctx.record = problem.recorded
        return out.clone()

    @staticmethod
    def backward(ctx, grad_out):
        if not ctx.problem.record_valid(ctx.record):
            raise RuntimeError("StencilFn.backward: the problem's workspace or coefficient field was overwritten "
                               "by a later forward run or set_coeff; use one VarCoefProblem per node")
        lam0, gk, _ = ctx.problem.backward_from(lam_T=grad_out)
        return lam0.to(ctx.u0_dtype, copy=True), gk.to(ctx.kappa_dtype, copy=True), None
