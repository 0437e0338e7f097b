/*
 * stencil.h -- C ABI of the GB300 stencil-sweep library (libstencil.so).
 *
 * The library computes repeated sweeps of a fixed-radius stencil over a
 * structured 2D/3D grid with a ghost (halo) region, the operation that the
 * CharmStencil abstraction ("An Adaptive Distributed Stencil Abstraction for
 * GPUs") compiles every slice-assignment expression into (Sec. III-A,
 * Example 1; Sec. III-C "Code generation"):
 *
 *     u_{t+1}[p] = sum_k w_k(p) * u_t[p + o_k]                      (1)
 *
 * with the per-point weights written in an affine form
 *
 *     w_k(p) = alpha_k + beta_k * kappa[p]                          (2)
 *
 * (beta = NULL: constant weights; otherwise one coefficient field kappa),
 * optionally in a two-level leapfrog form
 *
 *     u_{t+1}[p] = sum_k w_k(p) u_t[p + o_k] - u_{t-1}[p] + s_t [p == src]   (3)
 *
 * The output of a step is never an input of the same step (the paper's
 * dependency rule, Sec. III-A): two buffers are used and swap roles after
 * every step, as `u1, u2 = u2, u1` does in Example 1.
 *
 * Ghost region (Sec. III-C "Data layout"): its width is the largest offset
 * component over all points, as the paper's analysis pass derives it.  The
 * domain lives on one GPU, so the paper's ghost exchange between tiles
 * (Sec. III-C "DAG execution") becomes a device-local boundary rule folded
 * into the sweep: Dirichlet ghosts hold a constant that the sweep never
 * writes (Example 1's boundary ring); periodic neighbours wrap around.
 *
 * Conventions for every entry point
 *   - Return value: ST_OK or a negative st_status.  Nothing aborts or throws
 *     across the ABI; stencil_last_error() gives a thread-local message.
 *   - Device buffers are BORROWED: the caller allocates and frees them and
 *     keeps them alive while a handle uses them.  The library allocates only
 *     its own scratch (status word, reduction partials, source table, batch
 *     tables, tuning copies) in bind/set/tune calls, and the host staging
 *     buffer and copy streams in the first stencil_run_host that needs them;
 *     never in a step.
 *   - Work is enqueued on the caller's CUDA stream (cudaStream_t passed as
 *     void*, NULL = legacy default stream) and is asynchronous, except
 *     stencil_sync() and the *_tune() calls, which synchronise that stream.
 *   - Errors detected on the device (a bounded wait that ran out) set a
 *     per-handle status word that stencil_sync() reports.
 *   - A handle is not thread safe; distinct handles are independent.
 *
 * Layout of a field buffer (one per time level, plus the coefficient field)
 *   Padded C-order array  [nz + 2r][ny + 2r][pitch]  (3D)  or
 *                         [ny + 2r][pitch]           (2D),
 *   x fastest.  The interior point (z, y, x) sits at padded index
 *   (z + r, y + r, x + xl) where xl >= r is chosen so the first interior
 *   column is 16-byte aligned; pitch >= xl + nx + r is a multiple of 16 bytes.
 *   stencil_layout() returns the padded shape and the interior origin.  The
 *   buffer's base address must be 16-byte aligned.  Ghost cells belong to the
 *   library: it (re)writes them before a step when the buffer was bound or
 *   marked dirty, unless the handle was created with ST_FLAG_CALLER_GHOSTS.
 */
#ifndef STENCIL_H
#define STENCIL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct st_grid_s* st_grid_t;
typedef struct st_batch_s* st_batch_t;
typedef struct st_cavity_s* st_cavity_t;

typedef enum {
    ST_OK = 0,
    ST_ERR_ARG = -1,            /* invalid argument (shape, offset, pointer, slot, count) */
    ST_ERR_ALIAS = -2,          /* two bound buffers overlap (output would be read in the same step) */
    ST_ERR_UNSUPPORTED = -3,    /* valid request this build does not implement */
    ST_ERR_CUDA = -4,           /* a CUDA runtime call failed (message has the CUDA error) */
    ST_ERR_DEVICE_TIMEOUT = -5, /* a bounded device-side wait ran out (reported by stencil_sync) */
    ST_ERR_BOUNDS = -6,         /* a device-side bounds check fired (reported by stencil_sync) */
    ST_ERR_OOM = -7,            /* library scratch allocation failed */
    ST_ERR_STATE = -8           /* call out of order (e.g. step before bind) */
} st_status;

typedef enum { ST_F32 = 0, ST_F64 = 1 } st_dtype;
/* Boundary rules (the paper's ghost refresh, Sec. III-C, folded into one GPU):
 *   ST_DIRICHLET  ghost cells hold bc_value (or the caller's values with
 *                 ST_FLAG_CALLER_GHOSTS) and are never written by a sweep;
 *   ST_PERIODIC   neighbour indices wrap around each axis;
 *   ST_NEUMANN    zero flux: before every sweep each ghost cell takes the
 *                 value of its mirror image across the boundary face (index
 *                 i < 0 reads -1 - i, i >= n reads 2n - 1 - i, per axis);
 *                 needs every extent >= radius; constant weights, one time
 *                 level and single grids only (otherwise stencil_create
 *                 returns ST_ERR_UNSUPPORTED; the batched form ST_ERR_ARG);
 *                 2D grids take the one-thread-per-point kernel, 3D grids
 *                 single sweeps; stencil_step_ckpt and stencil_adjoint
 *                 give the gradient with respect to u_0 through the
 *                 transpose of the mirror-then-sweep step. */
typedef enum { ST_DIRICHLET = 0, ST_PERIODIC = 1, ST_NEUMANN = 2 } st_bc;

/* stencil_create flags */
#define ST_FLAG_GENERIC 1u   /* always use the one-thread-per-point kernel (the
                                paper's generated-kernel shape, Sec. III-C) */
#define ST_FLAG_TWO_STEP 2u  /* start with two sweeps per pass over HBM where
                                supported (FP32 constant symmetric 3D 7-point
                                star); stencil_tune may change the choice */
#define ST_FLAG_CALLER_GHOSTS 4u  /* Dirichlet ghost cells hold the caller's
                                values (any value per cell: per-face or
                                varying boundary data, such as Example 1's
                                boundary ring when its edges differ, Sec.
                                III-A): the library never writes them and every
                                sweep reads them, and bc_value is ignored.  The
                                caller fills the ghosts of both time-level
                                buffers (stencil_layout gives the layout).
                                Dirichlet only (ST_ERR_ARG with periodic);
                                2D grids then take the one-thread-per-point
                                kernel, 3D grids single sweeps; the adjoint
                                and stencil_step_ckpt return
                                ST_ERR_UNSUPPORTED */

#define ST_FLAG_TILE_PASSES 8u  /* FP64 2D grids whose offsets lie in the 3x3
                                neighbourhood (one time level, constant
                                weights, Dirichlet or periodic): start on the
                                tile kernel, k steps per shared-memory pass and
                                one dependent launch per pass, instead of the
                                one-thread-per-point kernel; stencil_tune
                                times both and keeps the faster either way.
                                Ignored for other grids */


#define ST_MAX_POINTS 64     /* most neighbour points per stencil */
#define ST_MAX_RADIUS 8      /* widest ghost region */

/* Slots of stencil_bind */
#define ST_SLOT_A 0          /* time level buffer A */
#define ST_SLOT_B 1          /* time level buffer B */
#define ST_SLOT_COEFF 2      /* coefficient field kappa of (2) */

/* Library version string. */
const char* stencil_version(void);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* stencil_last_error(void);

/*
 * Create a grid handle for the update (1)-(3).
 *   ndim        2 or 3.
 *   dims        interior extents in C order: {ny, nx} or {nz, ny, nx}, each >= 1.
 *   radius      ghost width; 0 derives it as max |offset component| (the
 *               paper's analysis pass, Sec. III-C); a larger value is kept.
 *   npts        number of neighbour points, 1..ST_MAX_POINTS.
 *   offsets     npts*ndim int32, point k's offset in C order ({dy,dx} or
 *               {dz,dy,dx}); |component| <= ST_MAX_RADIUS, and with a
 *               periodic boundary |component| < the extent of its axis.
 *   alpha       npts doubles (the constant part of each weight).
 *   beta        npts doubles, or NULL for constant weights; non-NULL
 *               requires a coefficient buffer bound at ST_SLOT_COEFF.
 *   bc          ST_DIRICHLET (ghosts = bc_value), ST_PERIODIC or ST_NEUMANN.
 *   dtype       storage and arithmetic type of the fields.
 *   time_levels 1: form (1); 2: leapfrog form (3).
 *   flags       0 or a combination of ST_FLAG_GENERIC, ST_FLAG_TWO_STEP,
 *               ST_FLAG_CALLER_GHOSTS and ST_FLAG_TILE_PASSES.
 * Copies all arrays; allocates only library scratch.  *out is NULL on error.
 */
st_status stencil_create(st_grid_t* out, int ndim, const int64_t* dims, int radius, int npts,
                         const int32_t* offsets, const double* alpha, const double* beta,
                         st_bc bc, double bc_value, st_dtype dtype, int time_levels,
                         uint32_t flags);

/*
 * Create a grid handle for per-cell diffusion in conservative (face-averaged)
 * form, the variable-coefficient operator of (1)-(2) written with face
 * coefficients so that a periodic grid conserves sum(u) whatever kappa is:
 *     u_{t+1}[p] = u_t[p] + sum over the 2*ndim axis neighbours q of p of
 *                  k_pq (u_t[q] - u_t[p]),
 *     k_pq = (kappa[p] + kappa[q]) / 2 for an interior (or wrapped) q,
 *     k_pq = kappa[p] for a Dirichlet ghost q (u_t[q] = bc_value).
 * Radius 1; the coefficient field is bound at ST_SLOT_COEFF.  Everything
 * else (bind, step, stencil_step_ckpt, stencil_adjoint, run_host, reductions)
 * works as for a stencil_create handle; the adjoint's gradient is dL/dkappa
 * of this operator (its matrix is symmetric, so a transposed step is the
 * same sweep on lambda).  One thread per point.  bc: ST_DIRICHLET or
 * ST_PERIODIC (ST_ERR_ARG otherwise); flags must be 0.
 */
st_status stencil_create_conservative(st_grid_t* out, int ndim, const int64_t* dims, st_bc bc, double bc_value,
                                      st_dtype dtype, uint32_t flags);

/* Release the handle and its scratch (not the borrowed buffers).  NULL is a no-op. */
st_status stencil_destroy(st_grid_t g);

/*
 * Layout of every field-shaped buffer of this grid (see the header comment).
 *   padded_dims  ndim int64: padded extents in C order (last one = pitch).
 *   origin       ndim int64: padded index of interior point 0.
 *   elems        total element count of one buffer.
 * Any output pointer may be NULL.
 */
st_status stencil_layout(st_grid_t g, int64_t* padded_dims, int64_t* origin, int64_t* elems);

/* Radius, point count and the kernel family the handle dispatches to
 * (name is a static string, e.g. "star3d_r1_tma"). */
st_status stencil_info(st_grid_t g, int* radius, int* npts, const char** kernel_name);

/*
 * Bind a device buffer (layout above, the grid's dtype) to a slot:
 * ST_SLOT_A / ST_SLOT_B (time levels) or ST_SLOT_COEFF.  Overlap with another
 * bound slot is ST_ERR_ALIAS.  Binding marks the buffer's ghosts stale.
 * Binding slot A makes it the current level.
 */
st_status stencil_bind(st_grid_t g, int slot, void* dev_ptr);

/* Tell the library the caller rewrote a bound buffer: its ghosts are
 * refreshed before the next step (the paper's generation epochs, Sec. III-C). */
st_status stencil_mark_dirty(st_grid_t g, int slot);

/* Which time-level slot (ST_SLOT_A or ST_SLOT_B) holds the newest level u_t.
 * With two time levels the other slot holds u_{t-1}; with one, the other
 * slot holds an older level (u_{t-1}, or u_{t-2} after a two-step pass). */
st_status stencil_current(st_grid_t g, int* slot);
st_status stencil_set_current(st_grid_t g, int slot);

/*
 * Defined by: the leapfrog acoustic-wave workload (a Ricker-wavelet point
 * source injected at the centre cell every step), which extends (1) to the
 * two-level form (3); the paper's own workloads have no source term.
 * Point source of the leapfrog form (3): amplitudes[t] is added at interior
 * point `index` (ndim int64, C order) by the step that computes level t+1,
 * where t is the handle's step counter.  Steps past `count` add nothing.
 * Copies the host amplitudes to library scratch.  count = 0 removes it.
 */
st_status stencil_set_source(st_grid_t g, const int64_t* index, const double* amplitudes,
                             int64_t count);

/* Set / read the step counter t used by the source (0 after create). */
st_status stencil_set_step_index(st_grid_t g, int64_t t);
st_status stencil_get_step_index(st_grid_t g, int64_t* t);

/*
 * Device-resident snapshot and restore of a grid's state, the single-process
 * form of the paper's rescale checkpoint (Sec. IV "Checkpoint and restart":
 * GPU data is parked in device memory owned by someone else, a memory daemon
 * there, and copied back device to device, avoiding the host link).
 *   stencil_snapshot_bytes: bytes of a snapshot = time_levels whole padded
 *     buffers (stencil_layout's elems each).
 *   stencil_snapshot: enqueues device-to-device copies of the newest level
 *     (then, with two time levels, the previous level) into dst (device,
 *     caller-owned, 16-byte aligned, >= stencil_snapshot_bytes) on `stream`
 *     and returns the step counter in *step_out.  The snapshot does not
 *     depend on the handle: dst may outlive it and its buffers.
 *   stencil_restore: enqueues the copies back into slot A (newest) and slot B
 *     (previous, two levels), makes slot A current and sets the step counter;
 *     the snapshot must come from a grid of the same layout and dtype.  Ghost
 *     cells owned by the library are rewritten before the next step; with
 *     ST_FLAG_CALLER_GHOSTS they are the snapshot's.
 * Both slots must be bound (ST_ERR_STATE otherwise).
 */
st_status stencil_snapshot_bytes(st_grid_t g, size_t* bytes);
st_status stencil_snapshot(st_grid_t g, void* dst, int64_t* step_out, void* stream);
st_status stencil_restore(st_grid_t g, const void* src, int64_t step, void* stream);

/*
 * Defined by: Sec. III-A, Example 1 (the loop that applies one stencil
 * expression per iteration and swaps the two arrays, `u1, u2 = u2, u1`) and
 * Sec. III-C "DAG execution" (a node runs in two phases: the ghost data of
 * its input arrays is brought up to date, only where the generation epochs
 * differ, then the kernel runs).  nsteps steps are nsteps such nodes.
 * Advance nsteps >= 0 steps on `stream`: refresh stale ghosts, then sweep,
 * each launch writing the other slot.  When stencil_tune chose two-step
 * passes (the constant symmetric 7-point star, FP32, no source) a launch
 * advances two steps, and when it chose the k-step static-tile kernel (FP64
 * 2D grids) a launch advances up to k steps (temporal blocking; the results
 * equal single steps bit for bit), so the newest level's slot follows the
 * launch count:
 * stencil_current() tells which.  Enqueued as one
 * CUDA graph per (handle, nsteps, current slot) after the first call with
 * that nsteps; the launch sequence is the same either way.
 */
st_status stencil_step(st_grid_t g, int nsteps, void* stream);

/*
 * Autotune the launch configuration of this grid for nsteps-step calls (2D
 * grids on the persistent tile kernel: tile shape, threads per block, steps
 * per shared-memory pass; FP64 2D grids within the 3x3 neighbourhood
 * (constant weights, no source): the one-thread-per-point kernel, the tuned
 * tile kernel with one dependent launch per pass, and a static-tile kernel
 * running k steps per launch in shared memory over several tile shapes and
 * k in 1..8 (the same bits as single sweeps), keeping the fastest; the FP32 constant
 * symmetric 3D 7-point star: one sweep or two sweeps per pass over HBM;
 * other families have nothing to tune and return ST_OK).  Times the candidates on the bound data and restores the
 * current level afterwards (the other slot is scratch); synchronises
 * `stream`.  With temporal blocking a call may leave the newest level in
 * either slot: stencil_current() tells which.
 */
st_status stencil_tune(st_grid_t g, int nsteps, void* stream);

/* The configuration in use (cfg[0] tile x, cfg[1] tile y, cfg[2] threads,
 * cfg[3] steps per pass; 3D 7-point star: zeros and the steps per pass);
 * zeros for families without one and for FP64 2D grids on the
 * one-thread-per-point kernel. */
st_status stencil_tune_config(st_grid_t g, int* cfg);

/*
 * Defined by: Sec. III-B, the frontend's arrays filled from host data and
 * read back with get() around the run of nodes that sync() executes; here
 * that round trip is one call.
 * End-to-end form of stencil_step for callers whose data is on the host:
 * copies host_u0 (dense interior, C order, the grid's dtype) into the current
 * level, runs nsteps, copies the newest level's interior to host_uT.  A
 * pinned (page-locked, device-mapped) host buffer is read or written directly
 * by the device (un)pack kernel.  Any other host buffer goes through a dense
 * device staging buffer: a contiguous copy split in four pieces on the
 * handle's own copy streams (forked from and joined back into `stream` by
 * events) plus the (un)pack kernel; the first such call allocates the buffer
 * (interior size) and the streams, later calls reuse them.  Everything is
 * ordered on `stream` and the call returns after enqueueing (with pageable
 * host memory the copies may block the calling thread).  One time level only.
 */
st_status stencil_run_host(st_grid_t g, int nsteps, const void* host_u0, void* host_uT,
                           void* stream);

/*
 * Defined by: the same round trip as stencil_run_host (Sec. III-B), for the
 * end-to-end measurement of a workload run again and again on new host
 * data; the paper has no batched form of it.
 * Pipelined form of stencil_run_host for a stream of independent jobs on
 * one grid (each its own initial field): for i in [0, njobs), copies
 * host_in[i] (dense interior, C order, the grid's dtype) into the current
 * level, runs nsteps, and copies the newest level's interior to
 * host_out[i].  The host copies run on the copy engines, on the handle's
 * copy streams: job i+1's input arrives and job i-1's result leaves while
 * job i sweeps, so with pinned host buffers the host traffic overlaps the
 * sweeps (pageable buffers work, but their copies may block the calling
 * thread and overlap nothing).  Inputs are copied by rows into a
 * field-layout buffer that the job's first sweep reads, and every job's
 * last sweep but the last job's writes another one that is copied out; a
 * zero-flux or caller-ghost boundary, a source, a 2D grid on the tile
 * kernel or nsteps = 0 use dense staging buffers and pack kernels instead.
 * The buffers (field or interior size) are allocated by the first call that
 * needs them and reused.  Every job's result has the bits stencil_run_host
 * gives for its input, and afterwards the current level holds the last
 * job's result.  Every copy and
 * kernel of the call is ordered after the caller's earlier work on
 * `stream`, and everything later on `stream` after all of them: the
 * results are on the host once `stream` reaches that point.  Jobs run in
 * order; host_out[i] may equal host_out[j] (the later job's result stays)
 * but must not overlap any host_in[k].  njobs = 0 does nothing.  One time
 * level only.
 */
st_status stencil_run_host_many(st_grid_t g, int nsteps, int njobs, const void* const* host_in,
                                void* const* host_out, void* stream);

/* Defined by: Sec. III-B "Execution graph" (the frontend's sync call hands
 * the recorded work to the backend and returns when it has run) and Sec.
 * II-A "Asynchronous detection of kernel completion" (the host learns of a
 * kernel's completion without blocking other work until it asks).
 * Synchronise the last stream used by this handle and report device-side
 * errors (ST_ERR_DEVICE_TIMEOUT, ST_ERR_BOUNDS); clears the status word. */
st_status stencil_sync(st_grid_t g);

/*
 * Defined by: the FP64 residual and norm reductions that the workloads keep
 * in double precision on the GPU (sums and error norms of a field, the
 * loss of the adjoint workload); the paper's Laplace and cavity programs
 * read results back with get() and have no reduction of their own.
 * Interior reductions in double precision over a (and b, if not NULL), two
 * buffers in this grid's layout and dtype:
 *   dev_out[0] = sum (a - b), dev_out[1] = sum (a - b)^2, dev_out[2] = max |a - b|.
 * dev_out: 3 doubles in device memory.  a and b must be 16-byte aligned
 * (ST_ERR_ARG otherwise; buffers from the library's own allocations and
 * torch's are).  Deterministic: fixed block partials summed in a fixed order
 * by a second pass.  A timed-out wait inside the FP32 kernel is reported by
 * the next stencil_sync (ST_ERR_DEVICE_TIMEOUT).
 */
st_status stencil_reduce(st_grid_t g, const void* a, const void* b, double* dev_out,
                         void* stream);

/*
 * Allocation-free form of stencil_reduce (the paper has no counterpart: its
 * runtime allocates freely).  For callers that cannot allocate device
 * memory at call time: an application whose device memory is entirely owned
 * by another allocator (a framework's caching pool that has reserved the
 * GPU), a latency-critical loop that cannot afford cudaMalloc's implicit
 * device synchronisation, or code that must not fail with out-of-memory
 * after start-up.  stencil_reduce takes its per-block partial sums from
 * handle scratch that its first call allocates; this entry point takes them
 * from a static device array instead and calls no cudaMalloc, cudaFree or
 * other allocating routine.
 *   Same arguments and results as stencil_reduce (a, b: 16-byte aligned
 *   field-layout buffers of the grid's dtype, b may be NULL; dev_out: 3
 *   doubles in device memory).
 *   Scratch: a static array of 4096 block partials (96 KB, held by every
 *   GPU that loads the library until the process exits).  The blocks walk
 *   the interior rows in a grid-stride loop, so grids of every size fit it
 *   and none is rejected.
 *   The first call on a device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   All calls share the one array: every call overwrites the partials it
 *   uses before reading them, so nothing needs clearing, but two calls whose
 *   work overlaps on the GPU (different streams, no ordering) race on it.
 *   Results agree with stencil_reduce up to summation order.
 */
st_status stencil_reduce_noalloc(st_grid_t g, const void* a, const void* b, double* dev_out, void* stream);

/*
 * Defined by: Sec. III-A, Example 1's loop of stencil steps followed by a
 * read of a result (the configurations reduce the field after its steps:
 * the heat workload's norms, in double precision).
 * stencil_step(g, nsteps) followed by stencil_reduce of the newest level
 * (dev_out[0..2] = sum u, sum u^2, max |u| over the interior, in double
 * precision).  For a constant symmetric 3D 7-point star in FP32 (Dirichlet or
 * periodic, no source) the last sweep computes the reduction of the values
 * it writes (compensated float pairs per thread, combined in double in a
 * fixed order), so the step reads its field once; results are deterministic
 * and agree with stencil_reduce to its precision (about 1e-13 relative to
 * sum |u|), not bit for bit.  Other grids run the two calls.  nsteps = 0
 * reduces the current level.
 */
st_status stencil_step_reduce(st_grid_t g, int nsteps, double* dev_out, void* stream);

/*
 * Defined by: the adjoint workload's loss L = 0.5 ||u_T - u_target||^2, whose
 * gradient dL/du_T = u_T - u_target seeds the transpose sweep; no
 * counterpart in the paper.
 * Loss residual: lambda = u - target on the interior (lambda's ghosts set to
 * 0) and dev_loss[0] = 0.5 * sum (u - target)^2 in double precision.
 * u, target and lambda must be 16-byte aligned (ST_ERR_ARG otherwise).
 */
st_status stencil_residual(st_grid_t g, const void* u, const void* target, void* lambda,
                           double* dev_loss, void* stream);

/*
 * Defined by: the adjoint workload (a hand-written transposed-stencil sweep
 * giving the gradients of a loss of u_T with respect to u_0 and to the
 * per-cell coefficients of (2), with the forward states checkpointed every
 * m steps and recomputed segment by segment); the paper differentiates
 * nothing, so the operation is the exact transpose of the linear map (1)-(2).
 * Adjoint with checkpoint-every-m recomputation (one time level only).
 * Workspace bytes for a run of nsteps with checkpoints every ckpt_every steps:
 * ceil(nsteps/ckpt_every) checkpoints, ckpt_every-1 levels for the
 * recomputation of a segment, and the ckpt_every-1 inner levels of the last
 * segment, which the forward run keeps so that the reverse pass need not
 * recompute them; for a 3D handle of stencil_create_conservative, also
 * ckpt_every-1 levels of lambda (its reverse pass runs a segment's
 * transposed steps first and the segment's coefficient gradient after, in
 * one pass over the kept lambda levels); for an FP32 handle of the 3D
 * symmetric 7-point star with per-cell weights (its fused two-step
 * transpose), also one level of FP32 for the partial coefficient gradient
 * of a segment.
 */
st_status stencil_adjoint_workspace(st_grid_t g, int nsteps, int ckpt_every, size_t* bytes);

/* Defined by: the adjoint workload's checkpoint-every-m forward run (see
 * stencil_adjoint_workspace); each step is the sweep of stencil_step.
 * Forward nsteps from the current level, storing u at t = 0, m, 2m, ... and
 * the inner levels of the last segment in `workspace` (device,
 * >= stencil_adjoint_workspace bytes, 16-byte aligned).  With two segments
 * or more it also stores the inner levels of the second-to-last segment, in
 * the recomputation levels (idle until the reverse pass reaches that
 * segment), so that the first stencil_adjoint on this record recomputes one
 * segment fewer; the handle remembers which workspace holds them. */
st_status stencil_step_ckpt(st_grid_t g, int nsteps, int ckpt_every, void* workspace,
                            void* stream);

/*
 * Defined by: the adjoint workload (see stencil_adjoint_workspace).
 * Reverse pass of a run recorded by stencil_step_ckpt with the same nsteps
 * and ckpt_every (it never writes the interiors of the checkpoints or the
 * last segment's levels, so it may run again on the same record; the
 * second-to-last segment is read from the recomputation levels on the first
 * reverse pass after the record and recomputed on later ones, whose
 * recomputations have overwritten them; with ST_NEUMANN it refreshes the
 * mirror ghosts of the levels it reads from their interiors).  lambda (in: dL/du_T, out: dL/du_0) and lambda_tmp are
 * field-layout buffers of the grid's dtype; grad_coeff (may be NULL) is a
 * field-layout buffer of DOUBLES into which
 *     sum_t lambda_{t+1}[p] * sum_k beta_k u_t[p + o_k]     (= dL/dkappa_p)
 * is ACCUMULATED (+=): in double per pass, except that an FP32 handle on
 * the fused 3D transpose (see stencil_adjoint_workspace) first sums a
 * checkpoint segment's terms in FP32 and adds that sum in double once per
 * segment, so its gradient depends on ckpt_every by those roundings.  The
 * transpose step is
 *     lambda_t[q] = sum_k w_k(q - o_k) lambda_{t+1}[q - o_k],
 * over the points q - o_k that are interior (wrapped when periodic); ghost
 * cells are boundary data, not variables.  With ST_NEUMANN a step reads
 * u[mirror(p + o_k)], so its transpose sends w_k lambda_{t+1}[p] to the
 * mirror image: lambda_t[q] = sum_k w_k sum over the cells g with
 * mirror(g) = q of lambda_{t+1}[g - o_k] (g - o_k interior; constant weights,
 * so grad_coeff must be NULL).  The current level is unchanged.
 * workspace, lambda, lambda_tmp and grad_coeff are 16-byte aligned
 * (ST_ERR_ARG otherwise).
 */
st_status stencil_adjoint(st_grid_t g, int nsteps, int ckpt_every, const void* workspace,
                          void* lambda, void* lambda_tmp, double* grad_coeff, void* stream);

/* ----------------------------------------------------------------------------
 * Batched form: many independent 2D grids with the same neighbour offsets,
 * their own sizes and weights, advanced by one persistent launch per call.
 * Defined by: the batched workload (many independent grids of uneven sizes
 * swept in one persistent launch under a captured CUDA graph, with the tile
 * shape, threads per block and temporal-blocking depth picked by an
 * autotuner); its nearest counterpart in the paper is node fusion (Sec.
 * III-B "Node fusion": independent updates of arrays of one output shape
 * compiled into one kernel to save launches), which the frontend lowers
 * onto this form.
 * --------------------------------------------------------------------------*/

/*
 * ngrids >= 1; dims: ngrids*2 int64 {ny, nx}; offsets: npts*2 int32 {dy, dx}
 * shared by all grids; weights: ngrids*npts doubles (constant per grid).
 */
st_status stencil_batch_create(st_batch_t* out, int ngrids, const int64_t* dims, int npts,
                               const int32_t* offsets, const double* weights, st_bc bc,
                               double bc_value, st_dtype dtype, uint32_t flags);
st_status stencil_batch_destroy(st_batch_t b);

/* Layout of grid g (same rules as stencil_layout, 2D). */
st_status stencil_batch_layout(st_batch_t b, int g, int64_t* padded_dims, int64_t* origin,
                               int64_t* elems);

/* Bind both time levels of every grid: host arrays of ngrids device pointers. */
st_status stencil_batch_bind(st_batch_t b, void* const* dev_ptrs_a, void* const* dev_ptrs_b);

/*
 * Autotune the launch configuration for nsteps-step calls: times each
 * candidate (tile shape, threads per block, steps per pass) on the bound data
 * and keeps the fastest; the bound buffers are restored afterwards.
 * Synchronises `stream`.  Without a call a default configuration is used.
 */
st_status stencil_batch_tune(st_batch_t b, int nsteps, void* stream);

/* The configuration in use: cfg[0] tile x, cfg[1] tile y, cfg[2] threads,
 * cfg[3] steps per pass. */
st_status stencil_batch_config(st_batch_t b, int* cfg);

/* Advance every grid nsteps steps.  With temporal blocking the result may end
 * in either slot: stencil_batch_current() tells which. */
st_status stencil_batch_step(st_batch_t b, int nsteps, void* stream);
st_status stencil_batch_current(st_batch_t b, int* slot);
st_status stencil_batch_sync(st_batch_t b);

/*
 * Failure-detection hook (no counterpart in the paper, whose runtime detects
 * no device failures): advances every grid one step with the persistent
 * kernel and then enters a grid-wide barrier that waits for one CTA more than
 * were launched.  The barrier's bounded wait runs out after timeout_ns
 * (1 ms .. 5 s), the kernel records ST_ERR_DEVICE_TIMEOUT in the status word
 * and returns; stencil_batch_sync() then reports ST_ERR_DEVICE_TIMEOUT and the
 * context stays usable.  ST_ERR_UNSUPPORTED for plans without the persistent
 * kernel (ST_FLAG_GENERIC or offsets beyond the 3x3 neighbourhood).
 */
st_status stencil_batch_selftest_barrier(st_batch_t b, uint64_t timeout_ns, void* stream);

/* ----------------------------------------------------------------------------
 * Lid-driven cavity flow: the paper's multi-field benchmark (Sec. V-B, a
 * Navier-Stokes solver written as NumPy slice assignments over u, v, p and a
 * pressure source b).  Arrays are dense (ny, nx), C order, boundary rows and
 * columns included, y along axis 0 and x along axis 1; the lid is the last
 * row.  One time step:
 *   1. b = rho ((ux + vy) / dt - ux^2 - 2 uy vx - vy^2) at interior points,
 *      central differences (ux = (u[j][i+1] - u[j][i-1]) / (2 dx), ...);
 *   2. nit Jacobi iterations p = ((p_e + p_w) dy^2 + (p_n + p_s) dx^2
 *      - b dx^2 dy^2) / (2 (dx^2 + dy^2)) at interior points, each followed
 *      by the boundary rule: right column = its left neighbour, bottom row =
 *      the row above, left column = its right neighbour, top row = 0;
 *   3. u, v from the old velocities (backward differences for advection,
 *      central for the pressure gradient and diffusion, viscosity nu,
 *      density rho), then u = v = 0 on the walls and u = lid, v = 0 on the
 *      top row.
 * The momentum updates of u and v run fused in one kernel.
 * --------------------------------------------------------------------------*/

/* ny, nx in [3, 2^19] x [3, 2^24]; dx, dy, dt, rho > 0; nu >= 0; nit >= 0. */
st_status stencil_cavity_create(st_cavity_t* out, int64_t ny, int64_t nx, double dx, double dy, double dt,
                                double rho, double nu, int nit, double lid, st_dtype dtype);
st_status stencil_cavity_destroy(st_cavity_t c);

/* Borrow the caller's u, v and p (device, ny*nx elements of the handle's
 * dtype each, element-aligned, not overlapping: ST_ERR_ALIAS).  The first
 * bind allocates the handle's scratch (a second buffer per field and b). */
st_status stencil_cavity_bind(st_cavity_t c, void* u, void* v, void* p);

/* Advance nsteps time steps on `stream`; the bound buffers hold the result
 * when the enqueued work completes. */
st_status stencil_cavity_step(st_cavity_t c, int nsteps, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* STENCIL_H */
