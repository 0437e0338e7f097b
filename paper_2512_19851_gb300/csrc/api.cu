// Host side of the C ABI declared in include/stencil.h: handle life cycle,
// argument validation, the padded layout, ghost refresh, the step driver
// (CUDA graphs of the sweep launches), checkpointed adjoint, reductions and
// the batched form.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

#include "cavity.cuh"
#include "common.cuh"
#include "families.cuh"

namespace st {

static thread_local std::string t_err;

void set_error(const std::string& msg) { t_err = msg; }

st_status fail(st_status code, const std::string& msg)
{
    t_err = msg;
    return code;
}

st_status cuda_fail(cudaError_t e, const char* what)
{
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    (void)cudaGetLastError();  // clear a sticky launch error of this thread
    return ST_ERR_CUDA;
}

static int64_t round_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

Geom make_geom(int ndim, const int64_t* dims, int r, int esize)
{
    Geom g{};
    g.ndim = ndim;
    g.r = r;
    g.rz = (ndim == 3) ? r : 0;
    g.esize = esize;
    g.nz = (ndim == 3) ? dims[0] : 1;
    g.ny = dims[ndim - 2];
    g.nx = dims[ndim - 1];
    const int64_t a = 16 / esize;  // elements per 16 bytes
    g.xl = round_up(r, a);
    g.pitch = round_up(g.xl + g.nx + r, a);
    g.pny = g.ny + 2 * r;
    g.pnz = g.nz + 2 * g.rz;
    g.plane = g.pny * g.pitch;
    g.elems = g.pnz * g.plane;
    g.origin = g.rz * g.plane + (int64_t)r * g.pitch + g.xl;
    g.npoints = g.nz * g.ny * g.nx;
    return g;
}

}  // namespace st

using namespace st;

// ---------------------------------------------------------------------------
// Grid handle
// ---------------------------------------------------------------------------
struct st_grid_s {
    Geom g{};
    int npts = 0;
    int radius = 0;
    std::vector<int32_t> off;  // npts * 3: dz, dy, dx (dz = 0 in 2D)
    std::vector<double> alpha, beta;
    bool has_beta = false;
    st_bc bc = ST_DIRICHLET;
    double bc_value = 0.0;
    st_dtype dtype = ST_F64;
    int levels = 1;
    uint32_t flags = 0;
    Family fam{};

    void* buf[3] = {nullptr, nullptr, nullptr};
    bool stale[3] = {false, false, false};
    int cur = ST_SLOT_A;
    int64_t step = 0;

    int64_t src = -1;
    double* d_src = nullptr;
    int64_t src_count = 0;

    bool scratch = false;
    int device = -1;
    int* d_status = nullptr;
    double* d_partials = nullptr;
    int red_blocks = 0;
    cudaStream_t cap = nullptr;
    cudaStream_t last = nullptr;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
    BatchPlan* plan = nullptr;  // 2D grids on the persistent tile kernel (a batch of one)
    bool plan_bound = false;
    // FP64 2D grids: the tile kernel (one launch per pass of k steps) is an
    // option that stencil_tune takes only where it times faster than the
    // one-thread-per-point kernel; plan_use tells which runs
    bool plan_optional = false;
    bool plan_use = true;
    // the same FP64 2D grids on k_tb2d: tile x, tile y, steps per launch
    // (tb[2] == 0: not in use); chosen by stencil_tune, or by ST_TB2D_CFG
    int tb[3] = {0, 0, 0};
    // the workspace whose recomputation levels hold the inner states of the
    // second-to-last segment, written by the last stencil_step_ckpt (run of
    // kept2_n steps, checkpoints every kept2_m); cleared once a reverse pass
    // overwrites them
    const void* kept2_ws = nullptr;
    int kept2_n = 0, kept2_m = 0;
    bool pairs = false;         // two-step passes chosen by stencil_tune (3D 7-point heat, FP32)
    bool caller_ghosts = false; // ST_FLAG_CALLER_GHOSTS: Dirichlet ghost cells hold the caller's values
    void* staging = nullptr;    // dense interior buffer of stencil_run_host
    void* staging2 = nullptr;   // stencil_run_host_many: the outgoing dense buffer
    // stencil_run_host_many: field-layout buffers that a job's first sweep
    // reads (its input copied in by the copy engines) and its last sweep
    // writes (copied out from there)
    void* pad_in = nullptr;
    void* pad_out = nullptr;
    // stencil_run_host splits each host copy over a few streams so that
    // several copy engines share it (created on first use)
    cudaStream_t cstream[4] = {};
    cudaEvent_t cfork = nullptr, cjoin[4] = {};
    cudaEvent_t cpack = nullptr, cunpack = nullptr;  // stencil_run_host_many hand-offs
};

static void drop_graphs(st_grid_t g)
{
    for (auto& kv : g->graphs) cudaGraphExecDestroy(kv.second);
    g->graphs.clear();
}

static st_status ensure_scratch(st_grid_t g)
{
    if (g->scratch) return ST_OK;
    ST_CUDA_TRY(cudaGetDevice(&g->device));
    g->red_blocks = reduce_blocks(g->g, 4096);
    if (cudaMalloc(&g->d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&g->d_partials, sizeof(double) * 3 * g->red_blocks) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ST_ERR_OOM, "stencil_bind: scratch allocation failed");
    }
    ST_CUDA_TRY(cudaMemset(g->d_status, 0, sizeof(int)));
    ST_CUDA_TRY(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
    g->scratch = true;
    return ST_OK;
}

static bool is_star(const std::vector<int32_t>& off, int npts, int ndim)
{
    for (int k = 0; k < npts; ++k) {
        int nz = (off[3 * k] != 0) + (off[3 * k + 1] != 0) + (off[3 * k + 2] != 0);
        if (nz > 1) return false;
        if (ndim == 2 && off[3 * k] != 0) return false;
    }
    return true;
}

extern "C" {

const char* stencil_version(void) { return "gb300-stencil 0.1 (sm_103a)"; }

const char* stencil_last_error(void) { return t_err.c_str(); }

st_status stencil_create(st_grid_t* out, int ndim, const int64_t* dims, int radius, int npts,
                         const int32_t* offsets, const double* alpha, const double* beta,
                         st_bc bc, double bc_value, st_dtype dtype, int time_levels,
                         uint32_t flags)
{
    if (!out) return fail(ST_ERR_ARG, "stencil_create: out is NULL");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(ST_ERR_ARG, "stencil_create: ndim must be 2 or 3");
    if (!dims || !offsets || !alpha) return fail(ST_ERR_ARG, "stencil_create: NULL dims/offsets/alpha");
    if (npts < 1 || npts > ST_MAX_POINTS) return fail(ST_ERR_ARG, "stencil_create: npts out of range");
    if (bc != ST_DIRICHLET && bc != ST_PERIODIC && bc != ST_NEUMANN) return fail(ST_ERR_ARG, "stencil_create: bad bc");
    if (dtype != ST_F32 && dtype != ST_F64) return fail(ST_ERR_ARG, "stencil_create: bad dtype");
    if (time_levels != 1 && time_levels != 2) return fail(ST_ERR_ARG, "stencil_create: time_levels must be 1 or 2");
    if (flags & ~(ST_FLAG_GENERIC | ST_FLAG_TWO_STEP | ST_FLAG_CALLER_GHOSTS | ST_FLAG_TILE_PASSES))
        return fail(ST_ERR_ARG, "stencil_create: unknown flags");
    if ((flags & ST_FLAG_CALLER_GHOSTS) && bc != ST_DIRICHLET)
        return fail(ST_ERR_ARG, "stencil_create: ST_FLAG_CALLER_GHOSTS needs a Dirichlet boundary");
    if (radius < 0 || radius > ST_MAX_RADIUS) return fail(ST_ERR_ARG, "stencil_create: radius out of range");
    int64_t d3[3] = {1, 1, 1};
    for (int i = 0; i < ndim; ++i) {
        if (dims[i] < 1 || dims[i] > (int64_t)1 << 24)
            return fail(ST_ERR_ARG, "stencil_create: extent out of range [1, 2^24]");
        d3[3 - ndim + i] = dims[i];
    }
    if (d3[0] > 65535) return fail(ST_ERR_ARG, "stencil_create: nz > 65535");
    if ((d3[0] + 2 * ST_MAX_RADIUS) * (d3[1] + 2 * ST_MAX_RADIUS) >= ((int64_t)1 << 32))
        return fail(ST_ERR_ARG, "stencil_create: nz * ny beyond 2^32 rows");
    std::vector<int32_t> off(3 * npts, 0);
    int derived = 0;
    for (int k = 0; k < npts; ++k) {
        for (int i = 0; i < ndim; ++i) {
            const int32_t o = offsets[k * ndim + i];
            if (o < -ST_MAX_RADIUS || o > ST_MAX_RADIUS)
                return fail(ST_ERR_ARG, "stencil_create: offset component beyond ST_MAX_RADIUS");
            if (bc == ST_PERIODIC && (int64_t)(o < 0 ? -o : o) >= d3[3 - ndim + i])
                return fail(ST_ERR_ARG, "stencil_create: periodic offset not smaller than the extent");
            off[3 * k + 3 - ndim + i] = o;
            derived = std::max(derived, o < 0 ? -o : o);
        }
    }
    if (radius == 0) radius = derived;
    if (radius < derived) return fail(ST_ERR_ARG, "stencil_create: radius smaller than the largest offset");
    if (bc == ST_NEUMANN && (time_levels != 1 || beta))
        return fail(ST_ERR_UNSUPPORTED, "stencil_create: ST_NEUMANN with one time level and constant weights only");
    if (bc == ST_NEUMANN)
        for (int i = 0; i < ndim; ++i)
            if (dims[i] < radius)
                return fail(ST_ERR_ARG, "stencil_create: a Neumann ghost's mirror image must be interior (extent >= radius)");
    if (bc == ST_DIRICHLET) {
        // the paper's limitation (Sec. III-D): dependence distance within the domain
        for (int i = 0; i < ndim; ++i)
            if (dims[i] < 1) return fail(ST_ERR_ARG, "stencil_create: empty extent");
    }
    for (int k = 0; k < npts; ++k)
        if (!(alpha[k] == alpha[k]) || (beta && !(beta[k] == beta[k])))
            return fail(ST_ERR_ARG, "stencil_create: NaN weight");

    st_grid_t g = new (std::nothrow) st_grid_s();
    if (!g) return fail(ST_ERR_OOM, "stencil_create: out of host memory");
    g->g = make_geom(ndim, dims, radius, dtype == ST_F64 ? 8 : 4);
    g->npts = npts;
    g->radius = radius;
    g->off = off;
    g->alpha.assign(alpha, alpha + npts);
    g->has_beta = beta != nullptr;
    g->beta.assign(npts, 0.0);
    if (beta) g->beta.assign(beta, beta + npts);
    g->bc = bc;
    g->bc_value = bc_value;
    g->dtype = dtype;
    g->levels = time_levels;
    g->flags = flags;
    g->caller_ghosts = (flags & ST_FLAG_CALLER_GHOSTS) != 0;
    // the two-step 3D pass substitutes bc_value for ghost reads, so caller
    // ghosts keep single sweeps
    g->pairs = (flags & ST_FLAG_TWO_STEP) != 0 && !g->caller_ghosts && bc != ST_NEUMANN;
    FamilyDesc d{};
    d.g = g->g;
    d.npts = npts;
    d.off = g->off.data();
    d.alpha = g->alpha.data();
    d.beta = g->beta.data();
    d.has_beta = g->has_beta;
    d.periodic = bc == ST_PERIODIC;
    d.levels = time_levels;
    d.star = is_star(g->off, npts, ndim);
    d.force_generic = (flags & ST_FLAG_GENERIC) != 0;
    g->fam = select_family(d);
    if (g->fam.kind == FAM_2D_TILE && (g->caller_ghosts || bc == ST_NEUMANN)) {
        // the persistent 2D tile kernel substitutes bc_value for points
        // outside the interior; the one-thread-per-point kernel reads the
        // ghost cells themselves
        d.force_generic = true;
        g->fam = select_family(d);
    }
    // FP64 2D grids within the 3x3 neighbourhood may run the tile kernel one
    // launch per pass of k steps (temporal blocking on the FP64 pipe costs
    // redundant halo work, so stencil_tune decides by timing both)
    bool small2d = ndim == 2 && npts <= 9;
    for (int k = 0; k < npts; ++k)
        for (int i = 1; i < 3; ++i)
            if (g->off[3 * k + i] < -1 || g->off[3 * k + i] > 1) small2d = false;
    if (g->fam.kind == FAM_GENERIC && small2d && dtype == ST_F64 && time_levels == 1 && !g->has_beta &&
        !g->caller_ghosts && bc != ST_NEUMANN && !(flags & ST_FLAG_GENERIC)) {
        g->plan_optional = true;
        g->plan_use = (flags & ST_FLAG_TILE_PASSES) != 0;
        // "TX,TY,K": run k_tb2d with that configuration (tests, tuning sweeps)
        const char* env = std::getenv("ST_TB2D_CFG");
        int tx = 0, ty = 0, tk = 0;
        if (!g->plan_use && env && std::sscanf(env, "%d,%d,%d", &tx, &ty, &tk) == 3 &&
            tb2d_fits(g->g.nx, g->g.ny, tx, ty, tk) && tb2d_supports(g->fam)) {
            g->tb[0] = tx;
            g->tb[1] = ty;
            g->tb[2] = tk;
        }
    }
    if (g->fam.kind == FAM_2D_TILE || g->plan_optional) {
        std::vector<int32_t> off2(2 * npts);
        for (int k = 0; k < npts; ++k) {
            off2[2 * k] = g->off[3 * k + 1];
            off2[2 * k + 1] = g->off[3 * k + 2];
        }
        g->plan = new (std::nothrow) BatchPlan(make_batch_plan(std::vector<Geom>{g->g}, npts, off2.data(),
                                                               g->alpha.data(), bc == ST_PERIODIC, dtype, false));
        if (!g->plan) {
            delete g;
            return fail(ST_ERR_OOM, "stencil_create: out of host memory");
        }
        g->plan->bc = bc_value;
        // one grid: small tiles so that every SM gets work; FP64 is bound by
        // the FP64 pipe, so no redundant halo work by default (k = 1)
        g->plan->cfg[0] = 32;
        g->plan->cfg[1] = 8;
        g->plan->cfg[2] = 128;
        g->plan->cfg[3] = dtype == ST_F64 ? 1 : 4;
    }
    *out = g;
    return ST_OK;
}

st_status stencil_create_conservative(st_grid_t* out, int ndim, const int64_t* dims, st_bc bc, double bc_value,
                                      st_dtype dtype, uint32_t flags)
{
    if (!out) return fail(ST_ERR_ARG, "stencil_create_conservative: out is NULL");
    *out = nullptr;
    if (ndim != 2 && ndim != 3) return fail(ST_ERR_ARG, "stencil_create_conservative: ndim must be 2 or 3");
    if (bc != ST_DIRICHLET && bc != ST_PERIODIC)
        return fail(ST_ERR_ARG, "stencil_create_conservative: Dirichlet or periodic boundary");
    if (flags != 0) return fail(ST_ERR_ARG, "stencil_create_conservative: no flags are defined");
    // centre, then -z, +z, -y, +y, -x, +x (2D: -y, +y, -x, +x); the weights
    // of the non-conservative form w = 1 - 2 ndim kappa, kappa only mark the
    // operator as per-cell (the conservative kernel builds its own)
    int32_t off[7 * 3] = {};
    double alpha[7] = {}, beta[7] = {};
    int n = 1;
    alpha[0] = 1.0;
    beta[0] = -2.0 * ndim;
    for (int ax = 0; ax < ndim; ++ax)
        for (int sgn = -1; sgn <= 1; sgn += 2) {
            off[n * ndim + ax] = sgn;
            beta[n] = 1.0;
            ++n;
        }
    st_status rc = stencil_create(out, ndim, dims, 1, n, off, alpha, beta, bc, bc_value, dtype, 1, ST_FLAG_GENERIC);
    if (rc != ST_OK) return rc;
    st_grid_t g = *out;
    g->fam.kind = FAM_CONS;
    g->fam.name = "cons_face_avg_point";
    // 3D grids sweep on the staged pipeline (variant 1), 2D grids and the
    // transposed step on the one-thread-per-column kernels
    if (star3d_cons_supported(g->g)) {
        g->fam.variant = 1;
        g->fam.name = "cons_face_avg_bulk";
    }
    return ST_OK;
}

st_status stencil_destroy(st_grid_t g)
{
    if (!g) return ST_OK;
    drop_graphs(g);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->d_status) cudaFree(g->d_status);
    if (g->d_partials) cudaFree(g->d_partials);
    if (g->d_src) cudaFree(g->d_src);
    if (g->plan) {
        free_batch_plan(*g->plan);
        delete g->plan;
    }
    if (g->staging) cudaFree(g->staging);
    if (g->staging2) cudaFree(g->staging2);
    if (g->pad_in) cudaFree(g->pad_in);
    if (g->pad_out) cudaFree(g->pad_out);
    if (g->cpack) cudaEventDestroy(g->cpack);
    if (g->cunpack) cudaEventDestroy(g->cunpack);
    for (int c = 0; c < 4; ++c) {
        if (g->cstream[c]) cudaStreamDestroy(g->cstream[c]);
        if (g->cjoin[c]) cudaEventDestroy(g->cjoin[c]);
    }
    if (g->cfork) cudaEventDestroy(g->cfork);
    delete g;
    return ST_OK;
}

st_status stencil_layout(st_grid_t g, int64_t* padded_dims, int64_t* origin, int64_t* elems)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_layout: NULL handle");
    const Geom& G = g->g;
    if (padded_dims) {
        if (G.ndim == 3) {
            padded_dims[0] = G.pnz;
            padded_dims[1] = G.pny;
            padded_dims[2] = G.pitch;
        } else {
            padded_dims[0] = G.pny;
            padded_dims[1] = G.pitch;
        }
    }
    if (origin) {
        if (G.ndim == 3) {
            origin[0] = G.rz;
            origin[1] = G.r;
            origin[2] = G.xl;
        } else {
            origin[0] = G.r;
            origin[1] = G.xl;
        }
    }
    if (elems) *elems = G.elems;
    return ST_OK;
}

st_status stencil_info(st_grid_t g, int* radius, int* npts, const char** kernel_name)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_info: NULL handle");
    if (radius) *radius = g->radius;
    if (npts) *npts = g->npts;
    if (kernel_name)
        *kernel_name = (g->plan_optional && g->plan_use) ? "tile2d_passes"
                       : (g->plan_optional && g->tb[2] > 0) ? "tb2d_passes"
                                                              : g->fam.name;
    return ST_OK;
}

st_status stencil_bind(st_grid_t g, int slot, void* ptr)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_bind: NULL handle");
    if (slot < 0 || slot > 2) return fail(ST_ERR_ARG, "stencil_bind: slot must be 0, 1 or 2");
    if (!ptr) return fail(ST_ERR_ARG, "stencil_bind: NULL pointer");
    if (((uintptr_t)ptr & 15u) != 0) return fail(ST_ERR_ARG, "stencil_bind: pointer not 16-byte aligned");
    const size_t bytes = (size_t)g->g.elems * g->g.esize;
    const uintptr_t lo = (uintptr_t)ptr, hi = lo + bytes;
    for (int s = 0; s < 3; ++s) {
        if (s == slot || !g->buf[s]) continue;
        const uintptr_t l2 = (uintptr_t)g->buf[s], h2 = l2 + bytes;
        if (lo < h2 && l2 < hi) return fail(ST_ERR_ALIAS, "stencil_bind: buffer overlaps another bound slot");
    }
    st_status rc = ensure_scratch(g);
    if (rc != ST_OK) return rc;
    cudaPointerAttributes at{};
    ST_CUDA_TRY(cudaPointerGetAttributes(&at, ptr));
    if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
        return fail(ST_ERR_ARG, "stencil_bind: not a device pointer");
    g->buf[slot] = ptr;
    g->stale[slot] = true;
    if (slot == ST_SLOT_A) g->cur = ST_SLOT_A;
    drop_graphs(g);
    if (g->plan && g->buf[ST_SLOT_A] && g->buf[ST_SLOT_B]) {
        void* a = g->buf[ST_SLOT_A];
        void* b = g->buf[ST_SLOT_B];
        rc = bind_batch_plan(*g->plan, std::vector<Geom>{g->g}, &a, &b, g->d_status);
        if (rc != ST_OK) return rc;
        bool moved = false;
        rc = reserve_batch_steps(*g->plan, 1024, &moved);
        if (rc != ST_OK) return rc;
        // the optional FP64 plan runs one launch per pass (a grid-wide barrier
        // per pass costs more than a dependent launch)
        if (g->plan_optional) batch_disable_coop(*g->plan);
        g->plan_bound = true;
    }
    return ST_OK;
}

st_status stencil_mark_dirty(st_grid_t g, int slot)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_mark_dirty: NULL handle");
    if (slot < 0 || slot > 2) return fail(ST_ERR_ARG, "stencil_mark_dirty: bad slot");
    g->stale[slot] = true;
    return ST_OK;
}

st_status stencil_current(st_grid_t g, int* slot)
{
    if (!g || !slot) return fail(ST_ERR_ARG, "stencil_current: NULL argument");
    *slot = g->cur;
    return ST_OK;
}

st_status stencil_set_current(st_grid_t g, int slot)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_set_current: NULL handle");
    if (slot != ST_SLOT_A && slot != ST_SLOT_B) return fail(ST_ERR_ARG, "stencil_set_current: slot must be 0 or 1");
    g->cur = slot;
    return ST_OK;
}

st_status stencil_set_source(st_grid_t g, const int64_t* index, const double* amplitudes, int64_t count)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_set_source: NULL handle");
    if (count < 0) return fail(ST_ERR_ARG, "stencil_set_source: negative count");
    if (g->d_src) {
        cudaFree(g->d_src);
        g->d_src = nullptr;
    }
    g->src = -1;
    g->src_count = 0;
    drop_graphs(g);
    if (count == 0) return ST_OK;
    if (!index || !amplitudes) return fail(ST_ERR_ARG, "stencil_set_source: NULL index/amplitudes");
    if (g->levels != 2) return fail(ST_ERR_UNSUPPORTED, "stencil_set_source: source needs the leapfrog form");
    const Geom& G = g->g;
    int64_t c[3] = {0, 0, 0};
    for (int i = 0; i < G.ndim; ++i) c[3 - G.ndim + i] = index[i];
    if (c[0] < 0 || c[0] >= G.nz || c[1] < 0 || c[1] >= G.ny || c[2] < 0 || c[2] >= G.nx)
        return fail(ST_ERR_ARG, "stencil_set_source: index outside the interior");
    if (cudaMalloc(&g->d_src, sizeof(double) * count) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ST_ERR_OOM, "stencil_set_source: allocation failed");
    }
    ST_CUDA_TRY(cudaMemcpy(g->d_src, amplitudes, sizeof(double) * count, cudaMemcpyHostToDevice));
    g->src = G.origin + c[0] * G.plane + c[1] * G.pitch + c[2];
    g->src_count = count;
    return ST_OK;
}

st_status stencil_set_step_index(st_grid_t g, int64_t t)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_set_step_index: NULL handle");
    if (t < 0) return fail(ST_ERR_ARG, "stencil_set_step_index: negative");
    g->step = t;
    return ST_OK;
}

st_status stencil_get_step_index(st_grid_t g, int64_t* t)
{
    if (!g || !t) return fail(ST_ERR_ARG, "stencil_get_step_index: NULL argument");
    *t = g->step;
    return ST_OK;
}

st_status stencil_snapshot_bytes(st_grid_t g, size_t* bytes)
{
    if (!g || !bytes) return fail(ST_ERR_ARG, "stencil_snapshot_bytes: NULL argument");
    *bytes = (size_t)g->levels * (size_t)g->g.elems * g->g.esize;
    return ST_OK;
}

// A snapshot is the newest level's whole padded buffer, then (two time
// levels) the previous level's: device-to-device copies on the caller's
// stream, so the state never leaves HBM.
st_status stencil_snapshot(st_grid_t g, void* dst, int64_t* step_out, void* stream)
{
    if (!g || !dst || !step_out) return fail(ST_ERR_ARG, "stencil_snapshot: NULL argument");
    if (((uintptr_t)dst & 15u) != 0) return fail(ST_ERR_ARG, "stencil_snapshot: dst not 16-byte aligned");
    if (!g->buf[ST_SLOT_A] || !g->buf[ST_SLOT_B])
        return fail(ST_ERR_STATE, "stencil_snapshot: both time-level slots must be bound");
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    const size_t bytes = (size_t)g->g.elems * g->g.esize;
    ST_CUDA_TRY(cudaMemcpyAsync(dst, g->buf[g->cur], bytes, cudaMemcpyDeviceToDevice, s));
    if (g->levels == 2)
        ST_CUDA_TRY(cudaMemcpyAsync((char*)dst + bytes, g->buf[1 - g->cur], bytes, cudaMemcpyDeviceToDevice, s));
    *step_out = g->step;
    return ST_OK;
}

st_status stencil_restore(st_grid_t g, const void* src, int64_t step, void* stream)
{
    if (!g || !src) return fail(ST_ERR_ARG, "stencil_restore: NULL argument");
    if (((uintptr_t)src & 15u) != 0) return fail(ST_ERR_ARG, "stencil_restore: src not 16-byte aligned");
    if (step < 0) return fail(ST_ERR_ARG, "stencil_restore: negative step index");
    if (!g->buf[ST_SLOT_A] || !g->buf[ST_SLOT_B])
        return fail(ST_ERR_STATE, "stencil_restore: both time-level slots must be bound");
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    const size_t bytes = (size_t)g->g.elems * g->g.esize;
    ST_CUDA_TRY(cudaMemcpyAsync(g->buf[ST_SLOT_A], src, bytes, cudaMemcpyDeviceToDevice, s));
    if (g->levels == 2)
        ST_CUDA_TRY(cudaMemcpyAsync(g->buf[ST_SLOT_B], (const char*)src + bytes, bytes, cudaMemcpyDeviceToDevice,
                                    s));
    g->cur = ST_SLOT_A;
    g->step = step;
    // the library's ghost values are rewritten before the next step (a
    // snapshot taken from a handle of another boundary value stays valid)
    g->stale[ST_SLOT_A] = g->stale[ST_SLOT_B] = true;
    return ST_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Step machinery
// ---------------------------------------------------------------------------
static SweepArgs sweep_args(st_grid_t g, const void* in, void* out, int64_t step)
{
    SweepArgs a{};
    a.in = in;
    a.out = out;
    a.prev = (g->levels == 2) ? out : nullptr;
    a.kappa = g->has_beta ? g->buf[ST_SLOT_COEFF] : nullptr;
    a.step = step;
    a.src = g->src;
    a.src_amp = g->d_src;
    a.src_count = g->src_count;
    a.status = g->d_status;
    return a;
}

// Ghost cells of the coefficient field: 0, except for the conservative
// operator, whose staged kernel reads a Dirichlet ghost face's coefficient
// as (kappa_p + kappa_ghost) / 2 and so needs each ghost to mirror its
// interior neighbour (then the face takes kappa_p exactly).
static cudaError_t coeff_ghosts(st_grid_t g, cudaStream_t s)
{
    if (g->fam.kind == FAM_CONS) return launch_mirror_ghosts(g->g.esize, g->buf[ST_SLOT_COEFF], g->g, s);
    return launch_fill_ghosts(g->g.esize, g->buf[ST_SLOT_COEFF], g->g, 0.0, s);
}

static st_status refresh_ghosts(st_grid_t g, cudaStream_t s)
{
    for (int slot = 0; slot < 3; ++slot) {
        if (!g->stale[slot] || !g->buf[slot]) continue;
        if (slot == ST_SLOT_COEFF) {
            ST_CUDA_TRY(coeff_ghosts(g, s));
        } else if (g->bc == ST_DIRICHLET && !g->caller_ghosts) {
            ST_CUDA_TRY(launch_fill_ghosts(g->g.esize, g->buf[slot], g->g, g->bc_value, s));
        }
        g->stale[slot] = false;
    }
    return ST_OK;
}

static st_status check_ready(st_grid_t g, const char* who)
{
    if (!g->buf[ST_SLOT_A] || !g->buf[ST_SLOT_B])
        return fail(ST_ERR_STATE, std::string(who) + ": both time-level slots must be bound");
    if (g->has_beta && !g->buf[ST_SLOT_COEFF])
        return fail(ST_ERR_STATE, std::string(who) + ": per-cell weights need ST_SLOT_COEFF bound");
    return ST_OK;
}

// Two-step passes (temporal blocking) where the family has them; a source
// term needs its step index per sweep, so it keeps single sweeps.
static bool use_pairs(st_grid_t g)
{
    return g->pairs && !g->caller_ghosts && g->bc != ST_NEUMANN && g->src < 0 && star3d_pair_supported(g->fam);
}

// k steps per launch on k_tb2d (small FP64 2D grids, chosen by stencil_tune)
static bool use_tb(st_grid_t g) { return g->plan_optional && !g->plan_use && g->tb[2] > 0 && g->src < 0; }

// Slot of the newest level after n steps from slot `cur`: every launch (one
// sweep or one two-step pass) writes the other slot.
static int final_slot(st_grid_t g, int cur, int n)
{
    const int launches = use_tb(g) ? (n + g->tb[2] - 1) / g->tb[2] : use_pairs(g) ? n / 2 + (n & 1) : n;
    return (launches & 1) ? 1 - cur : cur;
}

static st_status enqueue_steps(st_grid_t g, int cur, int64_t step0, int n, cudaStream_t s)
{
    if (use_tb(g)) {
        for (int i = 0; i < n;) {
            const int ks = std::min(g->tb[2], n - i);
            ST_CUDA_TRY(launch_tb2d(g->fam, g->buf[cur], g->buf[1 - cur], g->tb[0], g->tb[1], ks, g->bc_value, s));
            i += ks;
            cur = 1 - cur;
        }
        return ST_OK;
    }
    const bool pairs = use_pairs(g);
    for (int i = 0; i < n;) {
        const int nxt = 1 - cur;
        SweepArgs a = sweep_args(g, g->buf[cur], g->buf[nxt], step0 + i);
        if (pairs && n - i >= 2) {
            ST_CUDA_TRY(launch_star3d_pair(g->fam, a, g->bc_value, s));
            i += 2;
        } else {
            // zero-flux boundary: the input's ghosts mirror its interior
            // before every sweep (the device-local ghost exchange)
            if (g->bc == ST_NEUMANN) ST_CUDA_TRY(launch_mirror_ghosts(g->g.esize, g->buf[cur], g->g, s));
            ST_CUDA_TRY(launch_family(g->fam, a, s));
            i += 1;
        }
        cur = nxt;
    }
    return ST_OK;
}

extern "C" {

st_status stencil_step(st_grid_t g, int nsteps, void* stream)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_step: NULL handle");
    if (nsteps < 0) return fail(ST_ERR_ARG, "stencil_step: negative step count");
    st_status rc = check_ready(g, "stencil_step");
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    rc = refresh_ghosts(g, s);
    if (rc != ST_OK) return rc;
    if (nsteps == 0 || g->g.npoints == 0) return ST_OK;
    if (g->plan && g->plan_bound && g->plan_use && g->src < 0) {
        // 2D grid on the persistent tile kernel: one captured launch for all steps
        bool moved = false;
        rc = reserve_batch_steps(*g->plan, nsteps, &moved);
        if (rc != ST_OK) return rc;
        if (moved) drop_graphs(g);
        auto key = std::make_pair(nsteps, g->cur);
        auto it = g->graphs.find(key);
        for (int attempt = 0; it == g->graphs.end() && attempt < 2; ++attempt) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            ST_CUDA_TRY(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
            st_status erc = enqueue_batch_plan(*g->plan, nsteps, g->cur, g->cap);
            cudaError_t ce = cudaStreamEndCapture(g->cap, &graph);
            if (erc == ST_OK && ce == cudaSuccess) {
                ce = cudaGraphInstantiate(&exec, graph, 0);
                cudaGraphDestroy(graph);
                if (ce == cudaSuccess) {
                    it = g->graphs.emplace(key, exec).first;
                    break;
                }
            } else if (graph) {
                cudaGraphDestroy(graph);
            }
            (void)cudaGetLastError();
            if (attempt == 1) return erc != ST_OK ? erc : cuda_fail(ce, "tile graph capture");
            batch_disable_coop(*g->plan);
        }
        ST_CUDA_TRY(cudaGraphLaunch(it->second, s));
        g->cur = batch_final_slot(*g->plan, nsteps, g->cur);
        g->step += nsteps;
        return ST_OK;
    }
    // Sources change per step (step index is a launch parameter): launch directly.
    const bool use_graph = (g->src < 0) && nsteps >= 2;
    if (!use_graph) {
        rc = enqueue_steps(g, g->cur, g->step, nsteps, s);
        if (rc != ST_OK) return rc;
    } else {
        auto key = std::make_pair(nsteps, g->cur);
        auto it = g->graphs.find(key);
        if (it == g->graphs.end()) {
            cudaGraph_t graph = nullptr;
            cudaGraphExec_t exec = nullptr;
            ST_CUDA_TRY(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
            st_status erc = enqueue_steps(g, g->cur, g->step, nsteps, g->cap);
            cudaError_t ce = cudaStreamEndCapture(g->cap, &graph);
            if (erc != ST_OK) {
                if (graph) cudaGraphDestroy(graph);
                return erc;
            }
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaStreamEndCapture");
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce != cudaSuccess) return cuda_fail(ce, "cudaGraphInstantiate");
            it = g->graphs.emplace(key, exec).first;
        }
        ST_CUDA_TRY(cudaGraphLaunch(it->second, s));
    }
    g->cur = final_slot(g, g->cur, nsteps);
    g->step += nsteps;
    return ST_OK;
}

st_status stencil_tune(st_grid_t g, int nsteps, void* stream)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_tune: NULL handle");
    if (nsteps < 1) return fail(ST_ERR_ARG, "stencil_tune: nsteps >= 1");
    st_status rc = check_ready(g, "stencil_tune");
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    rc = refresh_ghosts(g, s);
    if (rc != ST_OK) return rc;
    if ((!g->plan || !g->plan_bound) && g->levels == 1 && g->src < 0 && !g->caller_ghosts &&
        g->bc != ST_NEUMANN && star3d_pair_supported(g->fam)) {
        // single sweeps or two-step passes: time both on the bound data, keep
        // the faster, and put the current level back
        const size_t bytes = (size_t)g->g.elems * g->g.esize;
        void* keep = nullptr;
        if (cudaMalloc(&keep, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(ST_ERR_OOM, "stencil_tune: backup allocation failed");
        }
        const int cur0 = g->cur;
        const int64_t step0 = g->step;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        float ms[2] = {0.f, 0.f};
        cudaError_t e = cudaEventCreate(&e0);
        if (e == cudaSuccess) e = cudaEventCreate(&e1);
        if (e == cudaSuccess) e = cudaMemcpyAsync(keep, g->buf[cur0], bytes, cudaMemcpyDeviceToDevice, s);
        for (int v = 0; v < 2 && e == cudaSuccess; ++v) {
            g->pairs = v == 1;
            for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {  // the first run warms up
                e = cudaEventRecord(e0, s);
                if (e == cudaSuccess && enqueue_steps(g, cur0, step0, nsteps, s) != ST_OK) e = cudaErrorUnknown;
                if (e == cudaSuccess) e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms[v], e0, e1);
                if (e == cudaSuccess) e = cudaMemcpyAsync(g->buf[cur0], keep, bytes, cudaMemcpyDeviceToDevice, s);
            }
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        g->pairs = e == cudaSuccess && ms[1] < ms[0];
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(keep);
        g->cur = cur0;
        g->step = step0;
        drop_graphs(g);
        if (e != cudaSuccess) return cuda_fail(e, "stencil_tune");
        return ST_OK;
    }
    if (!g->plan || !g->plan_bound) {
        ST_CUDA_TRY(cudaStreamSynchronize(s));
        return ST_OK;  // this family has nothing to tune
    }
    void* a = g->buf[ST_SLOT_A];
    void* b = g->buf[ST_SLOT_B];
    rc = tune_batch_plan(*g->plan, std::vector<Geom>{g->g}, &a, &b, nsteps, g->cur, s);
    drop_graphs(g);
    if (rc != ST_OK || !g->plan_optional) return rc;
    // the one-thread-per-point kernel, the tuned tile plan and k_tb2d over
    // tile shapes and steps per launch, each timed as the captured step
    // sequence stencil_step runs (second of two runs); the fastest is kept,
    // and the current level is put back after every run
    struct Cand {
        bool plan;
        int tb[3];
    };
    std::vector<Cand> cands = {{false, {0, 0, 0}}, {true, {0, 0, 0}}};
    if (tb2d_supports(g->fam)) {
        // fixed shapes, plus for one, two and three tiles per SM the shapes
        // with the least halo work (area of tile + 8-cell halo) that give at
        // most that many tiles: the busiest SM sets a pass's time, and
        // co-resident CTAs overlap one another's loads and stores with
        // arithmetic (256^2, 100 steps: 14 x 16 tiles, two per SM, 3 steps
        // per launch, 1.60 us per step against 2.20 for one launch per step)
        std::vector<std::pair<int, int>> shapes = {{32, 16}, {32, 8}, {16, 16}, {16, 8}, {64, 8}, {16, 32}};
        int nsm = 0, dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess)
            nsm = 0;
        (void)cudaGetLastError();
        const int64_t nx = g->g.nx, ny = g->g.ny;
        for (int per = 1; per <= 3 && nsm > 0; ++per) {
            std::vector<std::pair<int64_t, std::pair<int, int>>> best;
            for (int ty = 4; ty <= 64; ++ty) {
                const int64_t rows = (ny + ty - 1) / ty;
                const int64_t cols_max = (int64_t)per * nsm / rows;
                if (cols_max < 1) continue;
                const int tx = (int)std::max<int64_t>(4, (nx + cols_max - 1) / cols_max);
                if (tx > 128) continue;
                best.push_back({(int64_t)(tx + 8) * (ty + 8), {tx, ty}});
            }
            std::sort(best.begin(), best.end());
            for (size_t i = 0; i < best.size() && i < 3; ++i) shapes.push_back(best[i].second);
        }
        for (const auto& sh : shapes)
            for (int k : {1, 2, 3, 4, 5, 6, 8})
                if (k <= nsteps && tb2d_fits(nx, ny, sh.first, sh.second, k))
                    cands.push_back({false, {sh.first, sh.second, k}});
    }
    const size_t bytes = (size_t)g->g.elems * g->g.esize;
    void* keep = nullptr;
    if (cudaMalloc(&keep, bytes) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ST_ERR_OOM, "stencil_tune: backup allocation failed");
    }
    const int cur0 = g->cur;
    const int64_t step0 = g->step;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    std::vector<float> ms(cands.size(), 0.f);
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) e = cudaMemcpyAsync(keep, g->buf[cur0], bytes, cudaMemcpyDeviceToDevice, s);
    for (size_t v = 0; v < cands.size() && e == cudaSuccess && rc == ST_OK; ++v) {
        g->plan_use = cands[v].plan;
        std::memcpy(g->tb, cands[v].tb, sizeof(g->tb));
        drop_graphs(g);
        for (int rep = 0; rep < 2 && e == cudaSuccess && rc == ST_OK; ++rep) {
            e = cudaEventRecord(e0, s);
            if (e == cudaSuccess) rc = stencil_step(g, nsteps, stream);
            if (e == cudaSuccess && rc == ST_OK) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess && rc == ST_OK) e = cudaEventSynchronize(e1);
            if (e == cudaSuccess && rc == ST_OK) e = cudaEventElapsedTime(&ms[v], e0, e1);
            if (e == cudaSuccess) e = cudaMemcpyAsync(g->buf[cur0], keep, bytes, cudaMemcpyDeviceToDevice, s);
            g->cur = cur0;
            g->step = step0;
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    size_t best = 0;
    if (e == cudaSuccess && rc == ST_OK)
        for (size_t v = 1; v < cands.size(); ++v)
            if (ms[v] < ms[best]) best = v;
    g->plan_use = cands[best].plan;
    std::memcpy(g->tb, cands[best].tb, sizeof(g->tb));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(keep);
    drop_graphs(g);
    if (rc != ST_OK) return rc;
    if (e != cudaSuccess) return cuda_fail(e, "stencil_tune");
    return ST_OK;
}

st_status stencil_tune_config(st_grid_t g, int* cfg)
{
    if (!g || !cfg) return fail(ST_ERR_ARG, "stencil_tune_config: NULL argument");
    if (use_tb(g)) {
        cfg[0] = g->tb[0];
        cfg[1] = g->tb[1];
        cfg[2] = 512;
        cfg[3] = g->tb[2];
        return ST_OK;
    }
    if (!g->plan || !g->plan_use) {
        cfg[0] = cfg[1] = cfg[2] = 0;
        cfg[3] = star3d_pair_supported(g->fam) ? (g->pairs ? 2 : 1) : 0;
        return ST_OK;
    }
    batch_plan_config(*g->plan, cfg);
    return ST_OK;
}

st_status stencil_run_host(st_grid_t g, int nsteps, const void* host_u0, void* host_uT, void* stream)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_run_host: NULL handle");
    if (!host_u0 || !host_uT) return fail(ST_ERR_ARG, "stencil_run_host: NULL host buffer");
    if (g->levels != 1) return fail(ST_ERR_UNSUPPORTED, "stencil_run_host: one time level only");
    st_status rc = check_ready(g, "stencil_run_host");
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    const Geom& G = g->g;
    const size_t bytes = (size_t)G.npoints * G.esize;
    // Pinned host buffers are mapped into the device address space: the
    // (un)pack kernels then read and write them directly over the host link,
    // with many requests in flight.  Other host memory goes through a dense
    // device staging buffer and copy engines.
    auto mapped = [](const void* p) -> void* {
        cudaPointerAttributes a{};
        if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
            (void)cudaGetLastError();
            return nullptr;
        }
        return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
    };
    void* din = mapped(host_u0);
    void* dout = mapped(host_uT);
    if ((!din || !dout) && !g->staging) {
        // one dense interior buffer: a contiguous copy per direction runs at
        // link speed, where a row-strided 3D copy pays per row
        if (cudaMalloc(&g->staging, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(ST_ERR_OOM, "stencil_run_host: staging allocation failed");
        }
    }
    if ((!din || !dout) && !g->cfork) {
        for (int c = 0; c < 4; ++c) {
            ST_CUDA_TRY(cudaStreamCreateWithFlags(&g->cstream[c], cudaStreamNonBlocking));
            ST_CUDA_TRY(cudaEventCreateWithFlags(&g->cjoin[c], cudaEventDisableTiming));
        }
        ST_CUDA_TRY(cudaEventCreateWithFlags(&g->cfork, cudaEventDisableTiming));
    }
    // one host copy as four concurrent pieces, forked from and joined back
    // into the caller's stream
    auto copy4 = [&](void* dst, const void* src, cudaMemcpyKind kind) -> cudaError_t {
        const size_t piece = (bytes / 4 + 255) / 256 * 256;
        cudaError_t e = cudaEventRecord(g->cfork, s);
        for (int c = 0; c < 4 && e == cudaSuccess; ++c) {
            const size_t off = std::min(bytes, (size_t)c * piece), n = std::min(piece, bytes - off);
            e = cudaStreamWaitEvent(g->cstream[c], g->cfork, 0);
            if (e == cudaSuccess && n > 0)
                e = cudaMemcpyAsync((char*)dst + off, (const char*)src + off, n, kind, g->cstream[c]);
            if (e == cudaSuccess) e = cudaEventRecord(g->cjoin[c], g->cstream[c]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, g->cjoin[c], 0);
        }
        return e;
    };
    if (din) {
        ST_CUDA_TRY(launch_pack(G.esize, din, g->buf[g->cur], G, 0, s));
    } else {
        ST_CUDA_TRY(copy4(g->staging, host_u0, cudaMemcpyHostToDevice));
        ST_CUDA_TRY(launch_pack(G.esize, g->staging, g->buf[g->cur], G, 0, s));
    }
    rc = stencil_step(g, nsteps, stream);
    if (rc != ST_OK) return rc;
    if (dout) {
        ST_CUDA_TRY(launch_pack(G.esize, dout, g->buf[g->cur], G, 1, s));
    } else {
        ST_CUDA_TRY(launch_pack(G.esize, g->staging, g->buf[g->cur], G, 1, s));
        ST_CUDA_TRY(copy4(host_uT, g->staging, cudaMemcpyDeviceToHost));
    }
    return ST_OK;
}

st_status stencil_run_host_many(st_grid_t g, int nsteps, int njobs, const void* const* host_in,
                                void* const* host_out, void* stream)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_run_host_many: NULL handle");
    if (nsteps < 0) return fail(ST_ERR_ARG, "stencil_run_host_many: negative step count");
    if (njobs < 0 || (njobs > 0 && (!host_in || !host_out)))
        return fail(ST_ERR_ARG, "stencil_run_host_many: njobs >= 0 and two arrays of njobs host pointers");
    for (int i = 0; i < njobs; ++i)
        if (!host_in[i] || !host_out[i]) return fail(ST_ERR_ARG, "stencil_run_host_many: NULL host buffer");
    if (g->levels != 1) return fail(ST_ERR_UNSUPPORTED, "stencil_run_host_many: one time level only");
    st_status rc = check_ready(g, "stencil_run_host_many");
    if (rc != ST_OK) return rc;
    if (njobs == 0) return ST_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const Geom& G = g->g;
    const size_t bytes = (size_t)G.npoints * G.esize;
    const size_t fbytes = (size_t)G.elems * G.esize;
    // Direct form: a job's input is copied (by rows, at the same rate as a
    // contiguous copy) into the interior of pad_in, which its first sweep
    // reads; every job but the last writes its last sweep to pad_out, whose
    // interior is copied out.  No pack kernel runs, and the grid's own levels
    // hold the last job's states.  Boundaries whose sweeps need the input's
    // ghost cells refreshed from the grid (zero flux, caller-owned ghosts) or
    // a step index (a source) take the dense staging form: pack and unpack
    // kernels around the grid's levels; so do grids on the 2D tile plan,
    // whose kernel sums the offsets in its own order (the single sweeps at
    // both ends of a job would round differently from stencil_step).
    const bool direct = nsteps >= 1 && g->bc != ST_NEUMANN && !g->caller_ghosts && g->src < 0 &&
                        !(g->plan && g->plan_use);
    for (void** b : {&g->staging, &g->staging2, &g->pad_in, &g->pad_out}) {
        const bool need = (b == &g->staging2) || (b == &g->staging ? !direct : direct);
        if (need && !*b) {
            if (cudaMalloc(b, (b == &g->pad_in || b == &g->pad_out) ? fbytes : bytes) != cudaSuccess) {
                (void)cudaGetLastError();
                return fail(ST_ERR_OOM, "stencil_run_host_many: staging allocation failed");
            }
            // the first sweep reads pad_in's Dirichlet ghost cells
            if (b == &g->pad_in && g->bc == ST_DIRICHLET)
                ST_CUDA_TRY(launch_fill_ghosts(G.esize, g->pad_in, G, g->bc_value, s));
        }
    }
    if (!g->cfork) {
        for (int c = 0; c < 4; ++c) {
            ST_CUDA_TRY(cudaStreamCreateWithFlags(&g->cstream[c], cudaStreamNonBlocking));
            ST_CUDA_TRY(cudaEventCreateWithFlags(&g->cjoin[c], cudaEventDisableTiming));
        }
        ST_CUDA_TRY(cudaEventCreateWithFlags(&g->cfork, cudaEventDisableTiming));
    }
    if (!g->cpack) {
        ST_CUDA_TRY(cudaEventCreateWithFlags(&g->cpack, cudaEventDisableTiming));
        ST_CUDA_TRY(cudaEventCreateWithFlags(&g->cunpack, cudaEventDisableTiming));
    }
    // Copy engines carry the host traffic on the handle's copy streams, each
    // direction in two pieces: streams 0-1 bring job i's input in while job
    // i-1 sweeps, streams 2-3 take job i-1's result out while job i sweeps.
    // Hand-offs: an input copy waits until the previous job has read the
    // input buffer (cpack); the kernel that fills the output buffer waits
    // until the previous output copy has read it (cjoin[2..3]).  Both start
    // ordered after the caller's earlier work on `stream`.
    const size_t piece = (bytes / 2 + 255) / 256 * 256;
    auto dense_pieces = [&](int c0, cudaEvent_t after, void* dst, const void* src, cudaMemcpyKind kind) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            const int c = c0 + k;
            const size_t off = std::min(bytes, (size_t)k * piece), n = std::min(piece, bytes - off);
            e = cudaStreamWaitEvent(g->cstream[c], after, 0);
            if (e == cudaSuccess && n > 0)
                e = cudaMemcpyAsync((char*)dst + off, (const char*)src + off, n, kind, g->cstream[c]);
            if (e == cudaSuccess) e = cudaEventRecord(g->cjoin[c], g->cstream[c]);
        }
        return e;
    };
    // dense host field <-> interior of a field-layout buffer, planes split in two
    auto pad_pieces = [&](int c0, cudaEvent_t after, void* pad, void* host, bool to_device) -> cudaError_t {
        cudaError_t e = cudaSuccess;
        char* interior = (char*)pad + (size_t)G.origin * G.esize;
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
            const int c = c0 + k;
            const size_t z0 = (size_t)G.nz * k / 2, z1 = (size_t)G.nz * (k + 1) / 2;
            e = cudaStreamWaitEvent(g->cstream[c], after, 0);
            if (e == cudaSuccess && z1 > z0) {
                cudaMemcpy3DParms q = {};
                const cudaPitchedPtr hp = make_cudaPitchedPtr(host, (size_t)G.nx * G.esize, (size_t)G.nx * G.esize,
                                                              (size_t)G.ny);
                const cudaPitchedPtr dp = make_cudaPitchedPtr(interior, (size_t)G.pitch * G.esize,
                                                              (size_t)G.nx * G.esize, (size_t)G.pny);
                q.srcPtr = to_device ? hp : dp;
                q.dstPtr = to_device ? dp : hp;
                q.srcPos = make_cudaPos(0, 0, z0);
                q.dstPos = make_cudaPos(0, 0, z0);
                q.extent = make_cudaExtent((size_t)G.nx * G.esize, (size_t)G.ny, z1 - z0);
                q.kind = to_device ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost;
                e = cudaMemcpy3DAsync(&q, g->cstream[c]);
            }
            if (e == cudaSuccess) e = cudaEventRecord(g->cjoin[c], g->cstream[c]);
        }
        return e;
    };
    auto sweep = [&](const void* in, void* out) -> st_status {
        ST_CUDA_TRY(launch_family(g->fam, sweep_args(g, in, out, g->step), s));
        g->step += 1;
        return ST_OK;
    };
    ST_CUDA_TRY(cudaEventRecord(g->cpack, s));
    ST_CUDA_TRY(cudaEventRecord(g->cjoin[2], s));
    ST_CUDA_TRY(cudaEventRecord(g->cjoin[3], s));
    for (int i = 0; i < njobs; ++i) {
        const bool last = i == njobs - 1;
        if (direct)
            ST_CUDA_TRY(pad_pieces(0, g->cpack, g->pad_in, const_cast<void*>(host_in[i]), true));
        else
            ST_CUDA_TRY(dense_pieces(0, g->cpack, g->staging, host_in[i], cudaMemcpyHostToDevice));
        ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[0], 0));
        ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[1], 0));
        bool out_padded = false;
        if (!direct) {
            ST_CUDA_TRY(launch_pack(G.esize, g->staging, g->buf[g->cur], G, 0, s));
            ST_CUDA_TRY(cudaEventRecord(g->cpack, s));
            rc = stencil_step(g, nsteps, stream);
            if (rc != ST_OK) return rc;
        } else if (nsteps == 1 && !last) {
            ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[2], 0));
            ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[3], 0));
            rc = sweep(g->pad_in, g->pad_out);
            if (rc != ST_OK) return rc;
            ST_CUDA_TRY(cudaEventRecord(g->cpack, s));
            out_padded = true;
        } else {
            // the first sweep reads pad_in and writes the current level
            rc = refresh_ghosts(g, s);
            if (rc != ST_OK) return rc;
            rc = sweep(g->pad_in, g->buf[g->cur]);
            if (rc != ST_OK) return rc;
            ST_CUDA_TRY(cudaEventRecord(g->cpack, s));
            if (nsteps >= 3) {
                rc = stencil_step(g, nsteps - 2, stream);
                if (rc != ST_OK) return rc;
            }
            if (nsteps >= 2) {
                if (!last) {
                    ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[2], 0));
                    ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[3], 0));
                    rc = sweep(g->buf[g->cur], g->pad_out);
                    out_padded = true;
                } else {
                    rc = sweep(g->buf[g->cur], g->buf[1 - g->cur]);
                    g->cur = 1 - g->cur;
                }
                if (rc != ST_OK) return rc;
            }
        }
        if (out_padded) {
            ST_CUDA_TRY(cudaEventRecord(g->cunpack, s));
            ST_CUDA_TRY(pad_pieces(2, g->cunpack, g->pad_out, host_out[i], false));
        } else {
            ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[2], 0));
            ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[3], 0));
            ST_CUDA_TRY(launch_pack(G.esize, g->staging2, g->buf[g->cur], G, 1, s));
            ST_CUDA_TRY(cudaEventRecord(g->cunpack, s));
            ST_CUDA_TRY(dense_pieces(2, g->cunpack, host_out[i], g->staging2, cudaMemcpyDeviceToHost));
        }
    }
    // the last results are on the host once `stream` passes this point
    ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[2], 0));
    ST_CUDA_TRY(cudaStreamWaitEvent(s, g->cjoin[3], 0));
    g->last = s;
    return ST_OK;
}

st_status stencil_sync(st_grid_t g)
{
    if (!g) return fail(ST_ERR_ARG, "stencil_sync: NULL handle");
    ST_CUDA_TRY(cudaStreamSynchronize(g->last));
    if (!g->scratch) return ST_OK;
    int code = 0;
    ST_CUDA_TRY(cudaMemcpy(&code, g->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (code != 0) {
        ST_CUDA_TRY(cudaMemset(g->d_status, 0, sizeof(int)));
        if (code == ST_ERR_DEVICE_TIMEOUT) return fail(ST_ERR_DEVICE_TIMEOUT, "device: bounded wait ran out");
        return fail(ST_ERR_BOUNDS, "device: bounds check fired");
    }
    return ST_OK;
}

st_status stencil_reduce(st_grid_t g, const void* a, const void* b, double* dev_out, void* stream)
{
    if (!g || !a || !dev_out) return fail(ST_ERR_ARG, "stencil_reduce: NULL argument");
    if ((((uintptr_t)a) | ((uintptr_t)b)) & 15u) return fail(ST_ERR_ARG, "stencil_reduce: a, b must be 16-byte aligned");
    st_status rc = ensure_scratch(g);
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    ST_CUDA_TRY(launch_reduce(g->g.esize, a, b, g->g, g->d_partials, g->red_blocks, dev_out, 0, nullptr, g->d_status, s));
    return ST_OK;
}

st_status stencil_step_reduce(st_grid_t g, int nsteps, double* dev_out, void* stream)
{
    if (!g || !dev_out) return fail(ST_ERR_ARG, "stencil_step_reduce: NULL argument");
    if (nsteps < 0) return fail(ST_ERR_ARG, "stencil_step_reduce: negative step count");
    st_status rc = check_ready(g, "stencil_step_reduce");
    if (rc != ST_OK) return rc;
    rc = ensure_scratch(g);
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // the last sweep reduces the level it writes where the family has that
    // kernel (FP32 constant symmetric 3D star, no ghost refresh from outside
    // the sweep, no source); otherwise the sweeps, then stencil_reduce
    const bool fused = nsteps >= 1 && star3d_reduce_supported(g->fam) && g->levels == 1 && g->src < 0 &&
                       !g->caller_ghosts && g->bc != ST_NEUMANN && g->g.npoints > 0;
    if (!fused) {
        rc = stencil_step(g, nsteps, stream);
        if (rc != ST_OK) return rc;
        return stencil_reduce(g, g->buf[g->cur], nullptr, dev_out, stream);
    }
    rc = stencil_step(g, nsteps - 1, stream);  // also refreshes stale ghosts
    if (rc != ST_OK) return rc;
    g->last = s;
    SweepArgs a = sweep_args(g, g->buf[g->cur], g->buf[1 - g->cur], g->step);
    ST_CUDA_TRY(launch_star3d_reduce(g->fam, a, g->d_partials, g->red_blocks, dev_out, s));
    g->cur = 1 - g->cur;
    g->step += 1;
    return ST_OK;
}

st_status stencil_residual(st_grid_t g, const void* u, const void* target, void* lambda, double* dev_loss,
                           void* stream)
{
    if (!g || !u || !target || !lambda || !dev_loss) return fail(ST_ERR_ARG, "stencil_residual: NULL argument");
    if (lambda == u || lambda == target) return fail(ST_ERR_ALIAS, "stencil_residual: lambda aliases an input");
    if ((((uintptr_t)u) | ((uintptr_t)target) | ((uintptr_t)lambda)) & 15u)
        return fail(ST_ERR_ARG, "stencil_residual: u, target, lambda must be 16-byte aligned");
    st_status rc = ensure_scratch(g);
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    ST_CUDA_TRY(launch_fill_ghosts(g->g.esize, lambda, g->g, 0.0, s));
    ST_CUDA_TRY(launch_reduce(g->g.esize, u, target, g->g, g->d_partials, g->red_blocks, dev_loss, 1, lambda, g->d_status, s));
    return ST_OK;
}

static size_t state_bytes(st_grid_t g) { return (size_t)((g->g.elems * g->g.esize + 255) / 256 * 256); }

// Adjoint workspace, in levels: nck checkpoints, then (when there is more
// than one segment) the m-1 levels a segment is recomputed into, then the
// m-1 inner levels of the last segment kept by the forward run.
static int64_t ws_recompute_levels(int64_t nck, int m) { return nck > 1 ? m - 1 : 0; }
static size_t ws_last_offset(int64_t nck, int m, size_t sb) { return (size_t)(nck + ws_recompute_levels(nck, m)) * sb; }
// The conservative operator on the staged 3D pipeline runs its transposed
// steps as the forward sweep on lambda (the matrix is symmetric) and its
// coefficient gradient in a separate pass per segment, which reads the
// segment's lambda levels: m - 1 more levels after the last segment's.
static bool cons_split(st_grid_t g) { return g->fam.kind == FAM_CONS && g->fam.variant == 1; }
static size_t ws_lambda_offset(int64_t nck, int m, size_t sb) { return ws_last_offset(nck, m, sb) + (size_t)(m - 1) * sb; }
// FP32 grids on the fused transpose keep the checkpoint segment's gradient in
// an FP32 partial field (one more level, after the others), added to the
// FP64 gradient once per segment.
static bool grad_partial(st_grid_t g) { return g->g.esize == 4 && g->has_beta && star3d_adjoint_fuse(g->fam) > 0; }


st_status stencil_adjoint_workspace(st_grid_t g, int nsteps, int m, size_t* bytes)
{
    if (!g || !bytes) return fail(ST_ERR_ARG, "stencil_adjoint_workspace: NULL argument");
    if (nsteps < 0 || m < 1) return fail(ST_ERR_ARG, "stencil_adjoint_workspace: nsteps >= 0, ckpt_every >= 1");
    const int64_t nck = (nsteps + m - 1) / m;
    // checkpoints, the recomputation buffer of a segment, and the states of
    // the last segment kept from the forward run
    *bytes = state_bytes(g) * (size_t)(nck + ws_recompute_levels(nck, m) + (m - 1) + (cons_split(g) ? m - 1 : 0) +
                                        (grad_partial(g) ? 1 : 0));
    return ST_OK;
}

st_status stencil_step_ckpt(st_grid_t g, int nsteps, int m, void* ws, void* stream)
{
    if (!g || !ws) return fail(ST_ERR_ARG, "stencil_step_ckpt: NULL argument");
    if (nsteps < 0 || m < 1) return fail(ST_ERR_ARG, "stencil_step_ckpt: nsteps >= 0, ckpt_every >= 1");
    if (g->levels != 1) return fail(ST_ERR_UNSUPPORTED, "stencil_step_ckpt: one time level only");
    if (g->caller_ghosts) return fail(ST_ERR_UNSUPPORTED, "stencil_step_ckpt: not with ST_FLAG_CALLER_GHOSTS");
    if (((uintptr_t)ws & 15u) != 0) return fail(ST_ERR_ARG, "stencil_step_ckpt: workspace not 16-byte aligned");
    st_status rc = check_ready(g, "stencil_step_ckpt");
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    rc = refresh_ghosts(g, s);
    if (rc != ST_OK) return rc;
    const size_t sb = state_bytes(g);
    const size_t bytes = (size_t)g->g.elems * g->g.esize;
    const int64_t nck = (nsteps + m - 1) / m;
    char* last = (char*)ws + ws_last_offset(nck, m, sb);  // states t0 + 1 .. t0 + L - 1 of the last segment
    char* rec = (char*)ws + (size_t)nck * sb;               // the recomputation levels
    g->kept2_ws = nullptr;
    for (int t = 0; t < nsteps; t += m) {
        ST_CUDA_TRY(cudaMemcpyAsync((char*)ws + (size_t)(t / m) * sb, g->buf[g->cur], bytes,
                                    cudaMemcpyDeviceToDevice, s));
        const int seg = std::min(m, nsteps - t);
        const int64_t c = t / m;
        if (c < nck - 2) {
            rc = enqueue_steps(g, g->cur, g->step, seg, s);
            if (rc != ST_OK) return rc;
        } else {
            // the last two segments: their inner states go to the workspace
            // (the last segment's to its own levels, the one before to the
            // recomputation levels, which the reverse pass does not need
            // until it reaches that segment), where the reverse pass reads
            // them instead of recomputing them; the final state lands in the
            // slot a plain run would leave it in
            char* keep = c == nck - 1 ? last : rec;
            const int fin = final_slot(g, g->cur, seg);
            const void* in = g->buf[g->cur];
            for (int j = 1; j <= seg; ++j) {
                void* out = j < seg ? (void*)(keep + (size_t)(j - 1) * sb) : g->buf[fin];
                if (j < seg && g->bc == ST_DIRICHLET)
                    ST_CUDA_TRY(launch_fill_ghosts(g->g.esize, out, g->g, g->bc_value, s));
                // zero flux: the input's ghosts mirror its interior before every sweep
                if (g->bc == ST_NEUMANN) ST_CUDA_TRY(launch_mirror_ghosts(g->g.esize, const_cast<void*>(in), g->g, s));
                SweepArgs a = sweep_args(g, in, out, g->step + j - 1);
                ST_CUDA_TRY(launch_family(g->fam, a, s));
                in = out;
            }
        }
        g->cur = final_slot(g, g->cur, seg);
        g->step += seg;
    }
    if (nck >= 2) {
        g->kept2_ws = ws;
        g->kept2_n = nsteps;
        g->kept2_m = m;
    }
    return ST_OK;
}

st_status stencil_adjoint(st_grid_t g, int nsteps, int m, const void* ws, void* lambda, void* lambda_tmp,
                          double* grad, void* stream)
{
    if (!g || !ws || !lambda || !lambda_tmp) return fail(ST_ERR_ARG, "stencil_adjoint: NULL argument");
    if (nsteps < 0 || m < 1) return fail(ST_ERR_ARG, "stencil_adjoint: nsteps >= 0, ckpt_every >= 1");
    if (g->levels != 1) return fail(ST_ERR_UNSUPPORTED, "stencil_adjoint: one time level only");
    if (g->caller_ghosts) return fail(ST_ERR_UNSUPPORTED, "stencil_adjoint: not with ST_FLAG_CALLER_GHOSTS");
    if (lambda == lambda_tmp) return fail(ST_ERR_ALIAS, "stencil_adjoint: lambda and lambda_tmp alias");
    if ((((uintptr_t)ws) | ((uintptr_t)lambda) | ((uintptr_t)lambda_tmp) | ((uintptr_t)grad)) & 15u)
        return fail(ST_ERR_ARG, "stencil_adjoint: buffers must be 16-byte aligned");
    if (grad && !g->has_beta) return fail(ST_ERR_ARG, "stencil_adjoint: grad_coeff needs per-cell weights");
    if (g->has_beta && !g->buf[ST_SLOT_COEFF]) return fail(ST_ERR_STATE, "stencil_adjoint: ST_SLOT_COEFF not bound");
    st_status rc = ensure_scratch(g);
    if (rc != ST_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    g->last = s;
    if (g->stale[ST_SLOT_COEFF] && g->buf[ST_SLOT_COEFF]) {
        ST_CUDA_TRY(coeff_ghosts(g, s));
        g->stale[ST_SLOT_COEFF] = false;
    }
    ST_CUDA_TRY(launch_fill_ghosts(g->g.esize, lambda, g->g, 0.0, s));
    ST_CUDA_TRY(launch_fill_ghosts(g->g.esize, lambda_tmp, g->g, 0.0, s));
    if (nsteps == 0) return ST_OK;
    const size_t sb = state_bytes(g);
    const int64_t nck = (nsteps + m - 1) / m;
    char* base = (char*)const_cast<void*>(ws);
    char* seg = base + (size_t)nck * sb;
    auto state = [&](int64_t c, int j) -> void* {
        return j == 0 ? (void*)(base + (size_t)c * sb) : (void*)(seg + (size_t)(j - 1) * sb);
    };
    // the second-to-last segment's states are in the recomputation levels if
    // the forward run that filled this workspace left them there and no
    // reverse pass has recomputed another segment into them since
    const bool kept2 = nck >= 2 && g->kept2_ws == ws && g->kept2_n == nsteps && g->kept2_m == m;
    if (nck >= 3) g->kept2_ws = nullptr;
    // the recomputation levels' Dirichlet ghosts (that forward run set them
    // when it stored the kept states there)
    if (g->bc == ST_DIRICHLET && !kept2)
        for (int j = 1; j <= ws_recompute_levels(nck, m); ++j)
            ST_CUDA_TRY(launch_fill_ghosts(g->g.esize, state(0, j), g->g, g->bc_value, s));
    const int fuse = star3d_adjoint_fuse(g->fam);  // steps per optimised transpose launch (0: generic)
    const bool split = cons_split(g) && g->bc != ST_NEUMANN;
    // the FP32 partial gradient of a segment (after every other level): the
    // first pass of a segment stores its terms, the others add theirs, and
    // the sum goes into grad after the segment; cleared once here so that
    // its ghost and padding cells add 0
    void* gpart = nullptr;
    if (grad && grad_partial(g) && g->bc != ST_NEUMANN) {
        gpart = base + ws_lambda_offset(nck, m, sb) + (cons_split(g) ? (size_t)(m - 1) * sb : 0);
        ST_CUDA_TRY(cudaMemsetAsync(gpart, 0, (size_t)g->g.elems * g->g.esize, s));
    }
    char* lamws = base + ws_lambda_offset(nck, m, sb);  // lambda levels of a segment (split form)
    if (split && g->bc == ST_DIRICHLET)
        for (int j = 1; j < m; ++j) ST_CUDA_TRY(launch_fill_ghosts(g->g.esize, lamws + (size_t)(j - 1) * sb, g->g, 0.0, s));
    void* lin = lambda;
    void* lout = lambda_tmp;
    char* last = base + ws_last_offset(nck, m, sb);  // the last segment's states, kept by the forward run
    for (int64_t c = nck - 1; c >= 0; --c) {
        const int64_t t0 = c * m;
        const int L = (int)std::min<int64_t>(m, nsteps - t0);
        const bool kept = c == nck - 1;
        const bool recompute = !kept && !(kept2 && c == nck - 2);
        auto st = [&](int j) -> void* {
            return (kept && j > 0) ? (void*)(last + (size_t)(j - 1) * sb) : state(c, j);
        };
        for (int j = 1; j < L && recompute; ++j) {
            if (g->bc == ST_NEUMANN) ST_CUDA_TRY(launch_mirror_ghosts(g->g.esize, state(c, j - 1), g->g, s));
            SweepArgs a = sweep_args(g, state(c, j - 1), state(c, j), t0 + j - 1);
            ST_CUDA_TRY(launch_family(g->fam, a, s));
        }
        if (split) {
            // lambda_L (lin) down to lambda_0 (lout) by the forward sweep on
            // lambda, the inner levels kept; then the segment's gradient
            auto lv = [&](int jj) -> void* {
                return jj == L ? lin : (jj == 0 ? lout : (void*)(lamws + (size_t)(jj - 1) * sb));
            };
            for (int jj = L - 1; jj >= 0; --jj) ST_CUDA_TRY(launch_family(g->fam, sweep_args(g, lv(jj + 1), lv(jj), 0), s));
            const int gm = cons_grad_max_pairs();
            for (int hi = L - 1; grad && hi >= 0; hi -= gm) {
                const void* us[64];
                const void* ls[64];
                int n = 0;
                for (int jj = hi; jj >= 0 && n < gm; --jj, ++n) {
                    us[n] = st(jj);
                    ls[n] = lv(jj + 1);
                }
                ST_CUDA_TRY(launch_cons_grad(g->fam, us, ls, n, grad, s));
            }
            std::swap(lin, lout);
            continue;
        }
        int j = L - 1;
        while (j >= 0) {
            const int k = (fuse >= 2 && j >= 1) ? 2 : 1;
            AdjointArgs a{};
            a.u = st(j);
            a.u2 = k == 2 ? st(j - 1) : nullptr;
            a.lam_in = lin;
            a.lam_out = lout;
            a.kappa = g->has_beta ? g->buf[ST_SLOT_COEFF] : nullptr;
            a.gk = grad;
            a.gpart = gpart;
            a.gfirst = j == L - 1;
            a.steps = k;
            a.status = g->d_status;
            if (g->bc == ST_NEUMANN)  // the transpose of the mirror-then-sweep step
                ST_CUDA_TRY(launch_neumann_adjoint(g->g.esize, lin, lout, g->fam.gp, g->g.r, g->g.rz, s));
            else
                ST_CUDA_TRY(launch_family_adjoint(g->fam, a, s));
            std::swap(lin, lout);
            j -= k;
        }
        if (gpart) ST_CUDA_TRY(launch_grad_flush(gpart, grad, g->g.elems, s));
    }
    if (lin != lambda)
        ST_CUDA_TRY(cudaMemcpyAsync(lambda, lin, (size_t)g->g.elems * g->g.esize, cudaMemcpyDeviceToDevice, s));
    return ST_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Lid-driven cavity flow (several fields per step)
// ---------------------------------------------------------------------------
struct st_cavity_s {
    CavityParams P{};
    CavityBufs B{};
    void* scratch = nullptr;   // u, v, p second buffers and the pressure source
};

extern "C" {

st_status stencil_cavity_create(st_cavity_t* out, int64_t ny, int64_t nx, double dx, double dy, double dt, double rho,
                                double nu, int nit, double lid, st_dtype dtype)
{
    if (!out) return fail(ST_ERR_ARG, "stencil_cavity_create: out is NULL");
    *out = nullptr;
    if (ny < 3 || nx < 3 || ny > ((int64_t)1 << 19) || nx > ((int64_t)1 << 24))
        return fail(ST_ERR_ARG, "stencil_cavity_create: extents must be in [3, 2^19] (ny) and [3, 2^24] (nx)");
    if (!(dx > 0) || !(dy > 0) || !(dt > 0) || !(rho > 0) || !(nu >= 0))
        return fail(ST_ERR_ARG, "stencil_cavity_create: dx, dy, dt, rho > 0 and nu >= 0");
    if (nit < 0) return fail(ST_ERR_ARG, "stencil_cavity_create: nit >= 0");
    if (dtype != ST_F32 && dtype != ST_F64) return fail(ST_ERR_ARG, "stencil_cavity_create: bad dtype");
    st_cavity_t c = new (std::nothrow) st_cavity_s();
    if (!c) return fail(ST_ERR_OOM, "stencil_cavity_create: out of host memory");
    c->P = CavityParams{};
    c->P.ny = ny;
    c->P.nx = nx;
    c->P.dx = dx;
    c->P.dy = dy;
    c->P.dt = dt;
    c->P.rho = rho;
    c->P.nu = nu;
    c->P.lid = lid;
    c->P.nit = nit;
    c->P.esize = dtype == ST_F64 ? 8 : 4;
    c->P.tb = dtype == ST_F32 ? 1 : 0;  // FP32: pressure iterations in shared-memory passes
    cavity_constants(c->P);
    *out = c;
    return ST_OK;
}

st_status stencil_cavity_destroy(st_cavity_t c)
{
    if (!c) return ST_OK;
    if (c->scratch) cudaFree(c->scratch);
    delete c;
    return ST_OK;
}

st_status stencil_cavity_bind(st_cavity_t c, void* u, void* v, void* p)
{
    if (!c || !u || !v || !p) return fail(ST_ERR_ARG, "stencil_cavity_bind: NULL argument");
    const size_t bytes = (size_t)c->P.ny * (size_t)c->P.nx * (size_t)c->P.esize;
    const uintptr_t a[3] = {(uintptr_t)u, (uintptr_t)v, (uintptr_t)p};
    for (int i = 0; i < 3; ++i) {
        if (a[i] % (uintptr_t)c->P.esize) return fail(ST_ERR_ARG, "stencil_cavity_bind: misaligned buffer");
        for (int k = i + 1; k < 3; ++k)
            if (a[i] < a[k] + bytes && a[k] < a[i] + bytes)
                return fail(ST_ERR_ALIAS, "stencil_cavity_bind: u, v and p overlap");
    }
    if (!c->scratch) {
        const size_t stride = (bytes + 255) / 256 * 256;
        if (cudaMalloc(&c->scratch, 4 * stride) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(ST_ERR_OOM, "stencil_cavity_bind: scratch allocation failed");
        }
        char* sc = (char*)c->scratch;
        c->B.u[1] = sc;
        c->B.v[1] = sc + stride;
        c->B.p[1] = sc + 2 * stride;
        c->B.b = sc + 3 * stride;
    }
    c->B.u[0] = u;
    c->B.v[0] = v;
    c->B.p[0] = p;
    c->B.cu = c->B.cp = 0;
    return ST_OK;
}

st_status stencil_cavity_step(st_cavity_t c, int nsteps, void* stream)
{
    if (!c) return fail(ST_ERR_ARG, "stencil_cavity_step: NULL handle");
    if (nsteps < 0) return fail(ST_ERR_ARG, "stencil_cavity_step: negative step count");
    if (!c->B.u[0]) return fail(ST_ERR_STATE, "stencil_cavity_step: buffers not bound");
    cudaStream_t s = (cudaStream_t)stream;
    for (int k = 0; k < nsteps; ++k) ST_CUDA_TRY(cavity_step(c->P, c->B, s));
    // the results go back to the caller's buffers
    const size_t bytes = (size_t)c->P.ny * (size_t)c->P.nx * (size_t)c->P.esize;
    if (c->B.cu == 1) {
        ST_CUDA_TRY(cudaMemcpyAsync(c->B.u[0], c->B.u[1], bytes, cudaMemcpyDeviceToDevice, s));
        ST_CUDA_TRY(cudaMemcpyAsync(c->B.v[0], c->B.v[1], bytes, cudaMemcpyDeviceToDevice, s));
        c->B.cu = 0;
    }
    if (c->B.cp == 1) {
        ST_CUDA_TRY(cudaMemcpyAsync(c->B.p[0], c->B.p[1], bytes, cudaMemcpyDeviceToDevice, s));
        c->B.cp = 0;
    }
    return ST_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched form
// ---------------------------------------------------------------------------
struct st_batch_s {
    int ngrids = 0;
    int npts = 0;
    st_bc bc = ST_PERIODIC;
    double bc_value = 0.0;
    st_dtype dtype = ST_F32;
    uint32_t flags = 0;
    std::vector<int32_t> off;      // npts * 2
    std::vector<double> weights;   // ngrids * npts
    std::vector<Geom> geoms;
    std::vector<void*> a, b;
    bool bound = false;
    int cur = 0;
    BatchPlan plan;
    cudaStream_t last = nullptr;
    cudaStream_t cap = nullptr;
    std::map<int, cudaGraphExec_t> graphs;  // keyed by nsteps * 2 + cur
    int* d_status = nullptr;
};

static void drop_batch_graphs(st_batch_t b)
{
    for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

extern "C" {

st_status stencil_batch_create(st_batch_t* out, int ngrids, const int64_t* dims, int npts, const int32_t* offsets,
                               const double* weights, st_bc bc, double bc_value, st_dtype dtype, uint32_t flags)
{
    if (!out) return fail(ST_ERR_ARG, "stencil_batch_create: out is NULL");
    *out = nullptr;
    if (ngrids < 1 || !dims || !offsets || !weights) return fail(ST_ERR_ARG, "stencil_batch_create: bad arguments");
    if (npts < 1 || npts > ST_MAX_POINTS) return fail(ST_ERR_ARG, "stencil_batch_create: npts out of range");
    if (bc != ST_DIRICHLET && bc != ST_PERIODIC) return fail(ST_ERR_ARG, "stencil_batch_create: bad bc");
    if (dtype != ST_F32 && dtype != ST_F64) return fail(ST_ERR_ARG, "stencil_batch_create: bad dtype");
    if (flags & ~ST_FLAG_GENERIC) return fail(ST_ERR_ARG, "stencil_batch_create: unknown flags");
    int r = 0;
    for (int k = 0; k < 2 * npts; ++k) {
        const int32_t o = offsets[k];
        if (o < -ST_MAX_RADIUS || o > ST_MAX_RADIUS) return fail(ST_ERR_ARG, "stencil_batch_create: offset too large");
        r = std::max(r, o < 0 ? -o : o);
    }
    st_batch_t b = new (std::nothrow) st_batch_s();
    if (!b) return fail(ST_ERR_OOM, "stencil_batch_create: out of host memory");
    b->ngrids = ngrids;
    b->npts = npts;
    b->bc = bc;
    b->bc_value = bc_value;
    b->dtype = dtype;
    b->flags = flags;
    b->off.assign(offsets, offsets + 2 * npts);
    b->weights.assign(weights, weights + (size_t)ngrids * npts);
    for (int i = 0; i < ngrids; ++i) {
        const int64_t d[2] = {dims[2 * i], dims[2 * i + 1]};
        if (d[0] < 1 || d[1] < 1 || d[0] > (1 << 24) || d[1] > (1 << 24)) {
            delete b;
            return fail(ST_ERR_ARG, "stencil_batch_create: grid extent out of range");
        }
        if (bc == ST_PERIODIC && (r >= d[0] || r >= d[1])) {
            delete b;
            return fail(ST_ERR_ARG, "stencil_batch_create: periodic offset not smaller than a grid extent");
        }
        b->geoms.push_back(make_geom(2, d, r, dtype == ST_F64 ? 8 : 4));
    }
    b->a.assign(ngrids, nullptr);
    b->b.assign(ngrids, nullptr);
    b->plan = make_batch_plan(b->geoms, b->npts, b->off.data(), b->weights.data(), bc == ST_PERIODIC, dtype,
                              (flags & ST_FLAG_GENERIC) != 0);
    b->plan.bc = bc_value;
    *out = b;
    return ST_OK;
}

st_status stencil_batch_destroy(st_batch_t b)
{
    if (!b) return ST_OK;
    drop_batch_graphs(b);
    free_batch_plan(b->plan);
    if (b->cap) cudaStreamDestroy(b->cap);
    if (b->d_status) cudaFree(b->d_status);
    delete b;
    return ST_OK;
}

st_status stencil_batch_layout(st_batch_t b, int i, int64_t* padded_dims, int64_t* origin, int64_t* elems)
{
    if (!b) return fail(ST_ERR_ARG, "stencil_batch_layout: NULL handle");
    if (i < 0 || i >= b->ngrids) return fail(ST_ERR_ARG, "stencil_batch_layout: grid index out of range");
    const Geom& G = b->geoms[i];
    if (padded_dims) {
        padded_dims[0] = G.pny;
        padded_dims[1] = G.pitch;
    }
    if (origin) {
        origin[0] = G.r;
        origin[1] = G.xl;
    }
    if (elems) *elems = G.elems;
    return ST_OK;
}

st_status stencil_batch_bind(st_batch_t b, void* const* pa, void* const* pb)
{
    if (!b || !pa || !pb) return fail(ST_ERR_ARG, "stencil_batch_bind: NULL argument");
    for (int i = 0; i < b->ngrids; ++i) {
        if (!pa[i] || !pb[i]) return fail(ST_ERR_ARG, "stencil_batch_bind: NULL grid pointer");
        if ((((uintptr_t)pa[i]) | ((uintptr_t)pb[i])) & 15u)
            return fail(ST_ERR_ARG, "stencil_batch_bind: pointer not 16-byte aligned");
        const size_t bytes = (size_t)b->geoms[i].elems * b->geoms[i].esize;
        const uintptr_t l1 = (uintptr_t)pa[i], l2 = (uintptr_t)pb[i];
        if (l1 < l2 + bytes && l2 < l1 + bytes) return fail(ST_ERR_ALIAS, "stencil_batch_bind: A and B overlap");
    }
    if (!b->cap) ST_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
    if (!b->d_status) {
        if (cudaMalloc(&b->d_status, sizeof(int)) != cudaSuccess) {
            (void)cudaGetLastError();
            return fail(ST_ERR_OOM, "stencil_batch_bind: scratch allocation failed");
        }
        ST_CUDA_TRY(cudaMemset(b->d_status, 0, sizeof(int)));
    }
    b->a.assign(pa, pa + b->ngrids);
    b->b.assign(pb, pb + b->ngrids);
    drop_batch_graphs(b);
    st_status rc = bind_batch_plan(b->plan, b->geoms, b->a.data(), b->b.data(), b->d_status);
    if (rc != ST_OK) return rc;
    // Dirichlet ghosts of every grid
    if (b->bc == ST_DIRICHLET)
        for (int i = 0; i < b->ngrids; ++i) {
            ST_CUDA_TRY(launch_fill_ghosts(b->geoms[i].esize, b->a[i], b->geoms[i], b->bc_value, nullptr));
            ST_CUDA_TRY(launch_fill_ghosts(b->geoms[i].esize, b->b[i], b->geoms[i], b->bc_value, nullptr));
        }
    ST_CUDA_TRY(cudaStreamSynchronize(nullptr));
    b->bound = true;
    b->cur = 0;
    return ST_OK;
}

static st_status batch_enqueue(st_batch_t b, int n, int cur, cudaStream_t s)
{
    return enqueue_batch_plan(b->plan, n, cur, s);
}

st_status stencil_batch_step(st_batch_t b, int nsteps, void* stream)
{
    if (!b) return fail(ST_ERR_ARG, "stencil_batch_step: NULL handle");
    if (nsteps < 0) return fail(ST_ERR_ARG, "stencil_batch_step: negative step count");
    if (!b->bound) return fail(ST_ERR_STATE, "stencil_batch_step: bind first");
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    if (nsteps == 0) return ST_OK;
    bool moved = false;
    st_status rc = reserve_batch_steps(b->plan, nsteps, &moved);
    if (rc != ST_OK) return rc;
    if (moved) drop_batch_graphs(b);  // graphs captured earlier point at the old counters
    const int key = nsteps * 2 + b->cur;
    auto it = b->graphs.find(key);
    for (int attempt = 0; it == b->graphs.end() && attempt < 2; ++attempt) {
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        ST_CUDA_TRY(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        st_status erc = batch_enqueue(b, nsteps, b->cur, b->cap);
        cudaError_t ce = cudaStreamEndCapture(b->cap, &graph);
        if (erc == ST_OK && ce == cudaSuccess) {
            ce = cudaGraphInstantiate(&exec, graph, 0);
            cudaGraphDestroy(graph);
            if (ce == cudaSuccess) {
                it = b->graphs.emplace(key, exec).first;
                break;
            }
        } else if (graph) {
            cudaGraphDestroy(graph);
        }
        (void)cudaGetLastError();
        if (attempt == 1) return erc != ST_OK ? erc : cuda_fail(ce, "batch graph capture");
        batch_disable_coop(b->plan);  // retry with one launch per pass
    }
    ST_CUDA_TRY(cudaGraphLaunch(it->second, s));
    b->cur = batch_final_slot(b->plan, nsteps, b->cur);
    return ST_OK;
}

st_status stencil_batch_tune(st_batch_t b, int nsteps, void* stream)
{
    if (!b) return fail(ST_ERR_ARG, "stencil_batch_tune: NULL handle");
    if (nsteps < 1) return fail(ST_ERR_ARG, "stencil_batch_tune: nsteps >= 1");
    if (!b->bound) return fail(ST_ERR_STATE, "stencil_batch_tune: bind first");
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    st_status rc = tune_batch_plan(b->plan, b->geoms, b->a.data(), b->b.data(), nsteps, b->cur, s);
    drop_batch_graphs(b);
    return rc;
}

st_status stencil_batch_selftest_barrier(st_batch_t b, uint64_t timeout_ns, void* stream)
{
    if (!b) return fail(ST_ERR_ARG, "stencil_batch_selftest_barrier: NULL handle");
    if (!b->bound) return fail(ST_ERR_STATE, "stencil_batch_selftest_barrier: bind first");
    if (timeout_ns < 1000000ull || timeout_ns > 5000000000ull)
        return fail(ST_ERR_ARG, "stencil_batch_selftest_barrier: timeout must be 1 ms .. 5 s");
    cudaStream_t s = (cudaStream_t)stream;
    b->last = s;
    st_status rc = batch_barrier_selftest(b->plan, b->cur, s, timeout_ns);
    if (rc != ST_OK) return rc;
    b->cur = 1 - b->cur;  // the pass before the barrier advanced one step
    return ST_OK;
}

st_status stencil_batch_config(st_batch_t b, int* cfg)
{
    if (!b || !cfg) return fail(ST_ERR_ARG, "stencil_batch_config: NULL argument");
    batch_plan_config(b->plan, cfg);
    return ST_OK;
}

st_status stencil_batch_current(st_batch_t b, int* slot)
{
    if (!b || !slot) return fail(ST_ERR_ARG, "stencil_batch_current: NULL argument");
    *slot = b->cur;
    return ST_OK;
}

st_status stencil_batch_sync(st_batch_t b)
{
    if (!b) return fail(ST_ERR_ARG, "stencil_batch_sync: NULL handle");
    ST_CUDA_TRY(cudaStreamSynchronize(b->last));
    if (!b->d_status) return ST_OK;
    int code = 0;
    ST_CUDA_TRY(cudaMemcpy(&code, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (code != 0) {
        ST_CUDA_TRY(cudaMemset(b->d_status, 0, sizeof(int)));
        if (code == ST_ERR_DEVICE_TIMEOUT) return fail(ST_ERR_DEVICE_TIMEOUT, "device: bounded wait ran out");
        return fail(ST_ERR_BOUNDS, "device: bounds check fired");
    }
    return ST_OK;
}

}  // extern "C"

namespace st {
// Accessors for translation units that do not see st_grid_s.
const Geom* grid_geom(st_grid_t g) { return &g->g; }
int* grid_status(st_grid_t g) { return g->d_status; }
void grid_note_stream(st_grid_t g, cudaStream_t s) { g->last = s; }
}  // namespace st
