// Kernel families: which kernel a grid handle dispatches to, and the
// launch-argument structs shared by the step driver and the kernels.
#pragma once

#include <vector>

#include "common.cuh"

namespace st {

enum FamilyKind {
    FAM_GENERIC = 0,    // one thread per point, any stencil (k_generic.cu)
    FAM_STAR3D = 1,     // 3D star, z-streaming with bulk-copy staged planes (k_star3d.cu)
    FAM_2D_TILE = 2,    // 2D tile kernel (k_2d.cu)
    FAM_WAVE = 3,       // 3D radius-4 leapfrog star (k_wave.cu)
    FAM_CONS = 4,       // conservative face-averaged per-cell diffusion, one thread per point (k_cons.cu)
};

struct FamilyDesc {
    Geom g;
    int npts;
    const int32_t* off;  // npts * 3 (dz, dy, dx)
    const double* alpha;
    const double* beta;
    bool has_beta;
    bool periodic;
    int levels;
    bool star;
    bool force_generic;
};

// Star stencil coefficients in per-axis form: centre weight plus, for every
// axis a (0 = z, 1 = y, 2 = x), side s (0: -j, 1: +j) and distance j (1..R),
// the constant part ca and per-cell part cb of the weight.
struct StarCoef {
    int R;
    double c_a, c_b;
    double a[3][2][ST_MAX_RADIUS];
    double b[3][2][ST_MAX_RADIUS];
};

struct Family {
    FamilyKind kind;
    const char* name;
    GenParams gp;   // generic parameters (also used by the adjoint)
    StarCoef sc;    // star families
    Geom g;
    bool periodic;
    bool has_beta;
    int levels;
    int variant;    // family-specific launch variant
};

struct SweepArgs {
    const void* in;
    void* out;
    const void* prev;   // u_{t-1} (leapfrog; equals out)
    const void* kappa;
    int64_t step;
    int64_t src;
    const double* src_amp;
    int64_t src_count;
    int* status;
};

struct AdjointArgs {
    const void* u;       // u_t
    const void* u2;      // u_{t-1} (steps == 2)
    const void* lam_in;  // lambda_{t+1}
    void* lam_out;       // lambda_{t+1-steps}
    const void* kappa;
    double* gk;          // FP64 gradient accumulator (NULL: no gradient)
    void* gpart;         // FP32 grids on the fused kernel: the segment's FP32 partial gradient
    int gfirst;          // this pass is the first of its checkpoint segment (FP32 partial gradient)
    int steps;           // transpose steps fused in this launch (1 or 2)
    int* status;
};

Family select_family(const FamilyDesc& d);
cudaError_t launch_family(const Family& f, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_family_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s);

// Optimised kernels (return cudaErrorNotSupported when the case is not theirs)
cudaError_t launch_star3d(const Family& f, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_star3d_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s);
// One sweep of a constant symmetric FP32 3D star that also reduces the level it
// writes into out = (sum, sum of squares, max |u|) over the interior, through
// `partials` (3 doubles per block, room for `cap` blocks).
bool star3d_reduce_supported(const Family& f);
cudaError_t launch_star3d_reduce(const Family& f, const SweepArgs& a, double* partials, int cap, double* out,
                                 cudaStream_t s);
// gk += part (an FP32 partial gradient into the FP64 gradient), n elements, a
// multiple of 4, both buffers 16-byte aligned.
cudaError_t launch_grad_flush(void* part, double* gk, int64_t n, cudaStream_t s);
int star3d_adjoint_fuse(const Family& f);
// gk += part, part = 0 over n elements (part: FP32 partial gradient).
// Two sweeps per pass of the constant symmetric 7-point star (FP32): a.in -> a.out
bool star3d_pair_supported(const Family& f);
cudaError_t launch_star3d_pair(const Family& f, const SweepArgs& a, double bc_value, cudaStream_t s);
bool star3d_supports(const FamilyDesc& d, int* variant, const char** name);
cudaError_t launch_tile2d(const Family& f, const SweepArgs& a, cudaStream_t s);
bool wave_supports(const FamilyDesc& d);
cudaError_t launch_wave(const Family& f, const SweepArgs& a, cudaStream_t s);
bool tile2d_supports(const FamilyDesc& d, int* variant, const char** name);
// FP64 2D grids, offsets within the 3x3 neighbourhood, constant weights: ks
// steps of the sweep in one launch of TX x TY tiles (k_2d.cu); the same bits
// as ks single sweeps.  tb2d_smem: its dynamic shared memory for k steps.
bool tb2d_supports(const Family& f);
size_t tb2d_smem(int TX, int TY, int k);
// the launch limits of a TX x TY tile grid of k steps on an nx x ny grid
bool tb2d_fits(int64_t nx, int64_t ny, int TX, int TY, int k);
cudaError_t launch_tb2d(const Family& f, const void* in, void* out, int TX, int TY, int ks, double bc,
                        cudaStream_t s);
cudaError_t launch_cons_sweep(const Family& f, const SweepArgs& a, cudaStream_t s);
// The conservative operator's 3D forward on the staged pipeline of k_star1
// (variant 1 of FAM_CONS); its coefficient field's ghosts must mirror the
// interior (see stencil_create_conservative).
bool star3d_cons_supported(const Geom& g);
cudaError_t launch_star3d_cons(const Family& f, const SweepArgs& a, cudaStream_t s);
cudaError_t launch_cons_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s);
// The conservative operator's coefficient gradient of n <= cons_grad_max_pairs()
// transposed steps (3D): gk += sum over k of the step term of (u[k], lam[k]),
// u[k] the state u_t and lam[k] lambda_{t+1} of one step.
cudaError_t launch_cons_grad(const Family& f, const void* const* u, const void* const* lam, int n, double* gk,
                             cudaStream_t s);
int cons_grad_max_pairs();

// ---------------------------------------------------------------------------
// Batched plan (k_batch.cu)
// ---------------------------------------------------------------------------
struct BatchPlan {
    int ngrids = 0;
    int npts = 0;
    bool periodic = true;
    int esize = 4;
    bool generic = false;
    std::vector<GenParams> gp;     // per-grid generic parameters
    std::vector<void*> a, b;
    // persistent-kernel tables (device)
    void* d_desc = nullptr;        // per-grid descriptors
    void* d_work = nullptr;        // work items
    int nwork = 0;
    int cfg[4] = {0, 0, 0, 0};     // tile x, tile y, threads, steps per pass
    int* status = nullptr;
    int nsm = 0;
    std::vector<double> weights;
    std::vector<int32_t> off;
    double bc = 0.0;
    int shape = 0;                 // 0: 3x3 box, 1: five-point star
};

BatchPlan make_batch_plan(const std::vector<Geom>& geoms, int npts, const int32_t* off2, const double* weights,
                          bool periodic, st_dtype dtype, bool force_generic);
st_status bind_batch_plan(BatchPlan& p, const std::vector<Geom>& geoms, void* const* a, void* const* b, int* status);
st_status enqueue_batch_plan(BatchPlan& p, int nsteps, int cur, cudaStream_t s);
st_status tune_batch_plan(BatchPlan& p, const std::vector<Geom>& geoms, void* const* a, void* const* b, int nsteps,
                          int cur, cudaStream_t s);
void batch_plan_config(const BatchPlan& p, int* cfg);
void free_batch_plan(BatchPlan& p);
// Slot holding the result after nsteps from slot cur (temporal blocking writes once per pass).
int batch_final_slot(const BatchPlan& p, int nsteps, int cur);
// Allocate per-pass counters for calls of up to nsteps (before any graph
// capture); *moved tells that an existing table was replaced.
st_status reserve_batch_steps(BatchPlan& p, int nsteps, bool* moved);
// Use one launch per pass from now on (cooperative launch unavailable).
void batch_disable_coop(BatchPlan& p);
// Failure-detection hook: one pass, then a grid barrier that waits for one
// CTA more than launched, so its bounded wait must run out.
st_status batch_barrier_selftest(BatchPlan& p, int cur, cudaStream_t s, unsigned long long timeout_ns);

}  // namespace st
