// Internal declarations shared by the translation units of libstencil.
// Not part of the public ABI (that is include/stencil.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/stencil.h"

namespace st {

// ---------------------------------------------------------------------------
// Error reporting (thread-local message behind stencil_last_error)
// ---------------------------------------------------------------------------
void set_error(const std::string& msg);
st_status fail(st_status code, const std::string& msg);
st_status cuda_fail(cudaError_t e, const char* what);

#define ST_CUDA_TRY(expr)                                   \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) return ::st::cuda_fail(_e, #expr); \
    } while (0)

// Launch kernel k on stream s with a programmatic dependency on the previous
// kernel of the stream: k's CTAs may be scheduled (and run their prologue)
// while that kernel finishes, which hides the launch gap between the
// dependent sweeps of a step sequence.  k must call ptx::griddep_wait()
// before touching global memory that earlier work reads or writes.
template <typename... KP, typename... A>
cudaError_t launch_dependent(void (*k)(KP...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args)
{
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------------------
// Padded-grid geometry.  2D grids are stored as one plane: nz = 1, no z ghosts.
// ---------------------------------------------------------------------------
struct Geom {
    int ndim;        // 2 or 3
    int r;           // ghost width (x and y, and z in 3D)
    int rz;          // ghost width along z (0 in 2D)
    int esize;       // bytes per element
    int64_t nz, ny, nx;  // interior extents
    int64_t xl;      // padded column of interior x = 0 (16-byte aligned)
    int64_t pitch;   // padded row length in elements (multiple of 16 bytes)
    int64_t pny;     // padded rows per plane
    int64_t pnz;     // padded planes
    int64_t plane;   // elements per padded plane
    int64_t elems;   // elements per buffer
    int64_t origin;  // linear index of interior (0, 0, 0)
    int64_t npoints; // interior points
};

Geom make_geom(int ndim, const int64_t* dims, int r, int esize);

// Parameters of the one-thread-per-point kernels (passed by value).
struct GenParams {
    int64_t nz, ny, nx;
    int64_t pitch, plane, origin;
    int npts;
    int periodic;
    int leapfrog;
    int has_kappa;
    int64_t src;           // linear padded index of the source point, -1: none
    const double* src_amp; // device amplitudes
    int64_t src_count;
    int64_t step;          // step index of this launch (for the source)
    int32_t dz[ST_MAX_POINTS], dy[ST_MAX_POINTS], dx[ST_MAX_POINTS];
    int64_t lin[ST_MAX_POINTS];  // linear offset in the padded layout
    double alpha[ST_MAX_POINTS], beta[ST_MAX_POINTS];
    // the same weights rounded to float once on the host: an FP32 kernel that
    // converted them per point would keep the FP64 pipe (where the
    // conversion runs, 2 lanes per clock per SM on this GPU) busy
    float alpha_f[ST_MAX_POINTS], beta_f[ST_MAX_POINTS];
};

// Fill alpha_f / beta_f from alpha / beta.
void gen_params_floats(GenParams& P);

// Kernel launchers (k_generic.cu) -------------------------------------------
cudaError_t launch_generic_sweep(int esize, const void* in, void* out, const void* prev,
                                 const void* kappa, const GenParams& P, cudaStream_t s);
cudaError_t launch_generic_adjoint(int esize, const void* u_t, const void* lam_in, void* lam_out,
                                   const void* kappa, double* gk, const GenParams& P,
                                   cudaStream_t s);
// Transposed step of the zero-flux (Neumann) sweep, constant weights: the
// gather over the mirror pre-images of every interior cell.
cudaError_t launch_neumann_adjoint(int esize, const void* lam_in, void* lam_out, const GenParams& P, int r, int rz,
                                   cudaStream_t s);
cudaError_t launch_fill_ghosts(int esize, void* buf, const Geom& g, double value, cudaStream_t s);
// dev_out = the combination of nblocks (sum, sum of squares, max) partials
cudaError_t launch_reduce_final(const double* partials, int nblocks, double* out, cudaStream_t s);
cudaError_t launch_mirror_ghosts(int esize, void* buf, const Geom& g, cudaStream_t s);
cudaError_t launch_pack(int esize, void* dense, void* padded, const Geom& g, int dir, cudaStream_t s);
// Grid size of the reduction kernels for grid g: the blocks resident at once
// on this GPU, at most max_blocks and at most one per eight interior rows.
int reduce_blocks(const Geom& g, int max_blocks);
// status: the grid's device status word (a timed-out wait of the FP32 ring
// kernel records ST_ERR_DEVICE_TIMEOUT there); may be NULL.
cudaError_t launch_reduce(int esize, const void* a, const void* b, const Geom& g, double* partials,
                          int nblocks, double* out, int mode, void* lam_out, int* status, cudaStream_t s);

}  // namespace st
