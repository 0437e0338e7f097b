// 2D grids on the persistent tile kernel (k_batch.cu, a batch of one grid):
// which 2D stencils qualify, and the single-step launch used where a step
// must go from one explicit buffer to another (checkpointed forward and the
// recomputation inside the adjoint), which is the one-thread-per-point kernel.
//
// Small FP64 2D grids (the 256^2 heat workload: 100 dependent sweeps of
// 65,536 points) are bound by the dependency from one sweep to the next,
// not by HBM: every sweep pays a launch, an L2 round trip for its inputs
// and its own completion, about 1.7 us around 0.52 us of FP64 arithmetic.
// k_tb2d runs k steps per launch instead: each CTA owns a TX x TY tile,
// loads it with a k-cell halo into shared memory once, advances the region
// k times (it shrinks by one cell per step, so the halo work is redundant
// but the loads, the launch and the completion are paid once per k steps),
// and writes the tile.  Launches are static tile grids with programmatic
// dependencies, no tile counter and no grid barrier.  Each point is
// evaluated as the one-thread-per-point kernel does (acc = 0, then acc =
// fma(w_k, u[p + o_k], acc) over the offsets in order), so the results are
// the same bits.  stencil_tune picks TX, TY and k by timing.
#include <algorithm>

#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

struct TB2Params {
    int nx, ny;
    int64_t pitch, origin;
    int npts;
    int dy[9], dx[9];
    double w[9];
    int periodic;
    double bc;     // Dirichlet boundary value (the ghost cells' value)
    int TX, TY;    // output tile
    int ks;        // steps in this launch = halo width in cells
};

__device__ __forceinline__ int wrap_any(int i, int n)
{
    i %= n;
    return i < 0 ? i + n : i;
}

// c / w for 0 <= c < 2^20 and 1 <= w <= 2^10 by a float reciprocal, corrected
// to the exact quotient (one step each way suffices at these sizes)
__device__ __forceinline__ int div_small(int c, int w, float inv_w, int& rem)
{
    int q = __float2int_rz((float)c * inv_w);
    int r = c - q * w;
    if (r >= w) {
        ++q;
        r -= w;
    } else if (r < 0) {
        --q;
        r += w;
    }
    rem = r;
    return q;
}

constexpr int TB_THREADS = 512;

__global__ void __launch_bounds__(TB_THREADS) k_tb2d(const double* __restrict__ in, double* __restrict__ out,
                                                     const __grid_constant__ TB2Params P)
{
    extern __shared__ __align__(16) double tb_sm[];
    ptx::griddep_wait();  // the previous launch wrote `in` and read `out`
    ptx::griddep_trigger();
    const int h = P.ks;
    const int RW = P.TX + 2 * h, RH = P.TY + 2 * h;
    double* A = tb_sm;
    double* B = tb_sm + RW * RH;
    const int x0 = (int)blockIdx.x * P.TX - h, y0 = (int)blockIdx.y * P.TY - h;
    // weights and region offsets in registers (at most 9 points, loop unrolled)
    double wk[9];
    int ok[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        wk[k] = k < P.npts ? P.w[k] : 0.0;
        ok[k] = k < P.npts ? P.dy[k] * RW + P.dx[k] : 0;
    }
    // the region with its halo: wrapped when periodic; outside the interior
    // a Dirichlet region holds the boundary value, in both buffers, for good
    const float inv_rw = 1.0f / (float)RW;
    for (int c = threadIdx.x; c < RW * RH; c += blockDim.x) {
        int i;
        const int j = div_small(c, RW, inv_rw, i);
        int gx = x0 + i, gy = y0 + j;
        double v;
        if (P.periodic) {
            gx = wrap_any(gx, P.nx);
            gy = wrap_any(gy, P.ny);
            v = in[P.origin + (int64_t)gy * P.pitch + gx];
        } else {
            v = (gx >= 0 && gx < P.nx && gy >= 0 && gy < P.ny) ? in[P.origin + (int64_t)gy * P.pitch + gx] : P.bc;
        }
        A[c] = v;
        B[c] = v;
    }
    __syncthreads();
    for (int st = 1; st <= h; ++st) {
        // cells [st, RW - st) x [st, RH - st) hold level st after this step;
        // their neighbours lie in the region of level st - 1
        const int w = RW - 2 * st, hh = RH - 2 * st;
        const float inv_w = 1.0f / (float)w;
        for (int c = threadIdx.x; c < w * hh; c += blockDim.x) {
            int ii;
            const int jj = div_small(c, w, inv_w, ii);
            const int i = ii + st, j = jj + st;
            if (!P.periodic) {
                const int gx = x0 + i, gy = y0 + j;
                if (gx < 0 || gx >= P.nx || gy < 0 || gy >= P.ny) continue;
            }
            const double* a = A + j * RW + i;
            double acc = 0.0;
#pragma unroll
            for (int k = 0; k < 9; ++k)
                if (k < P.npts) acc = fma(wk[k], a[ok[k]], acc);
            B[j * RW + i] = acc;
        }
        __syncthreads();
        double* t = A;
        A = B;
        B = t;
    }
    const float inv_tx = 1.0f / (float)P.TX;
    for (int c = threadIdx.x; c < P.TX * P.TY; c += blockDim.x) {
        int ii;
        const int jj = div_small(c, P.TX, inv_tx, ii);
        const int gx = (int)blockIdx.x * P.TX + ii, gy = (int)blockIdx.y * P.TY + jj;
        if (gx < P.nx && gy < P.ny) out[P.origin + (int64_t)gy * P.pitch + gx] = A[(jj + h) * RW + ii + h];
    }
}

}  // namespace

size_t tb2d_smem(int TX, int TY, int k) { return 2 * (size_t)(TX + 2 * k) * (TY + 2 * k) * sizeof(double); }

bool tb2d_fits(int64_t nx, int64_t ny, int TX, int TY, int k)
{
    return TX >= 1 && TY >= 1 && k >= 1 && TX + 2 * k <= 1024 && (int64_t)TX * TY <= (1 << 18) &&
           tb2d_smem(TX, TY, k) <= 200 * 1024 && (nx + TX - 1) / TX <= 0x7fffffff && (ny + TY - 1) / TY <= 65535 &&
           nx < 0x7fffffff && ny < 0x7fffffff;
}

bool tb2d_supports(const Family& f)
{
    const GenParams& G = f.gp;
    if (f.g.ndim != 2 || f.g.esize != 8 || f.levels != 1 || f.has_beta || G.npts > 9) return false;
    for (int k = 0; k < G.npts; ++k)
        if (G.dy[k] < -1 || G.dy[k] > 1 || G.dx[k] < -1 || G.dx[k] > 1 || G.dz[k] != 0) return false;
    return true;
}

cudaError_t launch_tb2d(const Family& f, const void* in, void* out, int TX, int TY, int ks, double bc, cudaStream_t s)
{
    if (!tb2d_supports(f) || !tb2d_fits(f.g.nx, f.g.ny, TX, TY, ks)) return cudaErrorInvalidValue;
    const GenParams& G = f.gp;
    TB2Params P{};
    P.nx = (int)f.g.nx;
    P.ny = (int)f.g.ny;
    P.pitch = f.g.pitch;
    P.origin = f.g.origin;
    P.npts = G.npts;
    for (int k = 0; k < G.npts; ++k) {
        P.dy[k] = G.dy[k];
        P.dx[k] = G.dx[k];
        P.w[k] = G.alpha[k];
    }
    P.periodic = f.periodic ? 1 : 0;
    P.bc = bc;
    P.TX = TX;
    P.TY = TY;
    P.ks = ks;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_tb2d, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const dim3 grid((unsigned)((P.nx + TX - 1) / TX), (unsigned)((P.ny + TY - 1) / TY));
    return launch_dependent(k_tb2d, grid, dim3(TB_THREADS), tb2d_smem(TX, TY, ks), s, static_cast<const double*>(in),
                            static_cast<double*>(out), P);
}

bool tile2d_supports(const FamilyDesc& d, int* variant, const char** name)
{
    // FP32 only: for FP64 a grid barrier per step costs more than a graph
    // launch, and temporal blocking multiplies work on the slow FP64 pipe
    if (d.g.ndim != 2 || d.levels != 1 || d.has_beta || d.npts > 9 || d.g.esize != 4) return false;
    for (int k = 0; k < d.npts; ++k)
        for (int i = 1; i < 3; ++i)
            if (d.off[3 * k + i] < -1 || d.off[3 * k + i] > 1) return false;
    *variant = 1;
    *name = "tile2d_persistent";
    return true;
}

cudaError_t launch_tile2d(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    GenParams P = f.gp;
    P.src = a.src;
    P.src_amp = a.src_amp;
    P.src_count = a.src_count;
    P.step = a.step;
    return launch_generic_sweep(f.g.esize, a.in, a.out, a.prev, a.kappa, P, s);
}

}  // namespace st
