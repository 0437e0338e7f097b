// Lid-driven cavity flow, the paper's multi-field benchmark (Sec. V-B):
// incompressible Navier-Stokes on a uniform 2D grid, one explicit time step =
// pressure source from (u, v), nit Jacobi iterations of the pressure Poisson
// equation with its boundary rule, then u and v from the old velocities and
// the new pressure with the wall and lid values.  Arrays are dense (ny, nx),
// C order, boundary rows and columns included (y along axis 0, x along
// axis 1).
//
// GB300 design: every cell of the whole array has a thread (the pressure
// kernel: a thread per column walking 16 rows), so each kernel also writes
// its boundary cells and no separate boundary pass runs:
//  * the pressure iteration's boundary rule (right column copies its left
//    neighbour, bottom row the row above, left column its right neighbour,
//    then the top row is set to 0) leaves every boundary cell below the top
//    row equal to the new value of the interior cell at its index clamped
//    into [1, n - 2] on both axes, so a boundary thread recomputes that
//    interior update itself (same expression, same inputs, same result) and
//    the top row writes 0;
//  * the two momentum updates are fused in one kernel (the paper's node
//    fusion of updates with the same output shape): both read the same
//    neighbourhoods of u, v and p.
// FP64 is bound by the FP64 pipe, FP32 by memory latency and bandwidth.
#include "cavity.cuh"
#include "ptx.cuh"

namespace st {

namespace {

__device__ __forceinline__ int64_t clampi(int64_t i, int64_t n) { return i < 1 ? 1 : (i > n - 2 ? n - 2 : i); }

template <typename T>
__device__ __forceinline__ T cv(const CavityParams& P, int k)
{
    if constexpr (sizeof(T) == 4) return P.c32[k];
    else return P.c64[k];
}

template <typename T>
__global__ void __launch_bounds__(256) k_cav_source(const T* __restrict__ u, const T* __restrict__ v,
                                                    T* __restrict__ b, const __grid_constant__ CavityParams P)
{
    const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (i < 1 || j < 1 || i >= P.nx - 1 || j >= P.ny - 1) return;
    const int64_t c = j * P.nx + i;
    const T i2dx = cv<T>(P, CV_I2DX), i2dy = cv<T>(P, CV_I2DY);
    const T ux = (u[c + 1] - u[c - 1]) * i2dx;
    const T uy = (u[c + P.nx] - u[c - P.nx]) * i2dy;
    const T vx = (v[c + 1] - v[c - 1]) * i2dx;
    const T vy = (v[c + P.nx] - v[c - P.nx]) * i2dy;
    b[c] = cv<T>(P, CV_RHO) * ((ux + vy) * cv<T>(P, CV_IDT) - ux * ux - T(2) * uy * vx - vy * vy);
}

// One Jacobi update from its inputs: a single expression for every caller,
// so a boundary cell gets exactly its clamped interior cell's value.
template <typename T>
__device__ __forceinline__ T jacobi(T e, T w, T n, T s, T bb, const CavityParams& P)
{
    return ((e + w) * cv<T>(P, CV_DY2) + (n + s) * cv<T>(P, CV_DX2) - bb * cv<T>(P, CV_DX2DY2)) * cv<T>(P, CV_IPDEN);
}

// (Measured forms not kept, FP32 at 16384^2: one thread per cell gathering
// its four neighbours through L1, 274 GLUP/s; the block's cells and halo
// staged in shared memory, 159 GLUP/s.)
// A thread owns a column and walks RY rows of it, keeping the input pressure
// of the rows below, at and above its (clamped) centre in registers, so a
// cell costs one new row load, its two x neighbours (L1 hits: the warp
// loaded that row one step earlier) and its source value.  Boundary columns
// walk the clamped column (1 or nx - 2), boundary row 0 the clamped row 1.
constexpr int RY = 16;

template <typename T>
__global__ void __launch_bounds__(256) k_cav_pressure(const T* __restrict__ pin, T* __restrict__ pout,
                                                      const T* __restrict__ b, const __grid_constant__ CavityParams P)
{
    const int64_t i = (int64_t)blockIdx.x * 256 + threadIdx.x;
    if (i >= P.nx) return;
    const int64_t j0 = (int64_t)blockIdx.y * RY, j1 = j0 + RY < P.ny ? j0 + RY : P.ny;
    const int64_t ci = clampi(i, P.nx);
    int64_t r = clampi(j0, P.ny);              // centre row of the window
    T s = pin[(r - 1) * P.nx + ci], c = pin[r * P.nx + ci], n = pin[(r + 1) * P.nx + ci];
    for (int64_t j = j0; j < j1; ++j) {
        const int64_t o = j * P.nx + i;
        if (j == P.ny - 1) {  // the lid row: p = 0
            pout[o] = T(0);
            continue;
        }
        const int64_t rj = clampi(j, P.ny);
        if (rj != r) {  // advance the window by one row (rj == r + 1 here)
            r = rj;
            s = c;
            c = n;
            n = pin[(r + 1) * P.nx + ci];
        }
        const int64_t cc = r * P.nx + ci;
        pout[o] = jacobi(pin[cc + 1], pin[cc - 1], n, s, b[cc], P);
    }
}

// FP32 pressure iterations, k per pass (temporal blocking).  A block owns a
// tile of TBW x TBH cells and loads the tile plus a k-wide halo of p and of
// the source b (clipped to the array) into shared memory; each iteration
// updates the interior cells of a region that shrinks by one cell per
// iteration on every side facing another tile (the cells later iterations
// still need), then applies the boundary rule inside shared memory (a
// boundary cell below the top row takes the new value of its clamped
// interior cell, the top row 0), and the last iteration's tile is written
// back.  HBM traffic per k iterations: one read of the halo'd tile of p and
// b and one write of the tile, instead of k reads of p and b and k writes.
// Interior cells: a thread owns a 4-column group in a band of rows and walks
// down it with the rows above, at and below in registers (one 16-byte shared
// load of the next row, two edge loads, one 16-byte load of b and one store
// per 4 cells).
constexpr int TBW = 128, TBH = 32, TBK = 8, TBPAD = 4;

__host__ __device__ constexpr int tb_stride() { return TBW + 2 * TBK + 2 * TBPAD; }  // shared row stride

__device__ __forceinline__ void ld6f(const float* q, float (&v)[6])  // columns -1 .. 4 of a group
{
    v[0] = q[-1];
    const float4 t = *reinterpret_cast<const float4*>(q);
    v[1] = t.x;
    v[2] = t.y;
    v[3] = t.z;
    v[4] = t.w;
    v[5] = q[4];
}

__global__ void __launch_bounds__(256) k_cav_pressure_tb(const float* __restrict__ pin, float* __restrict__ pout,
                                                         const float* __restrict__ bsrc, int kp,
                                                         const __grid_constant__ CavityParams P)
{
    ptx::griddep_wait();  // the previous pass wrote this pass's input
    ptx::griddep_trigger();
    extern __shared__ __align__(16) float sm[];
    constexpr int RS = tb_stride();
    constexpr int RH = TBH + 2 * TBK;  // rows of a shared buffer
    float* s0 = sm;
    float* s1 = sm + RH * RS;
    float* sb = sm + 2 * RH * RS;
    const int nx = (int)P.nx, ny = (int)P.ny;
    const int x0 = blockIdx.x * TBW, y0 = blockIdx.y * TBH;
    // shared (ly, lx) holds the cell (y0 - kp + ly, x0 - kp + lx); a row's
    // element lx sits at ly * RS + TBPAD + lx (16-byte aligned groups)
    const int gx0 = x0 - kp, gy0 = y0 - kp;
    const int ry0 = max(0, gy0), ry1 = min(ny, y0 + TBH + kp);
    const int rx0 = max(0, gx0), rx1 = min(nx, x0 + TBW + kp);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int gy = ry0 + warp; gy < ry1; gy += 8) {
        const int ly = gy - gy0;
        const float* prow = pin + (int64_t)gy * nx;
        const float* brow = bsrc + (int64_t)gy * nx;
        for (int gx = rx0 + lane; gx < rx1; gx += 32) {
            const int o = ly * RS + TBPAD + (gx - gx0);
            ptx::cp_async_elem<4>(s0 + o, prow + gx);
            ptx::cp_async_elem<4>(sb + o, brow + gx);
        }
    }
    ptx::cp_async_wait_all();
    __syncthreads();
    const float dy2 = P.c32[CV_DY2], dx2 = P.c32[CV_DX2], dxy = P.c32[CV_DX2DY2], ipd = P.c32[CV_IPDEN];
    const float* in = s0 + TBPAD;
    float* outb = s1 + TBPAD;
    const float* bb = sb + TBPAD;
    // the boundary rule applies where the region (the tile and its halo)
    // reaches a boundary row or column, not only where the tile does
    const bool edge = gx0 <= 0 || gy0 <= 0 || x0 + TBW + kp >= nx || y0 + TBH + kp >= ny;
    for (int t = 1; t <= kp; ++t) {
        const int e = kp - t;  // the region: the tile grown by e cells, clipped to the array
        const int cy0 = max(0, y0 - e), cy1 = min(ny, y0 + TBH + e);
        const int cx0 = max(0, x0 - e), cx1 = min(nx, x0 + TBW + e);
        // interior cells of the region: rows [iy0, iy1), columns [ix0, ix1)
        const int iy0 = max(1, cy0), iy1 = min(ny - 1, cy1);
        const int ix0 = max(1, cx0), ix1 = min(nx - 1, cx1);
        if (iy0 < iy1 && ix0 < ix1) {
            const int lx0 = (ix0 - gx0) & ~3, lx1 = ix1 - gx0;  // group-aligned local columns
            const int ng = (lx1 - lx0 + 3) >> 2;
            const int nb = max(1, 256 / ng);
            const int gi = threadIdx.x % ng, band = threadIdx.x / ng;
            const int rows = iy1 - iy0, bh = (rows + nb - 1) / nb;
            const int r0 = iy0 - gy0 + band * bh, r1 = min(iy1 - gy0, r0 + bh);
            if (band < nb && r0 < r1) {
                const int lx = lx0 + 4 * gi;
                const float* q = in + (r0 - 1) * RS + lx;
                float A[6], B[6], C[6];
                ld6f(q, A);
                ld6f(q + RS, B);
                q += 2 * RS;
                auto row = [&](const float (&S)[6], const float (&M)[6], float (&N)[6], int ly) {
                    ld6f(q, N);
                    q += RS;
                    const float4 b4 = *reinterpret_cast<const float4*>(bb + ly * RS + lx);
                    const float bv[4] = {b4.x, b4.y, b4.z, b4.w};
                    float o[4];
#pragma unroll
                    for (int c = 0; c < 4; ++c)
                        o[c] = ((M[c + 2] + M[c]) * dy2 + (N[c + 1] + S[c + 1]) * dx2 - bv[c] * dxy) * ipd;
                    *reinterpret_cast<float4*>(outb + ly * RS + lx) = make_float4(o[0], o[1], o[2], o[3]);
                };
                int ly = r0;
                for (; ly + 3 <= r1; ly += 3) {
                    row(A, B, C, ly);
                    row(B, C, A, ly + 1);
                    row(C, A, B, ly + 2);
                }
                if (ly < r1) row(A, B, C, ly);
                if (ly + 1 < r1) row(B, C, A, ly + 1);
            }
        }
        __syncthreads();
        if (edge) {
            // the boundary rule on the region's boundary cells: below the top
            // row the new value of the clamped interior cell, the top row 0
            const int w = cx1 - cx0, h = cy1 - cy0;
            for (int idx = threadIdx.x; idx < 2 * (w + h); idx += 256) {
                int gy, gx;
                if (idx < w) {
                    gx = cx0 + idx;
                    gy = 0;
                } else if (idx < 2 * w) {
                    gx = cx0 + idx - w;
                    gy = ny - 1;
                } else if (idx < 2 * w + h) {
                    gy = cy0 + idx - 2 * w;
                    gx = 0;
                } else {
                    gy = cy0 + idx - 2 * w - h;
                    gx = nx - 1;
                }
                if (gy < cy0 || gy >= cy1 || gx < cx0 || gx >= cx1) continue;
                float val = 0.f;
                if (gy != ny - 1) {
                    const int cy = gy < 1 ? 1 : (gy > ny - 2 ? ny - 2 : gy);
                    const int cx = gx < 1 ? 1 : (gx > nx - 2 ? nx - 2 : gx);
                    val = outb[(cy - gy0) * RS + (cx - gx0)];
                }
                outb[(gy - gy0) * RS + (gx - gx0)] = val;
            }
            __syncthreads();
        }
        const float* tmp = in;
        in = outb;
        outb = const_cast<float*>(tmp);
    }
    // the tile of the last iteration
    const int ty1 = min(ny, y0 + TBH), tx1 = min(nx, x0 + TBW);
    for (int gy = y0 + warp; gy < ty1; gy += 8) {
        const float* srow = in + (gy - gy0) * RS;
        float* drow = pout + (int64_t)gy * nx;
        for (int gx = x0 + lane; gx < tx1; gx += 32) drow[gx] = srow[gx - gx0];
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_cav_velocity(const T* __restrict__ u, const T* __restrict__ v,
                                                      const T* __restrict__ p, T* __restrict__ u2,
                                                      T* __restrict__ v2, const __grid_constant__ CavityParams P)
{
    const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (i >= P.nx || j >= P.ny) return;
    const int64_t c = j * P.nx + i;
    if (j == P.ny - 1) {  // the lid
        u2[c] = cv<T>(P, CV_LID);
        v2[c] = T(0);
        return;
    }
    if (j == 0 || i == 0 || i == P.nx - 1) {  // the walls
        u2[c] = T(0);
        v2[c] = T(0);
        return;
    }
    const T nu = cv<T>(P, CV_NU), cx = cv<T>(P, CV_CX), cy = cv<T>(P, CV_CY), dxx = cv<T>(P, CV_DXX),
            dyy = cv<T>(P, CV_DYY);
    const T uc = u[c], ue = u[c + 1], uw = u[c - 1], un = u[c + P.nx], us = u[c - P.nx];
    const T vc = v[c], ve = v[c + 1], vw = v[c - 1], vn = v[c + P.nx], vs = v[c - P.nx];
    u2[c] = uc - uc * cx * (uc - uw) - vc * cy * (uc - us) - cv<T>(P, CV_GX) * (p[c + 1] - p[c - 1]) +
            nu * (dxx * (ue - T(2) * uc + uw) + dyy * (un - T(2) * uc + us));
    v2[c] = vc - uc * cx * (vc - vw) - vc * cy * (vc - vs) - cv<T>(P, CV_GY) * (p[c + P.nx] - p[c - P.nx]) +
            nu * (dxx * (ve - T(2) * vc + vw) + dyy * (vn - T(2) * vc + vs));
}

dim3 cav_grid(const CavityParams& P)
{
    return dim3((unsigned)((P.nx + 31) / 32), (unsigned)((P.ny + 7) / 8), 1);
}

template <typename T>
cudaError_t cav_step_t(const CavityParams& P, CavityBufs& B, cudaStream_t s)
{
    const dim3 g = cav_grid(P), blk(32, 8);
    const dim3 gp((unsigned)((P.nx + 255) / 256), (unsigned)((P.ny + RY - 1) / RY), 1);
    k_cav_source<T><<<g, blk, 0, s>>>((const T*)B.u[B.cu], (const T*)B.v[B.cu], (T*)B.b, P);
    if (sizeof(T) == 4 && P.tb) {
        // FP32: k pressure iterations per pass through shared memory
        const dim3 gt((unsigned)((P.nx + TBW - 1) / TBW), (unsigned)((P.ny + TBH - 1) / TBH), 1);
        const size_t smem = (size_t)3 * (TBH + 2 * TBK) * tb_stride() * sizeof(float);
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(k_cav_pressure_tb, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return e;
            attr = true;
        }
        for (int k = 0; k < P.nit; k += TBK) {
            const int kp = P.nit - k < TBK ? P.nit - k : TBK;
            cudaError_t e = launch_dependent(k_cav_pressure_tb, gt, dim3(256), smem, s, (const float*)B.p[B.cp],
                                             (float*)B.p[1 - B.cp], (const float*)B.b, kp, P);
            if (e != cudaSuccess) return e;
            B.cp = 1 - B.cp;
        }
    } else {
        for (int k = 0; k < P.nit; ++k) {
            k_cav_pressure<T><<<gp, 256, 0, s>>>((const T*)B.p[B.cp], (T*)B.p[1 - B.cp], (const T*)B.b, P);
            B.cp = 1 - B.cp;
        }
    }
    k_cav_velocity<T><<<g, blk, 0, s>>>((const T*)B.u[B.cu], (const T*)B.v[B.cu], (const T*)B.p[B.cp],
                                         (T*)B.u[1 - B.cu], (T*)B.v[1 - B.cu], P);
    B.cu = 1 - B.cu;
    return cudaGetLastError();
}

}  // namespace

void cavity_constants(CavityParams& P)
{
    double* c = P.c64;
    c[CV_I2DX] = 1.0 / (2.0 * P.dx);
    c[CV_I2DY] = 1.0 / (2.0 * P.dy);
    c[CV_IDT] = 1.0 / P.dt;
    c[CV_DX2] = P.dx * P.dx;
    c[CV_DY2] = P.dy * P.dy;
    c[CV_DX2DY2] = c[CV_DX2] * c[CV_DY2];
    c[CV_IPDEN] = 1.0 / (2.0 * (c[CV_DX2] + c[CV_DY2]));
    c[CV_CX] = P.dt / P.dx;
    c[CV_CY] = P.dt / P.dy;
    c[CV_DXX] = P.dt / c[CV_DX2];
    c[CV_DYY] = P.dt / c[CV_DY2];
    c[CV_GX] = P.dt / (2.0 * P.rho * P.dx);
    c[CV_GY] = P.dt / (2.0 * P.rho * P.dy);
    c[CV_RHO] = P.rho;
    c[CV_NU] = P.nu;
    c[CV_LID] = P.lid;
    for (int k = 0; k < 16; ++k) P.c32[k] = (float)c[k];
}

cudaError_t cavity_step(const CavityParams& P, CavityBufs& B, cudaStream_t s)
{
    return P.esize == 8 ? cav_step_t<double>(P, B, s) : cav_step_t<float>(P, B, s);
}

}  // namespace st
