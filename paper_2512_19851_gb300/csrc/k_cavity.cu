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
    for (int k = 0; k < P.nit; ++k) {
        k_cav_pressure<T><<<gp, 256, 0, s>>>((const T*)B.p[B.cp], (T*)B.p[1 - B.cp], (const T*)B.b, P);
        B.cp = 1 - B.cp;
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
