// Lid-driven cavity flow, the paper's multi-field benchmark (Sec. V-B):
// incompressible Navier-Stokes on a uniform 2D grid, one explicit time step =
// pressure source from (u, v), nit Jacobi iterations of the pressure Poisson
// equation with its boundary rule, then u and v from the old velocities and
// the new pressure with the wall and lid values.  Arrays are dense (ny, nx),
// C order, boundary rows and columns included (y along axis 0, x along
// axis 1).
//
// GB300 design: one thread per cell of the whole array, so each kernel also
// writes its boundary cells and no separate boundary pass runs:
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
// Each kernel is a gather over 5-point neighbourhoods through L1/L2; FP64 is
// bound by the FP64 pipe, FP32 by memory.
#include "cavity.cuh"

namespace st {

namespace {

__device__ __forceinline__ int64_t clampi(int64_t i, int64_t n) { return i < 1 ? 1 : (i > n - 2 ? n - 2 : i); }

template <typename T>
__global__ void __launch_bounds__(256) k_cav_source(const T* __restrict__ u, const T* __restrict__ v,
                                                    T* __restrict__ b, const __grid_constant__ CavityParams P)
{
    const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (i < 1 || j < 1 || i >= P.nx - 1 || j >= P.ny - 1) return;
    const int64_t c = j * P.nx + i;
    const T i2dx = T(P.i2dx), i2dy = T(P.i2dy);
    const T ux = (u[c + 1] - u[c - 1]) * i2dx;
    const T uy = (u[c + P.nx] - u[c - P.nx]) * i2dy;
    const T vx = (v[c + 1] - v[c - 1]) * i2dx;
    const T vy = (v[c + P.nx] - v[c - P.nx]) * i2dy;
    b[c] = T(P.rho) * ((ux + vy) * T(P.idt) - ux * ux - T(2) * uy * vx - vy * vy);
}

template <typename T>
__global__ void __launch_bounds__(256) k_cav_pressure(const T* __restrict__ pin, T* __restrict__ pout,
                                                      const T* __restrict__ b, const __grid_constant__ CavityParams P)
{
    const int64_t i = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t j = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (i >= P.nx || j >= P.ny) return;
    const int64_t o = j * P.nx + i;
    if (j == P.ny - 1) {  // the lid row: p = 0
        pout[o] = T(0);
        return;
    }
    const int64_t c = clampi(j, P.ny) * P.nx + clampi(i, P.nx);
    pout[o] = ((pin[c + 1] + pin[c - 1]) * T(P.dy2) + (pin[c + P.nx] + pin[c - P.nx]) * T(P.dx2) -
               b[c] * T(P.dx2dy2)) *
              T(P.ipden);
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
        u2[c] = T(P.lid);
        v2[c] = T(0);
        return;
    }
    if (j == 0 || i == 0 || i == P.nx - 1) {  // the walls
        u2[c] = T(0);
        v2[c] = T(0);
        return;
    }
    const T nu = T(P.nu), cx = T(P.cx), cy = T(P.cy), dxx = T(P.dxx), dyy = T(P.dyy);
    const T uc = u[c], ue = u[c + 1], uw = u[c - 1], un = u[c + P.nx], us = u[c - P.nx];
    const T vc = v[c], ve = v[c + 1], vw = v[c - 1], vn = v[c + P.nx], vs = v[c - P.nx];
    u2[c] = uc - uc * cx * (uc - uw) - vc * cy * (uc - us) - T(P.gx) * (p[c + 1] - p[c - 1]) +
            nu * (dxx * (ue - T(2) * uc + uw) + dyy * (un - T(2) * uc + us));
    v2[c] = vc - uc * cx * (vc - vw) - vc * cy * (vc - vs) - T(P.gy) * (p[c + P.nx] - p[c - P.nx]) +
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
    k_cav_source<T><<<g, blk, 0, s>>>((const T*)B.u[B.cu], (const T*)B.v[B.cu], (T*)B.b, P);
    for (int k = 0; k < P.nit; ++k) {
        k_cav_pressure<T><<<g, blk, 0, s>>>((const T*)B.p[B.cp], (T*)B.p[1 - B.cp], (const T*)B.b, P);
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
    P.i2dx = 1.0 / (2.0 * P.dx);
    P.i2dy = 1.0 / (2.0 * P.dy);
    P.idt = 1.0 / P.dt;
    P.dx2 = P.dx * P.dx;
    P.dy2 = P.dy * P.dy;
    P.dx2dy2 = P.dx2 * P.dy2;
    P.ipden = 1.0 / (2.0 * (P.dx2 + P.dy2));
    P.cx = P.dt / P.dx;
    P.cy = P.dt / P.dy;
    P.dxx = P.dt / P.dx2;
    P.dyy = P.dt / P.dy2;
    P.gx = P.dt / (2.0 * P.rho * P.dx);
    P.gy = P.dt / (2.0 * P.rho * P.dy);
}

cudaError_t cavity_step(const CavityParams& P, CavityBufs& B, cudaStream_t s)
{
    return P.esize == 8 ? cav_step_t<double>(P, B, s) : cav_step_t<float>(P, B, s);
}

}  // namespace st
