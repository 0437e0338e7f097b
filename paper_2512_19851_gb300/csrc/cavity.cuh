// Lid-driven cavity flow: parameters and buffers shared by the driver
// (api.cu) and the kernels (k_cavity.cu).
#pragma once

#include "common.cuh"

namespace st {

struct CavityParams {
    int64_t ny, nx;   // array extents, boundary rows and columns included
    double dx, dy, dt, rho, nu, lid;
    int nit;          // pressure iterations per time step
    int esize;        // 4 or 8
    // per-point constants computed once on the host in double precision, so
    // the kernels multiply instead of dividing (a divide is an iterative
    // sequence on the FP64 pipe)
    double i2dx, i2dy, idt;                 // 1/(2 dx), 1/(2 dy), 1/dt
    double dx2, dy2, dx2dy2, ipden;         // dx^2, dy^2, dx^2 dy^2, 1/(2 (dx^2 + dy^2))
    double cx, cy, dxx, dyy, gx, gy;        // dt/dx, dt/dy, dt/dx^2, dt/dy^2, dt/(2 rho dx), dt/(2 rho dy)
};

void cavity_constants(CavityParams& P);

// Two buffers per field: [0] is the caller's, [1] the handle's scratch;
// cu / cp tell which holds the current velocities / pressure.
struct CavityBufs {
    void* u[2];
    void* v[2];
    void* p[2];
    void* b;          // pressure source (scratch)
    int cu = 0, cp = 0;
};

// One time step on stream s; flips cu and, per pressure iteration, cp.
cudaError_t cavity_step(const CavityParams& P, CavityBufs& B, cudaStream_t s);

}  // namespace st
