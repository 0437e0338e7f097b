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
    int tb;           // FP32: pressure iterations in passes of several through shared memory
    // per-point constants computed once on the host in double precision and
    // also rounded to float there, so the kernels neither divide (a divide is
    // an iterative sequence on the FP64 pipe) nor convert (a double-to-float
    // conversion runs on the FP64 pipe too, 2 lanes per clock per SM here)
    double c64[16];
    float c32[16];
};

// indices into CavityParams::c64 / c32
enum CavityConst {
    CV_I2DX = 0,  // 1/(2 dx)
    CV_I2DY,      // 1/(2 dy)
    CV_IDT,       // 1/dt
    CV_DX2,       // dx^2
    CV_DY2,       // dy^2
    CV_DX2DY2,    // dx^2 dy^2
    CV_IPDEN,     // 1/(2 (dx^2 + dy^2))
    CV_CX,        // dt/dx
    CV_CY,        // dt/dy
    CV_DXX,       // dt/dx^2
    CV_DYY,       // dt/dy^2
    CV_GX,        // dt/(2 rho dx)
    CV_GY,        // dt/(2 rho dy)
    CV_RHO,
    CV_NU,
    CV_LID
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
