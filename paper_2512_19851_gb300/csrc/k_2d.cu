// 2D grids on the persistent tile kernel (k_batch.cu, a batch of one grid):
// which 2D stencils qualify, and the single-step launch used where a step
// must go from one explicit buffer to another (checkpointed forward and the
// recomputation inside the adjoint), which is the one-thread-per-point kernel.
#include "families.cuh"

namespace st {

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
