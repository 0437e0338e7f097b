// 2D tile sweeps (placeholder: no specialised kernel yet).
#include "families.cuh"

namespace st {

bool tile2d_supports(const FamilyDesc&, int*, const char**) { return false; }

cudaError_t launch_tile2d(const Family&, const SweepArgs&, cudaStream_t) { return cudaErrorNotSupported; }

}  // namespace st
