// stencil_reduce_noalloc: the interior reductions of stencil_reduce without
// any device allocation.  The per-block partial sums live in a file-scope
// static __device__ array instead of handle scratch.
#include <mutex>

#include "common.cuh"

namespace st {
const Geom* grid_geom(st_grid_t g);                    // api.cu
void grid_note_stream(st_grid_t g, cudaStream_t s);   // api.cu
int* grid_status(st_grid_t g);                         // api.cu
}  // namespace st

using namespace st;

namespace {

// One partial (sum, sum of squares, max) per block and at most 4096 blocks:
// 96 KB of device memory, held by every GPU that loads the library until
// exit.  The blocks walk the interior rows in a grid-stride loop, so a grid
// of any size needs no more partials than that.
constexpr int NOALLOC_MAX_BLOCKS = 4096;
constexpr int NOALLOC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_noalloc_partials[3 * NOALLOC_MAX_BLOCKS];

std::mutex g_noalloc_mu;
double* g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the static array on the current device.  In host code the
// array's name only stands for it, so the address is looked up once per
// device, with that device current.
st_status noalloc_scratch(double** out)
{
    int dev = 0;
    ST_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
        return fail(ST_ERR_UNSUPPORTED, "stencil_reduce_noalloc: device ordinal beyond 63");
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
        if (e != cudaSuccess) return cuda_fail(e, "stencil_reduce_noalloc: cudaGetSymbolAddress");
        g_noalloc_ptr[dev] = static_cast<double*>(p);
    }
    *out = g_noalloc_ptr[dev];
    return ST_OK;
}

}  // namespace

extern "C" st_status stencil_reduce_noalloc(st_grid_t g, const void* a, const void* b, double* dev_out,
                                            void* stream)
{
    if (!g || !a || !dev_out) return fail(ST_ERR_ARG, "stencil_reduce_noalloc: NULL argument");
    if ((((uintptr_t)a) | ((uintptr_t)b)) & 15u)
        return fail(ST_ERR_ARG, "stencil_reduce_noalloc: a, b must be 16-byte aligned");
    const Geom& G = *grid_geom(g);
    double* partials = nullptr;
    st_status rc = noalloc_scratch(&partials);
    if (rc != ST_OK) return rc;
    // as many blocks as are resident at once (at most the array's 4096), the
    // grid stencil_reduce uses as well
    const int nb = reduce_blocks(G, NOALLOC_MAX_BLOCKS);
    cudaStream_t s = (cudaStream_t)stream;
    // every block overwrites its own partial, so nothing needs clearing first
    ST_CUDA_TRY(launch_reduce(G.esize, a, b, G, partials, nb, dev_out, 0, nullptr, grid_status(g), s));
    grid_note_stream(g, s);
    return ST_OK;
}
