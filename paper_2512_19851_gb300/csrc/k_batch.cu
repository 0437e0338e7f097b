// Batched form: many independent 2D grids advanced together.
// First version: one generic launch per grid and step.
#include <cstring>

#include "families.cuh"

namespace st {

BatchPlan make_batch_plan(const std::vector<Geom>& geoms, int npts, const int32_t* off2, const double* weights,
                          bool periodic, st_dtype dtype, bool force_generic)
{
    BatchPlan p;
    p.ngrids = (int)geoms.size();
    p.npts = npts;
    p.periodic = periodic;
    p.esize = dtype == ST_F64 ? 8 : 4;
    p.generic = true;
    (void)force_generic;
    p.weights.assign(weights, weights + (size_t)p.ngrids * npts);
    p.off.assign(off2, off2 + 2 * npts);
    for (int i = 0; i < p.ngrids; ++i) {
        const Geom& g = geoms[i];
        GenParams P;
        std::memset(&P, 0, sizeof(P));
        P.nz = 1;
        P.ny = g.ny;
        P.nx = g.nx;
        P.pitch = g.pitch;
        P.plane = g.plane;
        P.origin = g.origin;
        P.npts = npts;
        P.periodic = periodic ? 1 : 0;
        P.src = -1;
        for (int k = 0; k < npts; ++k) {
            P.dy[k] = off2[2 * k];
            P.dx[k] = off2[2 * k + 1];
            P.lin[k] = (int64_t)P.dy[k] * g.pitch + P.dx[k];
            P.alpha[k] = weights[(size_t)i * npts + k];
        }
        p.gp.push_back(P);
    }
    p.cfg[0] = 32;
    p.cfg[1] = 8;
    p.cfg[2] = 256;
    p.cfg[3] = 1;
    return p;
}

st_status bind_batch_plan(BatchPlan& p, const std::vector<Geom>&, void* const* a, void* const* b, int* status)
{
    p.a.assign(a, a + p.ngrids);
    p.b.assign(b, b + p.ngrids);
    p.status = status;
    return ST_OK;
}

st_status enqueue_batch_plan(BatchPlan& p, int nsteps, int cur, cudaStream_t s)
{
    for (int t = 0; t < nsteps; ++t) {
        for (int i = 0; i < p.ngrids; ++i) {
            const void* in = cur == 0 ? p.a[i] : p.b[i];
            void* out = cur == 0 ? p.b[i] : p.a[i];
            ST_CUDA_TRY(launch_generic_sweep(p.esize, in, out, nullptr, nullptr, p.gp[i], s));
        }
        cur = 1 - cur;
    }
    return ST_OK;
}

st_status tune_batch_plan(BatchPlan&, const std::vector<Geom>&, void* const*, void* const*, int, int, cudaStream_t s)
{
    ST_CUDA_TRY(cudaStreamSynchronize(s));
    return ST_OK;
}

void batch_plan_config(const BatchPlan& p, int* cfg)
{
    for (int i = 0; i < 4; ++i) cfg[i] = p.cfg[i];
}

void free_batch_plan(BatchPlan& p)
{
    if (p.d_desc) cudaFree(p.d_desc);
    if (p.d_work) cudaFree(p.d_work);
    p.d_desc = p.d_work = nullptr;
}

}  // namespace st
