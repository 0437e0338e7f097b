// Batched 2D sweeps: many independent grids (uneven sizes, their own
// weights, same neighbour offsets within the 3x3 neighbourhood) advanced by
// one persistent launch.
//
//  * Work list: every grid is cut into tiles of at most TW x TH points; the
//    tiles of all grids form one list, largest first, handed out dynamically
//    (an atomic counter per pass) to persistent CTAs.
//  * Temporal blocking: a pass advances k steps.  A CTA loads its tile plus a
//    k-wide halo (indices wrapped for a periodic boundary; outside points are
//    the boundary value for Dirichlet) into shared memory, runs k steps there
//    on a region that shrinks by one cell per step, and writes only the tile's
//    interior of the last step to global memory.  HBM traffic per k steps is
//    one read of tile+halo and one write, instead of k reads and k writes.
//  * One launch covers all passes: CTAs meet at a grid-wide barrier between
//    passes (cooperative launch guarantees co-residency; the wait is bounded
//    and sets ST_ERR_DEVICE_TIMEOUT if it runs out).  The barrier's
//    gpu-scope acquire orders the next pass's tile copies after the other
//    SMs' writes.  If a cooperative launch is unavailable, one launch per pass
//    is used (same arithmetic).
//  * Tiles are copied into shared memory by asynchronous element copies
//    (cp.async), so a warp keeps a whole row of loads in flight.
//  * Arithmetic order is the same as the single-grid kernels: acc = 0, then
//    acc = fma(w_k, u[p + o_k], acc) over the offsets in the given order, so a
//    grid gives bit-identical results batched or alone.
#include <algorithm>
#include <cstring>
#include <numeric>
#include <vector>

#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

constexpr int BMAXP = 9;
constexpr int SHAPE_BOX9 = 0;   // any offsets in the 3x3 neighbourhood
constexpr int SHAPE_STAR5 = 1;  // no diagonal offsets: 5 FMAs per point

struct GridDesc {
    void* a;
    void* b;
    int64_t pitch, origin;
    int ny, nx;
    double w[9];  // row-major 3x3 weight table over (dy, dx), absent offsets 0
};

struct TileDesc {
    int g, x0, y0, tw, th, pad[3];
};

struct BatchParams {
    const GridDesc* grids;
    const TileDesc* tiles;
    int ntiles;
    int nsteps, k, npasses;
    int pass0, pass1;       // passes run by this launch [pass0, pass1)
    int cur;                // slot holding the input at pass 0
    int npts;
    int dy[BMAXP], dx[BMAXP];
    int periodic;
    double bc;
    int TW, TH;             // max tile size (smem sizing)
    int row_stride;         // shared-memory row stride of a tile buffer
    unsigned* counters;     // [npasses] tile counters, [npasses] barrier arrivals
    int* status;
    unsigned long long timeout_ns;
    int barrier_extra;      // test hook: arrivals the barrier waits for beyond the grid
};

__device__ __forceinline__ int wrapn(int i, int n)
{
    if (i >= 0 && i < n) return i;
    if (i < 0 && i >= -n) return i + n;
    if (i >= n && i < 2 * n) return i - n;
    i %= n;  // halos wider than the grid
    return i < 0 ? i + n : i;
}

__device__ bool grid_barrier(unsigned* arrivals, unsigned expected, const BatchParams& P)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        __threadfence();
        atomicAdd(arrivals, 1u);
        const uint64_t t0 = ptx::globaltimer_ns();
        while (true) {
            unsigned v;
            asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(arrivals) : "memory");
            if (v >= expected) break;
            __nanosleep(200);
            if (ptx::globaltimer_ns() - t0 > P.timeout_ns) {
                atomicCAS(P.status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
                ok = 0;
                break;
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Shared tile rows: element (row ly, column lx) of a tile buffer sits at
// ly * row_stride + BPAD + lx, so 4-column groups are 16-byte aligned and the
// columns -1 and W .. W+3 exist (their values are never used by an interior
// point).
constexpr int BPAD = 4;

template <typename T>
__device__ __forceinline__ void ld6(const T* p, T (&v)[6])  // columns -1 .. 4 around a group
{
    v[0] = p[-1];
    if constexpr (sizeof(T) == 4) {
        const float4 q = *reinterpret_cast<const float4*>(p);
        v[1] = q.x;
        v[2] = q.y;
        v[3] = q.z;
        v[4] = q.w;
    } else {
        const double2 q0 = *reinterpret_cast<const double2*>(p);
        const double2 q1 = *reinterpret_cast<const double2*>(p + 2);
        v[1] = q0.x;
        v[2] = q0.y;
        v[3] = q1.x;
        v[4] = q1.y;
    }
    v[5] = p[4];
}

template <typename T>
__device__ __forceinline__ void st4(T* p, const T (&o)[4])
{
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(o[0], o[1], o[2], o[3]);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(o[0], o[1]);
        *reinterpret_cast<double2*>(p + 2) = make_double2(o[2], o[3]);
    }
}

// One pass of kp steps over one tile.
//
// Load: tile + kp-wide halo into s0, rows by warps, columns by lanes (wrapped
// for a periodic boundary, the boundary value outside a Dirichlet domain).
// Each step: threads own 4-column groups in row bands; a thread walks its
// group down its band keeping the three rows of its 3x3 window (the group and
// one column on each side) in registers, so 4 points cost one 16-byte shared
// load, two scalar ones, 36 FMAs and one 16-byte store.  Groups reach past
// the shrinking region's edge; those columns hold values that no later
// interior point reads.  The weights sit in a row-major 3x3 table (absent
// offsets 0), so the FMA order is row-major over (dy, dx): the order of the
// box offsets.
template <typename T, int SHAPE, bool PERIODIC>
__device__ void run_tile(const BatchParams& P, const TileDesc& t, int kp, int src_slot, T* s0, T* s1)
{
    const GridDesc& G = P.grids[t.g];
    const T* src = reinterpret_cast<const T*>(src_slot == 0 ? G.a : G.b) + G.origin;
    T* dst = reinterpret_cast<T*>(src_slot == 0 ? G.b : G.a) + G.origin;
    const int W = t.tw + 2 * kp, H = t.th + 2 * kp;
    const int RS = P.row_stride;
    const int nx = G.nx, ny = G.ny;
    const int64_t pitch = G.pitch;
    const T bc = T(P.bc);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int ly = warp; ly < H; ly += nwarps) {
        int gy = t.y0 - kp + ly;
        const bool yout = !PERIODIC && (gy < 0 || gy >= ny);
        if (PERIODIC) gy = wrapn(gy, ny);
        const T* srow = src + (int64_t)gy * pitch;
        T* srow_s = s0 + BPAD + ly * RS;
        // asynchronous element copies: a warp issues its whole row without
        // waiting on any load
        for (int lx = lane; lx < W; lx += 32) {
            int gx = t.x0 - kp + lx;
            if (PERIODIC) {
                gx = wrapn(gx, nx);
                ptx::cp_async_elem<sizeof(T)>(srow_s + lx, srow + gx);
            } else if (yout || gx < 0 || gx >= nx) {
                srow_s[lx] = bc;
            } else {
                ptx::cp_async_elem<sizeof(T)>(srow_s + lx, srow + gx);
            }
        }
    }
    ptx::cp_async_wait_all();
    __syncthreads();
    T w[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) w[i] = T(G.w[i]);
    const int tid = threadIdx.x, nthr = blockDim.x;
    const T* in = s0 + BPAD;
    T* out = s1 + BPAD;
    for (int j = 1; j <= kp; ++j) {
        const bool last = j == kp;
        const int c0 = j, c1 = W - j;  // region of this step: columns [c0, c1), rows [j, H - j)
        const int g0 = c0 >> 2, ng = ((c1 - 1) >> 2) - g0 + 1;
        const int nb = max(1, nthr / ng);  // row bands
        const int gi = tid % ng, band = tid / ng;
        const int rh = H - 2 * j, bh = (rh + nb - 1) / nb;
        const int r0 = j + band * bh, r1 = min(H - j, r0 + bh);
        if (band < nb && r0 < r1) {
            const int lx = (g0 + gi) * 4;  // first column of the group
            const int gx0 = t.x0 - kp + lx;
            const T* pin = in + (r0 - 1) * RS + lx;  // row above the first output row
            T A[6], B[6];
            ld6(pin, A);
            pin += RS;
            ld6(pin, B);
            pin += RS;  // row below the current output row
            // one output row from the rows above (X), at (Y) and below (Z, loaded
            // here); the row walk is unrolled by three with the window rotating
            // through A, B, C, so no register is copied
            auto row_step = [&](const T (&X)[6], const T (&Y)[6], T (&Z)[6], int ly) {
                ld6(pin, Z);
                pin += RS;
                T o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    T acc;
                    if constexpr (SHAPE == SHAPE_BOX9) {
                        acc = fma(w[0], X[e], T(0));
                        acc = fma(w[1], X[e + 1], acc);
                        acc = fma(w[2], X[e + 2], acc);
                        acc = fma(w[3], Y[e], acc);
                        acc = fma(w[4], Y[e + 1], acc);
                        acc = fma(w[5], Y[e + 2], acc);
                        acc = fma(w[6], Z[e], acc);
                        acc = fma(w[7], Z[e + 1], acc);
                        acc = fma(w[8], Z[e + 2], acc);
                    } else {  // five-point star: the corners carry no weight
                        acc = fma(w[1], X[e + 1], T(0));
                        acc = fma(w[3], Y[e], acc);
                        acc = fma(w[4], Y[e + 1], acc);
                        acc = fma(w[5], Y[e + 2], acc);
                        acc = fma(w[7], Z[e + 1], acc);
                    }
                    o[e] = acc;
                }
                if (!last) {
                    if (!PERIODIC) {  // ghost points of the halo stay fixed
                        const int gy = t.y0 - kp + ly;
                        const bool yo = gy < 0 || gy >= ny;
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (yo || gx0 + e < 0 || gx0 + e >= nx) o[e] = bc;
                    }
                    st4(out + ly * RS + lx, o);
                } else {  // last step: the region is the tile interior, written to global memory
                    T* po = dst + (int64_t)(t.y0 - kp + ly) * pitch + gx0;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (lx + e >= c0 && lx + e < c1) po[e] = o[e];
                }
            };
            T C[6];
            int ly = r0;
            for (; ly + 3 <= r1; ly += 3) {
                row_step(A, B, C, ly);
                row_step(B, C, A, ly + 1);
                row_step(C, A, B, ly + 2);
            }
            if (ly < r1) row_step(A, B, C, ly);
            if (ly + 1 < r1) row_step(B, C, A, ly + 1);
        }
        __syncthreads();
        const T* tmp = in;
        in = out;
        out = const_cast<T*>(tmp);
    }
}

template <typename T, int SHAPE, bool PERIODIC>
__global__ void k_batch(const __grid_constant__ BatchParams P)
{
    // one launch per pass: the previous pass wrote this pass's input
    ptx::griddep_wait();
    ptx::griddep_trigger();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s0 = reinterpret_cast<T*>(smem_raw);
    T* s1 = s0 + (size_t)(P.TH + 2 * P.k) * P.row_stride;
    __shared__ int s_tile;
    for (int p = P.pass0; p < P.pass1; ++p) {
        const int kp = min(P.k, P.nsteps - p * P.k);
        const int src_slot = P.cur ^ (p & 1);
        unsigned* ctr = P.counters + p;
        while (true) {
            __syncthreads();
            if (threadIdx.x == 0) s_tile = (int)atomicAdd(ctr, 1u);
            __syncthreads();
            const int ti = s_tile;
            if (ti >= P.ntiles) break;
            const TileDesc t = P.tiles[ti];
            run_tile<T, SHAPE, PERIODIC>(P, t, kp, src_slot, s0, s1);
        }
        if (p + 1 < P.pass1) {
            const unsigned expected = gridDim.x + (unsigned)P.barrier_extra;
            if (!grid_barrier(P.counters + P.npasses + p, expected, P)) return;
        }
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
namespace {

struct Candidate {
    int TW, TH, threads, k;
};

int batch_sm_count()
{
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    return n;
}

size_t tile_smem(int TW, int TH, int k, int esize, int* row_stride)
{
    // BPAD columns before a row and at least 4 after it, 16-byte multiple
    const int rs = (TW + 2 * k + 8 + 3) / 4 * 4;
    *row_stride = rs;
    return (size_t)2 * (TH + 2 * k) * rs * esize;
}

void build_tiles(const BatchPlan& p, const std::vector<int>& ny, const std::vector<int>& nx, int TW, int TH,
                 std::vector<TileDesc>& out)
{
    out.clear();
    // equal tiles per grid (no thin slivers at the edges): each extent is
    // split into ceil(n / T) nearly equal parts of at most T points
    for (int g = 0; g < p.ngrids; ++g) {
        const int cx = (nx[g] + TW - 1) / TW, cy = (ny[g] + TH - 1) / TH;
        for (int iy = 0; iy < cy; ++iy)
            for (int ix = 0; ix < cx; ++ix) {
                TileDesc t{};
                t.g = g;
                t.x0 = (int)((int64_t)nx[g] * ix / cx);
                t.y0 = (int)((int64_t)ny[g] * iy / cy);
                t.tw = (int)((int64_t)nx[g] * (ix + 1) / cx) - t.x0;
                t.th = (int)((int64_t)ny[g] * (iy + 1) / cy) - t.y0;
                out.push_back(t);
            }
    }
    std::stable_sort(out.begin(), out.end(),
                     [](const TileDesc& a, const TileDesc& b) { return a.tw * a.th > b.tw * b.th; });
}

}  // namespace

struct BatchDev {
    GridDesc* grids = nullptr;
    TileDesc* tiles = nullptr;
    unsigned* counters = nullptr;
    int ncounters = 0;
    std::vector<int> ny, nx;
    bool coop_ok = true;
};

static BatchDev* dev_of(BatchPlan& p) { return reinterpret_cast<BatchDev*>(p.d_desc); }

BatchPlan make_batch_plan(const std::vector<Geom>& geoms, int npts, const int32_t* off2, const double* weights,
                          bool periodic, st_dtype dtype, bool force_generic)
{
    BatchPlan p;
    p.ngrids = (int)geoms.size();
    p.npts = npts;
    p.periodic = periodic;
    p.esize = dtype == ST_F64 ? 8 : 4;
    p.weights.assign(weights, weights + (size_t)p.ngrids * npts);
    p.off.assign(off2, off2 + 2 * npts);
    bool small = npts <= BMAXP;
    for (int k = 0; k < 2 * npts; ++k)
        if (off2[k] < -1 || off2[k] > 1) small = false;
    p.generic = force_generic || !small;
    p.shape = SHAPE_STAR5;
    for (int k = 0; k < npts; ++k)
        if (off2[2 * k] != 0 && off2[2 * k + 1] != 0) p.shape = SHAPE_BOX9;
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
        gen_params_floats(P);
        p.gp.push_back(P);
    }
    // default configuration (tile 128 x 32, 256 threads, 5 steps per pass)
    p.cfg[0] = 128;
    p.cfg[1] = 32;
    p.cfg[2] = 256;
    p.cfg[3] = 5;
    if (p.generic) {
        p.cfg[0] = 32;
        p.cfg[1] = 8;
        p.cfg[2] = 256;
        p.cfg[3] = 1;
    }
    BatchDev* d = new BatchDev();
    for (const Geom& g : geoms) {
        d->ny.push_back((int)g.ny);
        d->nx.push_back((int)g.nx);
    }
    p.d_desc = d;
    return p;
}

static st_status upload_tiles(BatchPlan& p, int TW, int TH)
{
    BatchDev* d = dev_of(p);
    std::vector<TileDesc> tiles;
    build_tiles(p, d->ny, d->nx, TW, TH, tiles);
    if (d->tiles) cudaFree(d->tiles);
    d->tiles = nullptr;
    if (cudaMalloc(&d->tiles, sizeof(TileDesc) * tiles.size()) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ST_ERR_OOM, "batch: tile table allocation failed");
    }
    ST_CUDA_TRY(cudaMemcpy(d->tiles, tiles.data(), sizeof(TileDesc) * tiles.size(), cudaMemcpyHostToDevice));
    p.nwork = (int)tiles.size();
    return ST_OK;
}

st_status bind_batch_plan(BatchPlan& p, const std::vector<Geom>& geoms, void* const* a, void* const* b, int* status)
{
    p.a.assign(a, a + p.ngrids);
    p.b.assign(b, b + p.ngrids);
    p.status = status;
    p.nsm = batch_sm_count();
    if (p.generic) return ST_OK;
    BatchDev* d = dev_of(p);
    std::vector<GridDesc> gd(p.ngrids);
    for (int i = 0; i < p.ngrids; ++i) {
        std::memset(&gd[i], 0, sizeof(GridDesc));
        gd[i].a = a[i];
        gd[i].b = b[i];
        gd[i].pitch = geoms[i].pitch;
        gd[i].origin = geoms[i].origin;
        gd[i].ny = (int)geoms[i].ny;
        gd[i].nx = (int)geoms[i].nx;
        for (int k = 0; k < p.npts; ++k) {
            const int cell = (p.off[2 * k] + 1) * 3 + (p.off[2 * k + 1] + 1);
            gd[i].w[cell] += p.weights[(size_t)i * p.npts + k];
        }
    }
    if (d->grids) cudaFree(d->grids);
    d->grids = nullptr;
    if (cudaMalloc(&d->grids, sizeof(GridDesc) * p.ngrids) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ST_ERR_OOM, "batch: descriptor allocation failed");
    }
    ST_CUDA_TRY(cudaMemcpy(d->grids, gd.data(), sizeof(GridDesc) * p.ngrids, cudaMemcpyHostToDevice));
    return upload_tiles(p, p.cfg[0], p.cfg[1]);
}

static st_status ensure_counters(BatchDev* d, int n)
{
    if (d->ncounters >= n) return ST_OK;
    if (d->counters) cudaFree(d->counters);
    d->counters = nullptr;
    d->ncounters = 0;
    if (cudaMalloc(&d->counters, sizeof(unsigned) * n) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ST_ERR_OOM, "batch: counter allocation failed");
    }
    d->ncounters = n;
    return ST_OK;
}

// Enqueue nsteps with the plan's configuration.  coop: one cooperative launch
// for all passes; otherwise one launch per pass.  barrier_extra/timeout are
// test hooks (0 / 2 s in normal use).
static st_status enqueue_tiled(BatchPlan& p, int nsteps, int cur, cudaStream_t s, bool coop, int barrier_extra,
                               unsigned long long timeout_ns)
{
    BatchDev* d = dev_of(p);
    const int TW = p.cfg[0], TH = p.cfg[1], threads = p.cfg[2], k = p.cfg[3];
    const int npasses = (nsteps + k - 1) / k;
    // counters must exist before any capture starts (stencil_batch_tune or bind allocate enough)
    if (d->ncounters < 2 * npasses) return fail(ST_ERR_STATE, "batch: counters not reserved for this step count");
    BatchParams P;
    std::memset(&P, 0, sizeof(P));
    P.grids = d->grids;
    P.tiles = d->tiles;
    P.ntiles = p.nwork;
    P.nsteps = nsteps;
    P.k = k;
    P.npasses = npasses;
    P.cur = cur;
    P.npts = p.npts;
    for (int i = 0; i < p.npts; ++i) {
        P.dy[i] = p.off[2 * i];
        P.dx[i] = p.off[2 * i + 1];
    }
    P.periodic = p.periodic ? 1 : 0;
    P.bc = p.bc;
    P.TW = TW;
    P.TH = TH;
    const size_t smem = tile_smem(TW, TH, k, p.esize, &P.row_stride);
    P.counters = d->counters;
    P.status = p.status;
    P.timeout_ns = timeout_ns;
    P.barrier_extra = barrier_extra;
    ST_CUDA_TRY(cudaMemsetAsync(d->counters, 0, sizeof(unsigned) * 2 * npasses, s));
    typedef void (*KFn)(const BatchParams);
    static const KFn table[2][2][2] = {  // [double][star][periodic]
        {{k_batch<float, SHAPE_BOX9, false>, k_batch<float, SHAPE_BOX9, true>},
         {k_batch<float, SHAPE_STAR5, false>, k_batch<float, SHAPE_STAR5, true>}},
        {{k_batch<double, SHAPE_BOX9, false>, k_batch<double, SHAPE_BOX9, true>},
         {k_batch<double, SHAPE_STAR5, false>, k_batch<double, SHAPE_STAR5, true>}}};
    const KFn kf = table[p.esize == 8][p.shape == SHAPE_STAR5][p.periodic ? 1 : 0];
    const void* fn = (const void*)kf;
    ST_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    if (coop && d->coop_ok) {
        int per_sm = 0;
        ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
        if (per_sm < 1) return fail(ST_ERR_UNSUPPORTED, "batch: tile configuration does not fit an SM");
        const int grid = std::min(per_sm * p.nsm, std::max(1, p.nwork));
        P.pass0 = 0;
        P.pass1 = npasses;
        cudaLaunchConfig_t lc{};
        lc.gridDim = dim3(grid);
        lc.blockDim = dim3(threads);
        lc.dynamicSmemBytes = smem;
        lc.stream = s;
        cudaLaunchAttribute at[1];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        lc.attrs = at;
        lc.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&lc, kf, P);
        if (e == cudaSuccess) return ST_OK;
        return cuda_fail(e, "batch cooperative launch");
    }
    int per_sm = 0;
    ST_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
    const int grid = std::min(std::max(1, per_sm) * p.nsm, std::max(1, p.nwork));
    for (int pass = 0; pass < npasses; ++pass) {
        P.pass0 = pass;
        P.pass1 = pass + 1;
        ST_CUDA_TRY(launch_dependent(kf, dim3(grid), dim3(threads), smem, s, P));
    }
    return ST_OK;
}

int batch_final_slot(const BatchPlan& p, int nsteps, int cur)
{
    if (p.generic) return (nsteps & 1) ? 1 - cur : cur;
    const int npasses = (nsteps + p.cfg[3] - 1) / p.cfg[3];
    return (npasses & 1) ? 1 - cur : cur;
}

st_status reserve_batch_steps(BatchPlan& p, int nsteps, bool* moved)
{
    *moved = false;
    if (p.generic) return ST_OK;
    BatchDev* d = dev_of(p);
    // one step per pass is the most passes any configuration uses; reserve a
    // generous table so that it rarely moves (captured graphs point into it)
    const int need = 2 * std::max(2, nsteps);
    if (d->ncounters >= need) return ST_OK;
    *moved = d->ncounters > 0;
    return ensure_counters(d, std::max(need, 2 * 1024));
}

void batch_disable_coop(BatchPlan& p)
{
    if (dev_of(p)) dev_of(p)->coop_ok = false;
}

st_status enqueue_batch_plan(BatchPlan& p, int nsteps, int cur, cudaStream_t s)
{
    if (!p.generic) return enqueue_tiled(p, nsteps, cur, s, p.cfg[3] > 0 && dev_of(p)->coop_ok, 0, 2000000000ull);
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

st_status batch_barrier_selftest(BatchPlan& p, int cur, cudaStream_t s, unsigned long long timeout_ns)
{
    if (p.generic) return fail(ST_ERR_UNSUPPORTED, "batch: no barrier in the generic plan");
    st_status rc = ensure_counters(dev_of(p), 4);
    if (rc != ST_OK) return rc;
    const int saved = p.cfg[3];
    p.cfg[3] = 1;
    rc = enqueue_tiled(p, 2, cur, s, true, 1, timeout_ns);
    p.cfg[3] = saved;
    return rc;
}

st_status tune_batch_plan(BatchPlan& p, const std::vector<Geom>& geoms, void* const* a, void* const* b, int nsteps,
                          int cur, cudaStream_t s)
{
    if (p.generic) {
        ST_CUDA_TRY(cudaStreamSynchronize(s));
        return ST_OK;
    }
    BatchDev* d = dev_of(p);
    st_status rc = ensure_counters(d, 2 * std::max(1, nsteps));
    if (rc != ST_OK) return rc;
    // back up the inputs of every grid (restored after tuning)
    std::vector<size_t> bytes(p.ngrids);
    size_t total = 0;
    for (int i = 0; i < p.ngrids; ++i) {
        bytes[i] = (size_t)geoms[i].elems * geoms[i].esize;
        total += (bytes[i] + 255) / 256 * 256;
    }
    char* backup = nullptr;
    if (cudaMalloc(&backup, total) != cudaSuccess) {
        (void)cudaGetLastError();
        return fail(ST_ERR_OOM, "stencil_batch_tune: backup allocation failed");
    }
    auto copy_all = [&](bool save) -> st_status {
        size_t off = 0;
        for (int i = 0; i < p.ngrids; ++i) {
            void* live = cur == 0 ? a[i] : b[i];
            if (save)
                ST_CUDA_TRY(cudaMemcpyAsync(backup + off, live, bytes[i], cudaMemcpyDeviceToDevice, s));
            else
                ST_CUDA_TRY(cudaMemcpyAsync(live, backup + off, bytes[i], cudaMemcpyDeviceToDevice, s));
            off += (bytes[i] + 255) / 256 * 256;
        }
        return ST_OK;
    };
    rc = copy_all(true);
    if (rc != ST_OK) {
        cudaFree(backup);
        return rc;
    }
    std::vector<Candidate> cands;
    // tile shapes from small (single grids, many SMs) to wide (big grids)
    const int tiles[][2] = {{32, 8}, {32, 16}, {64, 16}, {128, 16}, {128, 32}, {256, 16}, {64, 64}};
    const int ks[] = {1, 2, 4, 6, 10};
    for (auto& t : tiles)
        for (int k : ks)
            for (int th : {128, 256}) {
                int rs;
                if (tile_smem(t[0], t[1], k, p.esize, &rs) > 200 * 1024) continue;
                cands.push_back(Candidate{t[0], t[1], th, k});
            }
    cudaEvent_t e0, e1;
    ST_CUDA_TRY(cudaEventCreate(&e0));
    ST_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestc[4] = {p.cfg[0], p.cfg[1], p.cfg[2], p.cfg[3]};
    int curTW = p.cfg[0], curTH = p.cfg[1];
    for (const Candidate& c : cands) {
        if (c.TW != curTW || c.TH != curTH) {
            rc = upload_tiles(p, c.TW, c.TH);
            if (rc != ST_OK) break;
            curTW = c.TW;
            curTH = c.TH;
        }
        p.cfg[0] = c.TW;
        p.cfg[1] = c.TH;
        p.cfg[2] = c.threads;
        p.cfg[3] = c.k;
        float ms_best = 1e30f;
        bool ok = true;
        for (int rep = 0; rep < 2 && ok; ++rep) {
            ST_CUDA_TRY(cudaEventRecord(e0, s));
            if (enqueue_tiled(p, nsteps, cur, s, true, 0, 2000000000ull) != ST_OK) {
                (void)cudaGetLastError();
                ok = false;
                break;
            }
            ST_CUDA_TRY(cudaEventRecord(e1, s));
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                ok = false;
                break;
            }
            float ms = 0;
            cudaEventElapsedTime(&ms, e0, e1);
            ms_best = std::min(ms_best, ms);
            // trials advance the data; run time does not depend on the values,
            // so the inputs are restored once, after the last trial
        }
        if (rc != ST_OK) break;
        if (ok && ms_best < best) {
            best = ms_best;
            bestc[0] = c.TW;
            bestc[1] = c.TH;
            bestc[2] = c.threads;
            bestc[3] = c.k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    st_status rc2 = copy_all(false);
    ST_CUDA_TRY(cudaStreamSynchronize(s));
    cudaFree(backup);
    if (rc != ST_OK) return rc;
    if (rc2 != ST_OK) return rc2;
    p.cfg[0] = bestc[0];
    p.cfg[1] = bestc[1];
    p.cfg[2] = bestc[2];
    p.cfg[3] = bestc[3];
    int st_code = 0;
    ST_CUDA_TRY(cudaMemcpy(&st_code, p.status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st_code != 0) return fail(ST_ERR_DEVICE_TIMEOUT, "stencil_batch_tune: a candidate timed out");
    return upload_tiles(p, p.cfg[0], p.cfg[1]);
}

void batch_plan_config(const BatchPlan& p, int* cfg)
{
    for (int i = 0; i < 4; ++i) cfg[i] = p.cfg[i];
}

void free_batch_plan(BatchPlan& p)
{
    BatchDev* d = dev_of(p);
    if (d) {
        if (d->grids) cudaFree(d->grids);
        if (d->tiles) cudaFree(d->tiles);
        if (d->counters) cudaFree(d->counters);
        delete d;
    }
    p.d_desc = nullptr;
}

}  // namespace st
