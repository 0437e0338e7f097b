// Transpose (adjoint) sweep of the per-cell 7-point operator with K = 1 or 2
// steps fused per pass, plus the coefficient gradient (the backward pass of
// the variable-coefficient diffusion, Sec. 4 of the paper's stencil model
// differentiated by hand).
//
// Operator (symmetric star, one coefficient field):
//   w_c(p) = ac + bc kappa_p,  w_n(p) = an + bn kappa_p for all six neighbours.
// With mu = w_n * lambda_in, one transposed step lambda_in -> lambda_out is
//   lambda_out[q] = w_c(q) lambda_in[q] + sum over the six neighbours p of q of mu[p]
// (a constant-weight 7-point sum of mu plus a pointwise centre term), and the
// gradient term of that step is
//   g[q] += lambda_in[q] * (bc u_t[q] + bn * sum over the neighbours of u_t).
//
// Design (HBM-bound; two fused steps halve the lambda, kappa and gradient
// traffic per step):
//  * A unit is TY full rows streamed through a range of z planes; each CTA
//    takes an equal share of all (tile, plane) pairs, in tile-major order, as
//    one or more units.  A producer warp stages, per plane, lambda and kappa with a K-row y halo and
//    the states u_t (and u_{t-1}, one plane behind) with a 1-row halo into a
//    ring of NS stages by 1D bulk copies completing on mbarriers.  Only two
//    stages are read at a time (the centre plane and the plane above); the
//    rest are in flight.
//  * Consumer threads own fixed tasks: a pair of rows at one 16-byte x group.
//    The plane below lives in registers (z reuse), the pair shares its inner
//    y neighbours, x edges come from the neighbouring lanes by shuffles (from
//    shared memory at warp and row ends).
//  * Time skew (K = 2): at iteration j stage j has arrived, level 1 computes
//    the plane of stage j - 1 and level 2 the plane below it.  Level 1 runs on
//    the tile rows plus one halo row on each side (computed by halo warps) and
//    publishes its mu in a 3-plane shared ring; level 2 reads the ring for its
//    outer y neighbours and keeps everything else in registers.
//  * Outside the interior (Dirichlet) every level is 0 by selection, never by
//    arithmetic on ghost data: ghosts are boundary data, not variables.
//  * Each fused level evaluates exactly the expressions of a single-step pass
//    in the same order, so lambda rounds exactly like K single-step passes.
//    A single-step pass sends its gradient term of a point once; a fused
//    pass holds level 1's term of a plane in registers until level 2 reaches
//    that plane one iteration later and sends the two terms' sum (in T)
//    once, which halves the gradient traffic and shared-memory transposes.
//    FP64 grids send it to the FP64 gradient by reductions performed at L2
//    (the SMs never wait on them).  FP32 grids sum a checkpoint segment's
//    terms in an FP32 partial gradient, added to the FP64 gradient once per
//    segment (put_grad, k_grad_flush): the FP64 accumulation and its
//    conversions run once per segment rather than once per pass.  The gradient then depends on
//    how the steps are paired into passes (pairs are taken from the top of
//    each checkpoint segment) and, in FP32, on the segment length, by
//    roundings of T.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

// At most 12 warps per block (3 per SM sub-partition) leave 168 registers a
// thread for the carried planes.
constexpr int A_MAXCW = 11;                     // consumer warps at most
constexpr int A_BLOCK = (A_MAXCW + 1) * 32;     // + the producer warp
constexpr int A_RING = 3;                       // planes in the level-1 mu ring

struct AdjParams {
    int64_t nz, ny, nx, pitch, plane, origin;
    int rz, r, xl;
    int TY, NS, CW;                 // rows per tile, stages, consumer warps
    int nyt, nzc, units;
    int flat;                       // 1, 2: CTA b takes a contiguous range of the tile-major sequence
                                    // of the nyt * nz (tile, plane) pairs (UnitIter)
    int ngx, npair, pair_warps;     // row-pair tasks fill warps [0, pair_warps); halo row tasks the rest
    int halo_warps;                 // K == 2: halo warps; each covers x groups [32 w, 32 w + 32) and,
                                    // one warp count further, [32 (w + halo_warps), ...)
    uint32_t stage_elems, kap_off, ua_off, ub_off;  // lambda at offset 0 of a stage
    uint32_t ring_elems;            // one plane of the mu ring: TY + 2 rows
    int grad;                       // gradient requested
    int gfirst;                     // FP32 grids: the first pass of a checkpoint segment
    double ac, bc, an, bn;
    int* status;
};

template <typename T>
struct AV;
template <>
struct AV<float> {
    static constexpr int N = 4;
    typedef float4 type;
};
template <>
struct AV<double> {
    static constexpr int N = 2;
    typedef double2 type;
};

template <typename T>
__device__ __forceinline__ void vld(const T* p, T (&v)[AV<T>::N])
{
    const typename AV<T>::type t = *reinterpret_cast<const typename AV<T>::type*>(p);
    if constexpr (AV<T>::N == 4) {
        v[0] = t.x;
        v[1] = t.y;
        v[2] = t.z;
        v[3] = t.w;
    } else {
        v[0] = t.x;
        v[1] = t.y;
    }
}

template <typename T>
__device__ __forceinline__ void vst(T* p, const T (&v)[AV<T>::N])
{
    typename AV<T>::type t;
    if constexpr (AV<T>::N == 4) {
        t.x = v[0];
        t.y = v[1];
        t.z = v[2];
        t.w = v[3];
    } else {
        t.x = v[0];
        t.y = v[1];
    }
    *reinterpret_cast<typename AV<T>::type*>(p) = t;
}

__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }

__device__ __forceinline__ int64_t amin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t amax(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ void atimeout(int* status)
{
    if (status) atomicCAS(status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
}

// Flat mode: position in the tile-major sequence of (tile, plane) pairs of
// the point v of a cost axis on which every tile takes nz + w units, its
// first w standing for the w warm-up iterations a unit starting there costs.
__host__ __device__ __forceinline__ uint32_t flat_cut(uint64_t v, uint32_t nz, uint32_t nyt, uint32_t w)
{
    const uint64_t per = (uint64_t)nz + w;
    const uint64_t t = v / per;
    if (t >= nyt) return nyt * nz;
    const int64_t in = (int64_t)(v - t * per) - (int64_t)w;
    return (uint32_t)(t * nz + (in < 0 ? 0 : (uint64_t)in));
}

// The units of this CTA in order: a y tile and a z range [z0, z1).  Flat
// mode needs nyt * (nz + 2K) < 2^31 (checked on the host).
template <int K>
struct UnitIter {
    uint32_t a, b;  // flat: next and end (tile, plane) pair of this CTA; otherwise a = unit index
    __device__ UnitIter(const AdjParams& P)
    {
        if (P.flat) {
            // flat == 2: equal shares of the cost axis, so that a CTA whose
            // range crosses into the next tile, and pays a second pipeline
            // warm-up (2K iterations), gets correspondingly fewer planes;
            // flat == 1: equal shares of planes (the host picks the one whose
            // longest CTA is shorter)
            const uint32_t nz = (uint32_t)P.nz, nyt = (uint32_t)P.nyt, w = P.flat == 2 ? 2 * K : 0;
            const uint64_t V = (uint64_t)nyt * (nz + w);
            a = flat_cut(V * blockIdx.x / gridDim.x, nz, nyt, w);
            b = flat_cut(V * (blockIdx.x + 1) / gridDim.x, nz, nyt, w);
        } else {
            a = blockIdx.x;
            b = 0;
        }
    }
    __device__ bool next(const AdjParams& P, int& yt, int64_t& z0, int64_t& z1)
    {
        if (P.flat) {
            if (a >= b) return false;
            const uint32_t nz = (uint32_t)P.nz;
            yt = (int)(a / nz);
            const uint32_t zs = a - (uint32_t)yt * nz;
            const uint32_t ze = min(nz, zs + (b - a));
            z0 = zs;
            z1 = ze;
            a += ze - zs;
            return true;
        }
        if (a >= (uint32_t)P.units) return false;
        yt = (int)(a % (uint32_t)P.nyt);
        const int zc = (int)(a / (uint32_t)P.nyt);
        z0 = (int64_t)zc * P.nz / P.nzc;
        z1 = (int64_t)(zc + 1) * P.nz / P.nzc;
        a += gridDim.x;
        return true;
    }
};

// Per-thread constants of the x group a task owns.
struct XCtx {
    int x;        // first column of the group
    int cl, cr;   // columns of the left neighbour of element 0 and the right one of element VN-1
    int nx;
    bool fixl, fixr;  // that neighbour is not held by the adjacent lane
    bool wig;         // periodic row end inside the group: element nx-1-x wraps to column 0
    bool xfull;       // the whole group is interior
    // columns each lane loads for the x edges, unconditionally: its own cl / cr
    // where fixl / fixr, else those of lane 0 / lane 31, so that one broadcast
    // access serves the warp and no edge load needs a branch
    int lcl, lcr;
};

// The context of x group gx for this lane.  All lanes of the warp must call it.
template <int VN, bool PERIODIC>
__device__ __forceinline__ XCtx make_xctx(int gx, int lane, int ngx, int nx)
{
    XCtx X;
    X.nx = nx;
    X.x = gx * VN;
    X.fixl = lane == 0 || gx == 0;
    X.fixr = lane == 31 || gx == ngx - 1;
    X.wig = PERIODIC && X.x + VN > X.nx;
    X.cl = X.x > 0 ? X.x - 1 : (PERIODIC ? X.nx - 1 : -1);
    // (a Dirichlet ragged group reads the ghost column instead: its last
    // elements are not interior and their results are dropped)
    X.cr = X.x + VN >= X.nx ? (PERIODIC ? 0 : X.nx) : X.x + VN;
    X.xfull = X.x + VN <= X.nx;
    const int cl0 = __shfl_sync(0xffffffffu, X.cl, 0), cr31 = __shfl_sync(0xffffffffu, X.cr, 31);
    X.lcl = X.fixl ? X.cl : cl0;
    X.lcr = X.fixr ? X.cr : cr31;
    return X;
}

// Neighbour sum of one row of values v in the fixed order
//   z-1, y-1, y+1, x-1, x+1, z+1
// shared by every level and every pass.  `left`/`right` are the values at
// columns X.lcl / X.lcr; they are used where X.fixl / X.fixr, otherwise the
// edge values come from the adjacent lanes.  All lanes of the warp must call it.
template <typename T>
__device__ __forceinline__ void nsum(const XCtx& X, const T (&zm)[AV<T>::N], const T (&ym)[AV<T>::N],
                                     const T (&v)[AV<T>::N], const T (&yp)[AV<T>::N], const T (&zp)[AV<T>::N],
                                     T left, T right, T (&s)[AV<T>::N])
{
    constexpr int VN = AV<T>::N;
    const T l = __shfl_up_sync(0xffffffffu, v[VN - 1], 1);
    const T r = __shfl_down_sync(0xffffffffu, v[0], 1);
    left = X.fixl ? left : l;
    right = X.fixr ? right : r;
#pragma unroll
    for (int e = 0; e < VN; ++e) {
        const T xm = e == 0 ? left : v[e - 1];
        T xp = e == VN - 1 ? right : v[e + 1];
        if (X.wig && X.x + e + 1 == X.nx) xp = right;
        s[e] = ((((zm[e] + ym[e]) + yp[e]) + xm) + xp) + zp[e];
    }
}

// One point's gradient term (or pair of terms) of a pass.  FP64 grids add it
// to the FP64 gradient by a reduction performed at L2.  FP32 grids keep the
// terms of a checkpoint segment in an FP32 partial gradient (64 MB at 256^3;
// no FP64 instruction runs for it on the SM): the segment's first pass
// stores its term there (`first`, the same for the whole launch), the
// others add theirs by L2 reductions, and k_grad_flush adds the partial to
// the FP64 gradient after the segment's last pass.  No thread waits on any
// of these accesses.
template <typename T>
__device__ __forceinline__ void put_grad(T* __restrict__ gacc, bool first, int64_t i, T v)
{
    if (sizeof(T) == 4 && first) gacc[i] = v;
    else atomicAdd(gacc + i, v);
}

// Add one step's gradient terms of a row group (see put_grad).  FP32: a
// whole group goes out as one 16-byte store or vector reduction.  FP64:
// when the warp's 32 lanes hold 32 consecutive whole groups of one row
// (`fast`, warp-uniform) the terms are first exchanged through the warp's
// shared scratch so that each reduction instruction covers 32 consecutive
// doubles (8 sectors instead of 32).  Either way a point's terms all come
// from one thread, in step order, and same-thread accesses to one address
// take effect in program order, so every point sums its terms (or pairs of
// terms) in step order.
template <typename T>
__device__ __forceinline__ void add_grad(const XCtx& X, bool fast, T* wsc, int lane, int64_t off, bool ok,
                                         T* __restrict__ gacc, bool first, const T (&t)[AV<T>::N])
{
    constexpr int VN = AV<T>::N;
    if constexpr (sizeof(T) == 4) {
        if (ok && X.xfull) {
            if (first) vst(gacc + off, t);
            else ptx::red_add_v4(gacc + off, t[0], t[1], t[2], t[3]);
        } else if (ok) {
#pragma unroll
            for (int e = 0; e < VN; ++e)
                if (X.x + e < X.nx) put_grad(gacc, first, off + e, t[e]);
        }
        return;
    }
    if (fast) {
        const int64_t base = __shfl_sync(0xffffffffu, off, 0);
#pragma unroll
        for (int e = 0; e < VN; ++e) wsc[VN * lane + e] = t[e];
        __syncwarp();
#pragma unroll
        for (int e = 0; e < VN; ++e) put_grad(gacc, first, base + lane + 32 * e, wsc[lane + 32 * e]);
        __syncwarp();
    } else if (ok) {
#pragma unroll
        for (int e = 0; e < VN; ++e)
            if (X.xfull || X.x + e < X.nx) put_grad(gacc, first, off + e, t[e]);
    }
}

template <typename T>
__device__ __forceinline__ void store_row(const XCtx& X, T* p, const T (&v)[AV<T>::N])
{
    if (X.xfull) {
        vst(p, v);
    } else {
        for (int e = 0; e < AV<T>::N && X.x + e < X.nx; ++e) p[e] = v[e];  // columns past nx stay untouched
    }
}

// Store the two rows of a row-pair task (row i at p + i * stride).  `okw`
// (warp-uniform) says every lane's group is whole and both rows are in the
// tile, so the warp stores without per-lane checks.
template <typename T>
__device__ __forceinline__ void store_pair(bool okw, const XCtx& X, bool act, int rr0, int tye, T* p, int64_t stride,
                                           const T (&v)[2][AV<T>::N])
{
    if (okw) {
        vst(p, v[0]);
        vst(p + stride, v[1]);
    } else {
#pragma unroll
        for (int i = 0; i < 2; ++i)
            if (act && rr0 + i < tye) store_row(X, p + i * stride, v[i]);
    }
}

// UNIT: the neighbour weight is the coefficient itself (an = 0, bn = 1, the
// variable-diffusivity operator), so mu = kappa * lambda and the gradient's
// neighbour sum needs no scaling; the results are the same bits as the
// general expressions give for those weights (fma(1, k, 0) = k, 1 * s = s).
template <typename T, int K, bool PERIODIC, bool UNIT>
__global__ void __launch_bounds__(A_BLOCK, 1)
k_adjoint(const T* __restrict__ lam_in, T* __restrict__ lam_out, const T* __restrict__ kappa,
          const T* __restrict__ ua, const T* __restrict__ ub, T* __restrict__ g64,
          const __grid_constant__ AdjParams P)
{
    constexpr int VN = AV<T>::N;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* stg = reinterpret_cast<T*>(smem_raw);
    T* mring = stg + (size_t)P.NS * P.stage_elems;
    uint64_t* full = reinterpret_cast<uint64_t*>(mring + (K == 2 ? (size_t)A_RING * P.ring_elems : 0));
    uint64_t* empty = full + P.NS;
    uint64_t* rfull = empty + P.NS;    // K == 2: a ring plane is written (one arrival per consumer warp)
    uint64_t* rempty = rfull + A_RING;  // K == 2: a ring plane is read
    // per consumer warp: 32 x VN gradient terms in transit
    T* wscr = reinterpret_cast<T*>(rempty + A_RING) + (size_t)(threadIdx.x >> 5) * 32 * AV<T>::N;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.NS; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], P.CW);
        }
        if (K == 2)
            for (int s = 0; s < A_RING; ++s) {
                ptx::mbar_init(&rfull[s], P.CW);
                ptx::mbar_init(&rempty[s], P.CW);
            }
        ptx::fence_barrier_init();
    }
    // the ring's ghost columns stay 0 for good (only interior columns are written)
    if (K == 2)
        for (size_t i = threadIdx.x; i < (size_t)A_RING * P.ring_elems; i += blockDim.x) mring[i] = T(0);
    __syncthreads();
    ptx::griddep_wait();  // earlier kernels of the stream wrote our inputs / read our outputs
    ptx::griddep_trigger();
    const uint32_t rowb = (uint32_t)(P.pitch * sizeof(T));
    const bool grad = P.grad != 0;

    if (warp == P.CW) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        uint32_t gq = 0;
        UnitIter<K> it(P);
        int yt;
        int64_t z0, z1;
        while (it.next(P, yt, z0, z1)) {
            const int64_t y0 = (int64_t)yt * P.TY;
            const int tye = (int)amin(P.TY, P.ny - y0);
            const int nq = (int)(z1 - z0) + 2 * K;
            // rows [y0 - h, y0 + tye + h): periodic wraps, Dirichlet clips to the ghost shell
            auto rows_of = [&](int h, int64_t& lo, int64_t& hi) {
                lo = y0 - h;
                hi = y0 + tye + h;
                if (!PERIODIC) {
                    lo = amax(lo, -P.r);
                    hi = amin(hi, P.ny + P.r);
                }
            };
            auto plane_ok = [&](int64_t z) { return PERIODIC || (z >= -P.rz && z < P.nz + P.rz); };
            auto nbytes = [&](int h) {
                int64_t lo, hi;
                rows_of(h, lo, hi);
                return (uint32_t)(hi - lo) * rowb;
            };
            for (int q = 0; q < nq; ++q, ++gq) {
                const uint32_t s = gq % P.NS, k = gq / P.NS;
                if (k > 0 && !ptx::mbar_wait(&empty[s], (k - 1) & 1)) {
                    atimeout(P.status);
                    return;
                }
                const int64_t zi = z0 - K + q;  // plane of lambda, kappa, u_t in this stage
                const bool okz = plane_ok(zi);
                const bool okb = K == 2 && grad && plane_ok(zi - 1);  // u_{t-1} one plane behind
                uint32_t bytes = 0;
                if (okz) bytes += 2u * nbytes(K) + (grad ? nbytes(1) : 0u);
                if (okb) bytes += nbytes(1);
                ptx::mbar_arrive_expect_tx(&full[s], bytes);
                T* dst = stg + (size_t)s * P.stage_elems;
                auto copy = [&](const T* a, T* d, int h, int64_t z) {
                    int64_t lo, hi;
                    rows_of(h, lo, hi);
                    T* dd = d + (size_t)(lo - (y0 - h)) * P.pitch;
                    if (!PERIODIC) {
                        const T* src = a + (z + P.rz) * P.plane + (lo + P.r) * P.pitch;
                        ptx::bulk_g2s(dd, src, (uint32_t)(hi - lo) * rowb, &full[s]);
                    } else {
                        const int64_t zw = ((z % P.nz) + P.nz) % P.nz;
                        const T* pl = a + (zw + P.rz) * P.plane + (int64_t)P.r * P.pitch;
                        const int nrows = (int)(hi - lo);
                        int jr = 0;
                        while (jr < nrows) {
                            int64_t row = lo + jr;
                            row = ((row % P.ny) + P.ny) % P.ny;
                            const int run = (int)amin(nrows - jr, P.ny - row);
                            ptx::bulk_g2s(dd + (size_t)jr * P.pitch, pl + row * P.pitch, (uint32_t)run * rowb,
                                          &full[s]);
                            jr += run;
                        }
                    }
                };
                if (okz) {
                    copy(lam_in, dst, K, zi);
                    copy(kappa, dst + P.kap_off, K, zi);
                    if (grad) copy(ua, dst + P.ua_off, 1, zi);
                }
                if (okb) copy(ub, dst + P.ub_off, 1, zi - 1);
            }
        }
        // wait until every issued copy has landed before leaving
        for (uint32_t d = 0; d < (uint32_t)P.NS && d < gq; ++d) {
            const uint32_t g = gq - 1 - d;
            if (!ptx::mbar_wait(&full[g % P.NS], (g / P.NS) & 1)) atimeout(P.status);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ngx = P.ngx, pitch = (int)P.pitch;
    const bool pairw = warp < P.pair_warps;
    int gx = 0, rp = 0;
    bool act = false;
    if (pairw) {
        const int t = threadIdx.x;
        act = t < P.npair;
        if (act) {
            rp = t / ngx;
            gx = t - rp * ngx;
        }
    } else if (K == 2) {
        // both halo rows (above and below the tile) of one x group (the first
        // of the warp's two halo sub-tasks)
        const int t = threadIdx.x - 32 * P.pair_warps;
        act = t < ngx;
        if (act) gx = t;
    }
    const XCtx X = make_xctx<VN, PERIODIC>(gx, lane, ngx, (int)P.nx);
    const int x = X.x;
    const T ac = T(P.ac), bc = T(P.bc), an = T(P.an), bn = T(P.bn);
    // mu = w_n * lambda of a staged (lambda, kappa) pair; the product is
    // rounded on its own (never contracted into a later add), so every level
    // and every pass gets the same mu whatever code surrounds it
    auto mu_of = [&](T l, T k) -> T {
        if constexpr (UNIT) return mul_rn(k, l);
        else return mul_rn(fma(bn, k, an), l);
    };
    // the gradient factor bc u + bn (sum of the six neighbours of u)
    auto gfac = [&](T u, T nb) -> T {
        if constexpr (UNIT) return fma(bc, u, nb);
        else return fma(bc, u, mul_rn(bn, nb));
    };

    bool dead = false;
    uint32_t gq = 0, gr = 0;
    UnitIter<K> uit(P);
    int yt;
    int64_t z0, z1;
    while (uit.next(P, yt, z0, z1)) {
        const int64_t y0 = (int64_t)yt * P.TY;
        const int tye = (int)amin(P.TY, P.ny - y0);
        const int nq = (int)(z1 - z0) + 2 * K;
        const uint32_t base = gq;
        uint32_t sj = base % P.NS, pj = (base / P.NS) & 1, sp = 0;
        // Ring planes are numbered per CTA: iteration j >= 2 of this unit writes
        // plane rbase + j - 2 into slot (number mod 3); level 2 of iteration
        // j + 1 reads it.  Warps synchronise only through these barriers, so
        // they may drift apart by an iteration.
        const uint32_t rbase = gr;

        // first tile row of a row-pair task; halo tasks own rows -1 and tye
        const int rr0 = 2 * rp;
        // gradient reductions through the warp scratch: the warp holds 32
        // consecutive whole groups of both rows of one row pair
        const bool okw = pairw && __all_sync(0xffffffffu, act && X.xfull && rr0 + 1 < tye);
        const bool fastw = okw && (ngx % 32 == 0);
        // carried state (registers), per owned row: mu and u_t of the plane below the level-1 centre
        T m0p[2][VN], uap[2][VN];
        // level 2 (K == 2): lambda_1 and w_c at its centre, u_{t-1} below its centre (its mu_1
        // planes are read back from the ring).  A halo warp's second sub-task carries its mu
        // rows in uap, which halo warps have no other use for (one register set fewer)
        T l1p[2][VN], wcp[2][VN], ubp[2][VN];
        // level-1 results of this iteration, handed to level 2
        T l1n[2][VN], wcn[2][VN], m1n[2][VN], g1n[2][VN];  // g1n: this step's gradient term
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int e = 0; e < VN; ++e) {
                m0p[i][e] = uap[i][e] = T(0);
                l1p[i][e] = wcp[i][e] = ubp[i][e] = T(0);
                l1n[i][e] = wcn[i][e] = m1n[i][e] = g1n[i][e] = T(0);
            }

        for (int j = 0; j < nq; ++j) {
            // A wait that runs out is recorded and the warp carries on without
            // waiting: every consumer warp must keep reaching the named barrier.
            if (!dead && !ptx::mbar_wait_warp(&full[sj], pj)) {
                atimeout(P.status);
                dead = true;
            }
            const T* S1 = stg + (size_t)sj * P.stage_elems + P.xl;  // plane above the level-1 centre (column 0)
            const T* S0 = stg + (size_t)sp * P.stage_elems + P.xl;  // level-1 centre plane
            const int64_t c1 = z0 - K - 1 + j;                       // level-1 centre plane (j >= 1)
            const bool zout1 = !PERIODIC && (c1 < 0 || c1 >= P.nz);
            const bool own1 = c1 >= z0 && c1 < z1;
            // ring plane written by level 1 of this iteration (K == 2, j >= 2):
            // its slot's previous plane must have been read by every warp
            const uint32_t wn = rbase + (uint32_t)j - 2u, wslot = wn % A_RING;
            if (K == 2 && j >= 2 && wn >= (uint32_t)A_RING && !dead &&
                !ptx::mbar_wait_warp(&rempty[wslot], (wn / A_RING - 1u) & 1u)) {
                atimeout(P.status);
                dead = true;
            }

            if (pairw) {
                if constexpr (K == 2) {
                    if (grad && j >= 3) {
                        // ------------------------------------ row pair, level-2 gradient
                        // Level 2's centre this iteration is plane c1 - 1, which level 1
                        // computed last iteration; its term there is still in g1n.  The
                        // two steps' terms of a point are added in FP (T) and the pair
                        // goes to the FP64 accumulator in one reduction.
                        const T* UB = S0 + P.ub_off + rr0 * pitch;  // u_{t-1} row rr0 - 1 at plane c1 - 1
                        if (j == 3) {
                            // u_{t-1} of the plane below the first level-2 centre
#pragma unroll
                            for (int i = 0; i < 2; ++i) vld(UB + (i + 1) * pitch + x, ubp[i]);
                        } else {
                            const int64_t c2 = c1 - 1;
                            T uv[4][VN], uz[2][VN];
#pragma unroll
                            for (int i = 0; i < 4; ++i) vld(UB + i * pitch + x, uv[i]);
#pragma unroll
                            for (int i = 0; i < 2; ++i) vld(S1 + P.ub_off + (rr0 + 1 + i) * pitch + x, uz[i]);
#pragma unroll
                            for (int i = 0; i < 2; ++i) {
                                const T* Ur = UB + (i + 1) * pitch;
                                const T left = Ur[X.lcl], right = Ur[X.lcr];
                                T nb[VN], gp[VN];
                                nsum(X, ubp[i], uv[i], uv[i + 1], uv[i + 2], uz[i], left, right, nb);
#pragma unroll
                                for (int e = 0; e < VN; ++e) {
                                    const T g2 = mul_rn(l1p[i][e], gfac(uv[i + 1][e], nb[e]));
                                    gp[e] = add_rn(g1n[i][e], g2);
                                    ubp[i][e] = uv[i + 1][e];
                                }
                                add_grad(X, fastw, wscr, lane, P.origin + c2 * P.plane + (y0 + rr0 + i) * P.pitch + x,
                                         act && rr0 + i < tye, g64, P.gfirst != 0, gp);
                            }
                        }
                    }
                }
                // ------------------------------------------------ row pair, level 1
                const T* L = S0 + (rr0 - 1 + K) * pitch;  // lambda row rr0 - 1
                const T* Kp = L + P.kap_off;
                const T* U = S0 + P.ua_off + rr0 * pitch;  // u_t row rr0 - 1
                if (j == 1) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        T lv[VN], kv[VN];
                        vld(L + (i + 1) * pitch + x, lv);
                        vld(Kp + (i + 1) * pitch + x, kv);
#pragma unroll
                        for (int e = 0; e < VN; ++e) m0p[i][e] = mu_of(lv[e], kv[e]);
                        if (grad) vld(U + (i + 1) * pitch + x, uap[i]);
                    }
                } else if (j >= 2) {
                    T mv[4][VN], lc[2][VN], kc[2][VN], mz[2][VN];
#pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        T lv[VN], kv[VN];
                        vld(L + i * pitch + x, lv);
                        vld(Kp + i * pitch + x, kv);
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            mv[i][e] = mu_of(lv[e], kv[e]);
                            if (i == 1 || i == 2) {
                                lc[i - 1][e] = lv[e];
                                kc[i - 1][e] = kv[e];
                            }
                        }
                    }
                    {
                        const T* L1 = S1 + (rr0 + K) * pitch;
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            T lv[VN], kv[VN];
                            vld(L1 + i * pitch + x, lv);
                            vld(L1 + P.kap_off + i * pitch + x, kv);
#pragma unroll
                            for (int e = 0; e < VN; ++e) mz[i][e] = mu_of(lv[e], kv[e]);
                        }
                    }
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const T* Lr = L + (i + 1) * pitch;
                        const T left = mu_of(Lr[X.lcl], Lr[P.kap_off + X.lcl]);
                        const T right = mu_of(Lr[X.lcr], Lr[P.kap_off + X.lcr]);
                        T s[VN];
                        nsum(X, m0p[i], mv[i], mv[i + 1], mv[i + 2], mz[i], left, right, s);
                        const bool out = zout1 || (!PERIODIC && y0 + rr0 + i >= P.ny);
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            const T wc = fma(bc, kc[i][e], ac);
                            const T l1 = fma(wc, lc[i][e], s[e]);
                            l1n[i][e] = out ? T(0) : l1;
                            wcn[i][e] = wc;
                            T mu1 = out ? T(0) : mu_of(l1, kc[i][e]);
                            if (!PERIODIC && x + e >= X.nx) mu1 = T(0);  // ghost column of a ragged group
                            m1n[i][e] = mu1;
                            m0p[i][e] = mv[i + 1][e];
                        }
                    }
                    // gradient term of this step on the owned rows of an owned plane
                    if (grad) {
                        T uv[4][VN], uz[2][VN];
#pragma unroll
                        for (int i = 0; i < 4; ++i) vld(U + i * pitch + x, uv[i]);
#pragma unroll
                        for (int i = 0; i < 2; ++i) vld(S1 + P.ua_off + (rr0 + 1 + i) * pitch + x, uz[i]);
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const T* Ur = U + (i + 1) * pitch;
                            const T left = Ur[X.lcl], right = Ur[X.lcr];
                            T nb[VN];
                            nsum(X, uap[i], uv[i], uv[i + 1], uv[i + 2], uz[i], left, right, nb);
#pragma unroll
                            for (int e = 0; e < VN; ++e) {
                                g1n[i][e] = mul_rn(lc[i][e], gfac(uv[i + 1][e], nb[e]));
                                uap[i][e] = uv[i + 1][e];
                            }
                        }
                    }
                    if constexpr (K == 1) {
                        // final level: lambda_out of the owned rows
                        store_pair(okw, X, act, rr0, tye, lam_out + P.origin + c1 * P.plane + (y0 + rr0) * P.pitch + x,
                                   P.pitch, l1n);
                    } else {
                        // publish mu_1 of the owned rows for level 2's y neighbours
                        T* M = mring + (size_t)wslot * P.ring_elems + P.xl + (rr0 + 1) * pitch;
                        store_pair(okw, X, act, rr0, tye, M + x, (int64_t)pitch, m1n);
                    }
                    // K == 1: this step's gradient term goes to the accumulator now.
                    // K == 2: it stays in g1n until the next iteration, where level 2's
                    // term of the same plane joins it (one reduction per point and pass)
                    if (K == 1 && grad && own1) {
#pragma unroll
                        for (int i = 0; i < 2; ++i)
                            add_grad(X, fastw, wscr, lane, P.origin + c1 * P.plane + (y0 + rr0 + i) * P.pitch + x,
                                     act && rr0 + i < tye, g64, P.gfirst != 0, g1n[i]);
                    }
                }
            } else if (K == 2) {
                // ------------------------------------------------ halo rows, level 1 only
                // Two sub-tasks per halo warp (x groups 32 apart by the halo warp
                // count); the second keeps its carried mu rows in uap.
                auto halo = [&](const XCtx& Xh, bool acth, T (&m0)[2][VN]) {
                    const int xh = Xh.x;
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const int rh = i == 0 ? -1 : tye;
                        const T* L = S0 + (rh - 1 + K) * pitch;  // lambda row rh - 1
                        const T* Kp = L + P.kap_off;
                        if (j == 1) {
                            T lv[VN], kv[VN];
                            vld(L + pitch + xh, lv);
                            vld(Kp + pitch + xh, kv);
#pragma unroll
                            for (int e = 0; e < VN; ++e) m0[i][e] = mu_of(lv[e], kv[e]);
                        } else if (j >= 2) {
                            T mv[3][VN], lc[VN], kc[VN], mz[VN];
#pragma unroll
                            for (int r3 = 0; r3 < 3; ++r3) {
                                T lv[VN], kv[VN];
                                vld(L + r3 * pitch + xh, lv);
                                vld(Kp + r3 * pitch + xh, kv);
#pragma unroll
                                for (int e = 0; e < VN; ++e) {
                                    mv[r3][e] = mu_of(lv[e], kv[e]);
                                    if (r3 == 1) {
                                        lc[e] = lv[e];
                                        kc[e] = kv[e];
                                    }
                                }
                            }
                            {
                                const T* L1 = S1 + (rh + K) * pitch;
                                T lv[VN], kv[VN];
                                vld(L1 + xh, lv);
                                vld(L1 + P.kap_off + xh, kv);
#pragma unroll
                                for (int e = 0; e < VN; ++e) mz[e] = mu_of(lv[e], kv[e]);
                            }
                            const T* Lr = L + pitch;
                            const T left = mu_of(Lr[Xh.lcl], Lr[P.kap_off + Xh.lcl]);
                            const T right = mu_of(Lr[Xh.lcr], Lr[P.kap_off + Xh.lcr]);
                            T s[VN];
                            nsum(Xh, m0[i], mv[0], mv[1], mv[2], mz, left, right, s);
                            const int64_t yabs = y0 + rh;
                            const bool out = zout1 || (!PERIODIC && (yabs < 0 || yabs >= P.ny));
                            T mu1[VN];
#pragma unroll
                            for (int e = 0; e < VN; ++e) {
                                const T wc = fma(bc, kc[e], ac);
                                const T l1 = fma(wc, lc[e], s[e]);
                                mu1[e] = out ? T(0) : mu_of(l1, kc[e]);
                                m0[i][e] = mv[1][e];
                            }
                            if (acth)
                                store_row(Xh, mring + (size_t)wslot * P.ring_elems + P.xl + (rh + 1) * pitch + xh,
                                          mu1);
                        }
                    }
                };
                halo(X, act, m0p);
                const int s2 = warp - P.pair_warps + P.halo_warps;  // second sub-task (warp-uniform)
                if (32 * s2 < ngx) {
                    const int gx2 = 32 * s2 + lane;
                    halo(make_xctx<VN, PERIODIC>(gx2, lane, ngx, (int)P.nx), gx2 < ngx, uap);
                }
            }

            if constexpr (K == 2) {
                if (j >= 2) {  // this warp's rows of the ring plane are written
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&rfull[wslot]);
                }
                // the ring planes of the previous two iterations: level 2's centre
                // (rn, plane c1 - 1) and the plane below it (rn - 1, plane c1 - 2);
                // the plane above is this iteration's level-1 output, still in m1n
                const uint32_t rn = rbase + (uint32_t)j - 3u, rslot = rn % A_RING;
                const uint32_t ra = rn - 1u, aslot = ra % A_RING;
                if (pairw && j >= 4 && !dead &&
                    (!ptx::mbar_wait_warp(&rfull[rslot], (rn / A_RING) & 1u) ||
                     !ptx::mbar_wait_warp(&rfull[aslot], (ra / A_RING) & 1u))) {
                    atimeout(P.status);
                    dead = true;
                }
                if (pairw && j >= 4) {
                    // ------------------------------------------------ row pair, level 2
                    {
                        const int64_t c2 = c1 - 1;
                        const T* M = mring + (size_t)rslot * P.ring_elems + P.xl + rr0 * pitch;  // mu_1 row rr0 - 1
                        const T* MA = mring + (size_t)aslot * P.ring_elems + P.xl + (rr0 + 1) * pitch;  // row rr0
                        T mup[VN], mdn[VN], mc[2][VN], ma[2][VN];
                        vld(M + x, mup);
                        vld(M + pitch + x, mc[0]);
                        vld(M + 2 * pitch + x, mc[1]);
                        vld(M + 3 * pitch + x, mdn);
                        vld(MA + x, ma[0]);
                        vld(MA + pitch + x, ma[1]);
                        T l2[2][VN], s[2][VN];
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            const T* Mr = M + (i + 1) * pitch;
                            const T left = Mr[X.lcl], right = Mr[X.lcr];
                            nsum(X, ma[i], i == 0 ? mup : mc[0], mc[i], i == 0 ? mc[1] : mdn, m1n[i], left, right,
                                 s[i]);
#pragma unroll
                            for (int e = 0; e < VN; ++e) l2[i][e] = fma(wcp[i][e], l1p[i][e], s[i][e]);
                        }
                        store_pair(okw, X, act, rr0, tye, lam_out + P.origin + c2 * P.plane + (y0 + rr0) * P.pitch + x,
                                   P.pitch, l2);
                    }
                }
                if (pairw && j >= 2) {
#pragma unroll
                    for (int i = 0; i < 2; ++i)
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            l1p[i][e] = l1n[i][e];
                            wcp[i][e] = wcn[i][e];
                        }
                }
                // plane rn - 1 has had its last reader (level 2 of this iteration, as
                // the plane below its centre); halo warps never read the ring but
                // count among its readers
                if (j >= 4) {
                    __syncwarp();
                    if (lane == 0) ptx::mbar_arrive(&rempty[aslot]);
                }
            }

            // staged plane j - 1 is no longer needed
            if (j >= 1) {
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&empty[sp]);
            }
            sp = sj;
            if (++sj == (uint32_t)P.NS) {
                sj = 0;
                pj ^= 1u;
            }
        }
        __syncwarp();
        if (lane == 0) {
            ptx::mbar_arrive(&empty[sp]);  // the last staged plane
            // the unit's last two ring planes get no further reader: release them
            if (K == 2) {
                ptx::mbar_arrive(&rempty[(rbase + (uint32_t)nq - 4u) % A_RING]);
                ptx::mbar_arrive(&rempty[(rbase + (uint32_t)nq - 3u) % A_RING]);
            }
        }
        gq = base + nq;
        if (K == 2) gr = rbase + (uint32_t)nq - 2u;
    }
}

int adj_sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

constexpr size_t A_SMEM = 220 * 1024;

struct AdjCfg {
    int K, TY, NS, CW, pair_warps, npair, nzc;
    size_t stage_bytes, ring_bytes;
};

size_t adj_stage_rows(int TY, int K) { return 2 * (size_t)(TY + 2 * K) + (size_t)K * (TY + 2); }

// Tile rows, stages and z chunks for K fused steps.  Tiles take as many row
// pairs as one task per consumer thread allows (at most A_MAXCW warps, halo
// warps included, each halo warp covering two 32-group sub-tasks) and shared
// memory holds with at least one stage in flight: the halo rows a taller tile
// saves are worth more than extra stages (256^3 FP32: 10-row tiles, 117.5 us
// per reverse step, against 118.9 with 8 rows and one sub-task per halo warp).
bool adj_cfg(const Geom& g, int K, AdjCfg* c)
{
    const int VN = g.esize == 8 ? 2 : 4;
    const int ngx = (int)((g.nx + VN - 1) / VN);
    const size_t rowb = (size_t)g.pitch * g.esize;
    int eTY = 0, eNS = 0, eNZC = 0;
    const char* env = std::getenv("ST_ADJ_CFG");  // "TY,NS,nzc" for tuning sweeps
    const bool use_env = env && std::sscanf(env, "%d,%d,%d", &eTY, &eNS, &eNZC) == 3 && eTY >= 2 && eTY % 2 == 0 &&
                         eNS >= 3 && eNZC >= 1;
    AdjCfg best{};
    bool have = false;
    {
        const int min_ns = 3;
        for (int TY = 16; TY >= 2; TY -= 2) {
            if (use_env && TY != eTY) continue;
            if (TY > 2 && TY - 2 >= g.ny) continue;  // no taller than the grid
            const int npair = (TY / 2) * ngx;
            const int pw = (npair + 31) / 32;
            const int hw = K == 2 ? ((ngx + 31) / 32 + 1) / 2 : 0;  // two halo sub-tasks per warp
            if (pw + hw > A_MAXCW) continue;
            const size_t sb = (adj_stage_rows(TY, K) * rowb + 127) / 128 * 128;
            const size_t rb = K == 2 ? (size_t)A_RING * (TY + 2) * rowb : 0;
            const size_t fixed = rb + 512 + (size_t)(pw + hw) * 32 * VN * 8;  // ring, barriers, warp scratch
            if (fixed + 3 * sb > A_SMEM) continue;
            int NS = (int)std::min<size_t>(8, (A_SMEM - fixed) / sb);
            if (use_env) NS = std::min(NS, eNS);
            if (NS < min_ns && !use_env) continue;
            best = AdjCfg{K, TY, NS, pw + hw, pw, npair, 1, sb, rb};
            have = true;
            break;
        }
    }
    if (!have) return false;
    // z chunks of the tiles-by-chunks grid (used only when the flat
    // distribution cannot be): balance the per-CTA critical path against the
    // extra planes each chunk stages (2K of them)
    const int nyt = (int)((g.ny + best.TY - 1) / best.TY);
    const int64_t nsm = adj_sm_count();
    double bestcost = 1e300;
    for (int64_t nzc = 1; nzc <= g.nz; ++nzc) {
        const int64_t units = nyt * nzc;
        const int64_t zmax = (g.nz + nzc - 1) / nzc;
        const double waves = (double)((units + nsm - 1) / nsm);
        const double path = waves * (double)(zmax + 2 * K);
        const double total = (double)nyt * (double)(g.nz + 2 * K * nzc) / (double)nsm;
        const double cost = std::max(path, total);
        if (cost < bestcost - 1e-9) {
            bestcost = cost;
            best.nzc = (int)nzc;
        }
        if (units > 64 * nsm) break;
    }
    if (use_env) best.nzc = (int)std::min<int64_t>(eNZC, g.nz);
    *c = best;
    return true;
}

template <typename T, int K, bool PERIODIC>
cudaError_t launch_adj_t(const Family& f, const AdjointArgs& a, const AdjCfg& c, cudaStream_t s)
{
    const Geom& g = f.g;
    AdjParams P;
    std::memset(&P, 0, sizeof(P));
    P.nz = g.nz;
    P.ny = g.ny;
    P.nx = g.nx;
    P.pitch = g.pitch;
    P.plane = g.plane;
    P.origin = g.origin;
    P.rz = g.rz;
    P.r = g.r;
    P.xl = (int)g.xl;
    P.TY = c.TY;
    P.NS = c.NS;
    P.CW = c.CW;
    P.nyt = (int)((g.ny + c.TY - 1) / c.TY);
    P.nzc = c.nzc;
    P.units = P.nyt * P.nzc;
    // Flat distribution: every CTA gets an equal share of the (tile, plane)
    // pairs, cut from the tile-major sequence, so all SMs take part however
    // the tile count divides (256^3 FP32: 26 tiles of 10 rows give 130
    // tile-by-chunk units for 152 SMs; flat: 106.3 instead of 113.2 us per
    // reverse step, 75.0 instead of 82.1 with every state kept).  A CTA's
    // range may end inside one tile and go on in the next; neighbouring
    // tiles then meet their shared halo rows at different times, so those
    // come from DRAM more often.  The tiles-by-chunks grid remains for
    // sequences too long for 32-bit positions.
    P.flat = (int64_t)P.nyt * (g.nz + 2 * K) < ((int64_t)1 << 31);
    const int grid = (int)std::min<int64_t>(P.flat ? (int64_t)P.nyt * P.nz : P.units, adj_sm_count());
    if (P.flat) {
        // iterations of the longest CTA under either split (256^3 FP32: 49
        // on the cost axis against 52 with equal shares of planes)
        auto longest = [&](uint32_t w) {
            const uint32_t nz = (uint32_t)g.nz, nyt = (uint32_t)P.nyt;
            const uint64_t V = (uint64_t)nyt * (nz + w);
            int64_t worst = 0;
            for (int b = 0; b < grid; ++b) {
                const uint32_t lo = flat_cut(V * b / grid, nz, nyt, w), hi = flat_cut(V * (b + 1) / grid, nz, nyt, w);
                int64_t cost = 0;
                for (uint32_t p = lo; p < hi;) {
                    const uint32_t e = std::min(hi, (p / nz + 1) * nz);
                    cost += (int64_t)(e - p) + 2 * K;
                    p = e;
                }
                worst = std::max(worst, cost);
            }
            return worst;
        };
        P.flat = longest(2 * K) < longest(0) ? 2 : 1;
    }
    P.ngx = (int)((g.nx + AV<T>::N - 1) / AV<T>::N);
    P.npair = c.npair;
    P.pair_warps = c.pair_warps;
    P.halo_warps = c.CW - c.pair_warps;
    P.stage_elems = (uint32_t)(c.stage_bytes / sizeof(T));
    P.kap_off = (uint32_t)((c.TY + 2 * K) * g.pitch);
    P.ua_off = 2 * P.kap_off;
    P.ub_off = P.ua_off + (uint32_t)((c.TY + 2) * g.pitch);
    P.ring_elems = (uint32_t)((c.TY + 2) * g.pitch);
    P.grad = a.gk != nullptr ? 1 : 0;
    if (P.grad && sizeof(T) == 4 && !a.gpart) return cudaErrorInvalidValue;
    P.gfirst = a.gfirst;
    const StarCoef& k = f.sc;
    P.ac = k.c_a;
    P.bc = k.c_b;
    P.an = k.a[0][0][0];
    P.bn = k.b[0][0][0];
    P.status = a.status;
    const size_t smem = c.ring_bytes + (size_t)c.NS * c.stage_bytes + sizeof(uint64_t) * (2 * c.NS + 2 * A_RING) +
                        (size_t)c.CW * 32 * AV<T>::N * sizeof(double);
    // the variable-diffusivity operator's weights (an = 0, bn = 1) take the
    // specialised kernel
    const bool unit = P.an == 0.0 && P.bn == 1.0;
    auto fn = unit ? k_adjoint<T, K, PERIODIC, true> : k_adjoint<T, K, PERIODIC, false>;
    static bool attr[2] = {false, false};
    if (!attr[unit]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr[unit] = true;
    }
    T* gacc = sizeof(T) == 8 ? reinterpret_cast<T*>(a.gk) : static_cast<T*>(a.gpart);
    return launch_dependent(fn, dim3(grid), dim3((c.CW + 1) * 32), smem, s, (const T*)a.lam_in, (T*)a.lam_out,
                            (const T*)a.kappa, (const T*)a.u, (const T*)a.u2, gacc, P);
}

}  // namespace

// Largest number of fused steps the optimised adjoint handles for this
// family (0: use the one-thread-per-point transpose).
int star3d_adjoint_fuse(const Family& f)
{
    if (f.kind != FAM_STAR3D || !f.has_beta || f.levels != 1) return 0;
    const StarCoef& k = f.sc;
    for (int ax = 0; ax < 3; ++ax)
        for (int sd = 0; sd < 2; ++sd)
            if (k.a[ax][sd][0] != k.a[0][0][0] || k.b[ax][sd][0] != k.b[0][0][0]) return 0;
    AdjCfg c;
    if (adj_cfg(f.g, 2, &c)) return 2;
    return adj_cfg(f.g, 1, &c) ? 1 : 0;
}

// The exact double of a finite nonzero normal float, by rebiasing its
// exponent field (IEEE 754 binary32 -> binary64) on the integer units, so
// that k_grad_flush issues one FP64 instruction per point (the add); zeros,
// subnormals, infinities and NaNs take the hardware conversion.
__device__ __forceinline__ double widen_exact(float f)
{
    const uint32_t b = __float_as_uint(f);
    const uint32_t e = (b >> 23) & 0xffu;
    if (e == 0u || e == 0xffu) return (double)f;
    const uint64_t bits = ((uint64_t)(b >> 31) << 63) | ((uint64_t)(e + (1023u - 127u)) << 52) |
                          ((uint64_t)(b & 0x7fffffu) << 29);
    return __longlong_as_double((long long)bits);
}

// gk += part over the whole padded buffer (the partial's ghost and padding
// cells stay 0: the buffer is cleared once per reverse pass and the passes
// write interior points only).  16-byte groups; n is a multiple of 4.
__global__ void __launch_bounds__(256) k_grad_flush(const float4* __restrict__ part, double2* __restrict__ gk, int64_t n4)
{
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
        const float4 v = part[i];
        double2 a = gk[2 * i], b = gk[2 * i + 1];
        a.x += widen_exact(v.x);
        a.y += widen_exact(v.y);
        b.x += widen_exact(v.z);
        b.y += widen_exact(v.w);
        gk[2 * i] = a;
        gk[2 * i + 1] = b;
    }
}

cudaError_t launch_grad_flush(void* part, double* gk, int64_t n, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    if (n % 4 != 0 || ((uintptr_t)part | (uintptr_t)gk) % 16 != 0) return cudaErrorInvalidValue;
    const int64_t n4 = n / 4;
    return launch_dependent(k_grad_flush, dim3((unsigned)std::min<int64_t>((n4 + 255) / 256, (int64_t)1 << 30)), dim3(256),
                            0, s, static_cast<const float4*>(part), reinterpret_cast<double2*>(gk), n4);
}

cudaError_t launch_star3d_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s)
{
    if (a.steps < 1 || a.steps > 2 || star3d_adjoint_fuse(f) < a.steps) return cudaErrorNotSupported;
    AdjCfg c;
    if (!adj_cfg(f.g, a.steps, &c)) return cudaErrorNotSupported;
    const bool dbl = f.g.esize == 8;
    if (a.steps == 2) {
        if (dbl) return f.periodic ? launch_adj_t<double, 2, true>(f, a, c, s) : launch_adj_t<double, 2, false>(f, a, c, s);
        return f.periodic ? launch_adj_t<float, 2, true>(f, a, c, s) : launch_adj_t<float, 2, false>(f, a, c, s);
    }
    if (dbl) return f.periodic ? launch_adj_t<double, 1, true>(f, a, c, s) : launch_adj_t<double, 1, false>(f, a, c, s);
    return f.periodic ? launch_adj_t<float, 1, true>(f, a, c, s) : launch_adj_t<float, 1, false>(f, a, c, s);
}

}  // namespace st
