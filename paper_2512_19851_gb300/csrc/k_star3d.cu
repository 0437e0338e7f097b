// 3D radius-1 star sweep (7-point), constant or per-cell weights, one time
// level: the 3D heat workloads and the variable-coefficient diffusion.
//
// Design (one GPU, HBM-bound):
//  * A CTA owns a tile of TY full rows (all of x) and streams it through a
//    chunk of ZC planes.  Plane tiles (TY + 2 rows, halo included; the
//    coefficient tile without halo) are staged in shared memory by 1D bulk
//    copies (the TMA engine, cp.async.bulk) into a ring of NS stages, each
//    completing on its own mbarrier; a dedicated producer warp issues them, so
//    several planes are in flight per SM while 8 consumer warps compute.
//  * Full rows make the x halo free: x-1/x+1 come from the same shared row
//    (wrapped inside the row for a periodic boundary, the ghost columns for a
//    Dirichlet one).  The y halo rows and the z planes are copied with wrapped
//    row/plane indices when periodic, so ghost cells are never needed there.
//  * CTAs are persistent (one per SM) and walk (y-tile, z-chunk) units with y
//    fastest, so tiles that share halo rows run at the same time and the halo
//    re-reads hit L2.
//  * Consumers load 16-byte vectors from shared memory and store 16-byte
//    vectors straight to global memory (coalesced, one write per point).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

// Consumer warps per CTA: 16, or 12 for the conservative form, whose thread
// carries twice the planes (u and kappa) and needs up to 128 registers.
template <bool CONS>
__host__ __device__ constexpr int consumer_warps() { return CONS ? 12 : 16; }
template <bool CONS>
__host__ __device__ constexpr int block_threads() { return (consumer_warps<CONS>() + 1) * 32; }

struct Star1Params {
    int64_t nz, ny, nx, pitch, plane, origin;
    int rz, r, xl;
    int TY, ZC, NS;
    int nyt, nzc, units;
    uint32_t stage_elems;  // per stage: u tile then coefficient tile
    uint32_t u_elems;      // (TY + 2) * pitch
    double wc, wxm, wxp, wym, wyp, wzm, wzp;  // constant parts (alpha)
    double bc, bxm, bxp, bym, byp, bzm, bzp;  // per-cell parts (beta)
    int* status;
    double* red;  // RED: per-block (sum, sum of squares, max |u|) of the written level, 3 doubles per block
};

template <typename T>
struct V;
template <>
struct V<float> {
    static constexpr int N = 4;
    typedef float4 type;
};
template <>
struct V<double> {
    static constexpr int N = 2;
    typedef double2 type;
};

template <typename T>
__device__ __forceinline__ void ldv(const T* p, T (&v)[V<T>::N])
{
    typename V<T>::type t = *reinterpret_cast<const typename V<T>::type*>(p);
    if constexpr (V<T>::N == 4) {
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
__device__ __forceinline__ void stv(T* p, const T (&v)[V<T>::N])
{
    typename V<T>::type t;
    if constexpr (V<T>::N == 4) {
        t.x = v[0];
        t.y = v[1];
        t.z = v[2];
        t.w = v[3];
    } else {
        t.x = v[0];
        t.y = v[1];
    }
    *reinterpret_cast<typename V<T>::type*>(p) = t;
}

__device__ __forceinline__ int64_t imin64(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ int64_t wrapi(int64_t i, int64_t n)
{
    i = i < 0 ? i + n : i;
    return i >= n ? i - n : i;
}

// One output point from its centre, six neighbours and (optionally) kappa.
template <typename T, bool KAPPA, bool SYM>
__device__ __forceinline__ T point(const Star1Params& P, T c, T xm, T xp, T ym, T yp, T zm, T zp, T k)
{
    if constexpr (SYM) {
        const T nb = ((((xm + xp) + ym) + yp) + zm) + zp;
        if constexpr (KAPPA) {
            const T wc = fma(T(P.bc), k, T(P.wc));
            const T wn = fma(T(P.bxm), k, T(P.wxm));
            return fma(wc, c, wn * nb);
        } else {
            return fma(T(P.wc), c, T(P.wxm) * nb);
        }
    } else {
        T wc = T(P.wc), a = T(P.wxm), b = T(P.wxp), d = T(P.wym), e = T(P.wyp), f = T(P.wzm), g = T(P.wzp);
        if constexpr (KAPPA) {
            wc = fma(T(P.bc), k, wc);
            a = fma(T(P.bxm), k, a);
            b = fma(T(P.bxp), k, b);
            d = fma(T(P.bym), k, d);
            e = fma(T(P.byp), k, e);
            f = fma(T(P.bzm), k, f);
            g = fma(T(P.bzp), k, g);
        }
        T acc = wc * c;
        acc = fma(a, xm, acc);
        acc = fma(b, xp, acc);
        acc = fma(d, ym, acc);
        acc = fma(e, yp, acc);
        acc = fma(f, zm, acc);
        acc = fma(g, zp, acc);
        return acc;
    }
}

// One output point of the conservative face-averaged form: each face's
// coefficient is the mean of the two cells' kappa, and a Dirichlet ghost
// face takes kappa of the cell itself, which the kernel gets by the same
// expression because the coefficient field's ghost cells mirror their
// interior neighbours ((k + k) / 2 = k exactly).  Faces in the order -z, +z,
// -y, +y, -x, +x.
template <typename T>
__device__ __forceinline__ T cons_point(T c, T k, T xm, T kxm, T xp, T kxp, T ym, T kym, T yp, T kyp, T zm, T kzm,
                                        T zp, T kzp)
{
    const T h = T(0.5);
    T acc = ((k + kzm) * h) * (zm - c);
    acc = fma((k + kzp) * h, zp - c, acc);
    acc = fma((k + kym) * h, ym - c, acc);
    acc = fma((k + kyp) * h, yp - c, acc);
    acc = fma((k + kxm) * h, xm - c, acc);
    acc = fma((k + kxp) * h, xp - c, acc);
    return c + acc;
}

__device__ __forceinline__ void set_timeout(int* status)
{
    if (status) atomicCAS(status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
}

// RED: the thread's running sum and sum of squares as compensated float pairs
// (Knuth's two-sum on each addition, the low part gathering the rounding
// errors; about 48 bits), in two streams (even and odd values) advanced
// together by packed FP32x2 instructions, and max |v|.
__device__ __forceinline__ float2 padd2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 psub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

struct RedAcc {
    float2 hs{0.f, 0.f}, ls{0.f, 0.f}, hq{0.f, 0.f}, lq{0.f, 0.f};
    float m = 0.f;
    __device__ __forceinline__ static void two_sum(float2& hi, float2& lo, float2 x)
    {
        const float2 s = padd2(hi, x);
        const float2 bp = psub2(s, hi);
        const float2 e = padd2(psub2(hi, psub2(s, bp)), psub2(x, bp));
        hi = s;
        lo = padd2(lo, e);
    }
    // two written values (a ragged end passes 0 for the second: an exact no-op)
    __device__ __forceinline__ void put(float2 x)
    {
        two_sum(hs, ls, x);
        const float2 p = __fmul2_rn(x, x);
        two_sum(hq, lq, p);
        lq = padd2(lq, __ffma2_rn(x, x, make_float2(-p.x, -p.y)));  // the square's exact rounding error
        m = fmaxf(m, fmaxf(fabsf(x.x), fabsf(x.y)));
    }
};

// CONS: the conservative face-averaged operator (KAPPA set): the coefficient
// tile carries the same halo rows as u and is staged for every plane.
// RED (FP32): the sweep also reduces the level it writes, as stencil_reduce
// would (sum, sum of squares, max |u| over the interior), so the step that
// ends with a reduction reads its field once: every consumer thread adds its
// written values to compensated float pairs, the consumer warps combine them
// in double in a fixed order, and the block's partial goes to P.red.
template <typename T, bool KAPPA, bool SYM, bool PERIODIC, int G, bool CONS = false, bool RED = false>
__global__ void __launch_bounds__(block_threads<CONS>(), 1)
k_star1(const T* __restrict__ in, T* __restrict__ out, const T* __restrict__ kappa, const __grid_constant__ Star1Params P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)P.NS * P.stage_elems * sizeof(T));
    uint64_t* empty = full + P.NS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int VN = V<T>::N;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.NS; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], consumer_warps<CONS>());
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();
    ptx::griddep_wait();  // earlier kernels of the stream wrote our inputs / read our outputs
    ptx::griddep_trigger();

    const uint32_t rowb = (uint32_t)(P.pitch * sizeof(T));

    if (warp == consumer_warps<CONS>()) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        uint32_t gq = 0;
        for (int u = blockIdx.x; u < P.units; u += gridDim.x) {
            const int yt = u % P.nyt, zc = u / P.nyt;
            const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
            const int tye = (int)imin64(P.TY, P.ny - y0);
            const int zce = (int)imin64(P.ZC, P.nz - z0);
            for (int q = 0; q < zce + 2; ++q, ++gq) {
                const uint32_t s = gq % P.NS, k = gq / P.NS;
                if (k > 0 && !ptx::mbar_wait(&empty[s], (k - 1) & 1)) {
                    set_timeout(P.status);
                    return;
                }
                const int64_t zi = z0 - 1 + q;
                const bool need_k = KAPPA && (CONS || (q >= 1 && q <= zce));
                const uint32_t krows = CONS ? (uint32_t)(tye + 2) : (uint32_t)tye;
                const uint32_t bytes = (uint32_t)(tye + 2) * rowb + (need_k ? krows * rowb : 0u);
                T* dst = ring + (size_t)s * P.stage_elems;
                ptx::mbar_arrive_expect_tx(&full[s], bytes);
                // the tile rows y0 - 1 .. y0 + tye of plane zi of a field
                auto tile = [&](const T* fld, T* d) {
                    if (!PERIODIC) {
                        const T* src = fld + (zi + P.rz) * P.plane + (y0 - 1 + P.r) * P.pitch;
                        ptx::bulk_g2s(d, src, (uint32_t)(tye + 2) * rowb, &full[s]);
                    } else {
                        const T* pl = fld + (wrapi(zi, P.nz) + P.rz) * P.plane + (int64_t)P.r * P.pitch;
                        int j = 0;
                        while (j < tye + 2) {
                            int64_t row = y0 - 1 + j;
                            row = ((row % P.ny) + P.ny) % P.ny;
                            const int run = (int)imin64(tye + 2 - j, P.ny - row);
                            ptx::bulk_g2s(d + (size_t)j * P.pitch, pl + row * P.pitch, (uint32_t)run * rowb, &full[s]);
                            j += run;
                        }
                    }
                };
                tile(in, dst);
                if constexpr (CONS) {
                    tile(kappa, dst + P.u_elems);
                } else if (need_k) {
                    const T* ks = kappa + (zi + P.rz) * P.plane + (y0 + P.r) * P.pitch;
                    ptx::bulk_g2s(dst + P.u_elems, ks, (uint32_t)tye * rowb, &full[s]);
                }
            }
        }
        // drain: wait until every issued copy has landed before leaving
        for (uint32_t d = 0; d < (uint32_t)P.NS && d < gq; ++d) {
            const uint32_t g = gq - 1 - d;
            if (!ptx::mbar_wait(&full[g % P.NS], (g / P.NS) & 1)) set_timeout(P.status);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    // Each thread owns G column tasks per unit: a pair of rows (2 rp, 2 rp + 1)
    // at one VN-wide x group.  It keeps the two rows of the planes below, at
    // and above the output plane in registers (z reuse), and the pair shares
    // its inner y neighbours (y reuse); only the plane above, the pair's outer
    // y neighbours and the x edges are read from shared memory.
    const int ct = threadIdx.x;
    const int NC = consumer_warps<CONS>() * 32;
    const int ngx = (int)((P.nx + VN - 1) / VN);
    const unsigned FULLM = 0xffffffffu;
    RedAcc racc;  // RED: this thread's written values
    // A wait that runs out records the timeout and leaves; with RED it leaves
    // the streaming loop for the consumers' final combination instead.
    uint32_t gq = 0;
    for (int u = blockIdx.x; u < P.units; u += gridDim.x) {
        const int yt = u % P.nyt, zc = u / P.nyt;
        const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
        const int tye = (int)imin64(P.TY, P.ny - y0);
        const int zce = (int)imin64(P.ZC, P.nz - z0);
        const uint32_t base = gq;
        const int ntasks = ((tye + 1) / 2) * ngx;
        int trow[G], tgx[G];
        bool tact[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            const int t = ct + g * NC;
            tact[g] = t < ntasks;
            const int rp = tact[g] ? t / ngx : 0;
            trow[g] = 2 * rp;
            tgx[g] = tact[g] ? t - rp * ngx : 0;
        }
        auto stage = [&](int q) -> const T* {
            return ring + (size_t)((base + q) % P.NS) * P.stage_elems + P.xl;
        };
        auto wait_q = [&](int q) -> bool {
            const uint32_t gg = base + q;
            return ptx::mbar_wait_warp(&full[gg % P.NS], (gg / P.NS) & 1);
        };
        auto release = [&](int q) {
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[(base + q) % P.NS]);
        };
        T bel[G][2][VN], cen[G][2][VN], abv[G][2][VN];
        // CONS: the coefficient's planes below, at and above (same layout as u)
        T kbl[CONS ? G : 1][2][VN], kcn[CONS ? G : 1][2][VN], kab[CONS ? G : 1][2][VN];
        if (!wait_q(0) || !wait_q(1)) {
            set_timeout(P.status);
            if constexpr (RED) goto red_combine;
            else return;
        }
#pragma unroll
        for (int g = 0; g < G; ++g)
#pragma unroll
            for (int r = 0; r < 2; ++r) {
                const int off = (trow[g] + r + 1) * (int)P.pitch + tgx[g] * VN;
                ldv(stage(0) + off, bel[g][r]);
                ldv(stage(1) + off, cen[g][r]);
                if constexpr (CONS) {
                    ldv(stage(0) + P.u_elems + off, kbl[g][r]);
                    ldv(stage(1) + P.u_elems + off, kcn[g][r]);
                }
            }
        release(0);
        // running ring slots of the centre plane (i + 1) and the plane above
        // (i + 2), and the phase parity of the latter
        uint32_t slot_c = (base + 1) % P.NS, slot_a = (base + 2) % P.NS;
        uint32_t par_a = ((base + 2) / P.NS) & 1;
        for (int i = 0; i < zce; ++i) {
            if (!ptx::mbar_wait_warp(&full[slot_a], par_a)) {
                set_timeout(P.status);
                if constexpr (RED) goto red_combine;
                else return;
            }
            const T* sa = ring + (size_t)slot_a * P.stage_elems + P.xl;
            const T* sc = ring + (size_t)slot_c * P.stage_elems + P.xl;
            const T* sk = sc + P.u_elems;
            T* oplane = out + P.origin + (z0 + i) * P.plane + y0 * P.pitch;
#pragma unroll
            for (int g = 0; g < G; ++g) {
                const int x = tgx[g] * VN;
                // periodic only: the row end falls inside this group (ragged last group)
                const bool wrap_in_group = PERIODIC && x + VN > P.nx;
                const int rbase = trow[g] * (int)P.pitch + x;  // smem offset of row trow - 1
                T up[VN], dn[VN], kv[2][VN], kup[VN], kdn[VN];
#pragma unroll
                for (int r = 0; r < 2; ++r) ldv(sa + rbase + (r + 1) * (int)P.pitch, abv[g][r]);
                ldv(sc + rbase, up);
                ldv(sc + rbase + 3 * (int)P.pitch, dn);
                if constexpr (CONS) {
#pragma unroll
                    for (int r = 0; r < 2; ++r) ldv(sa + P.u_elems + rbase + (r + 1) * (int)P.pitch, kab[g][r]);
                    ldv(sk + rbase, kup);
                    ldv(sk + rbase + 3 * (int)P.pitch, kdn);
                } else if constexpr (KAPPA) {
                    ldv(sk + rbase, kv[0]);
                    ldv(sk + rbase + (int)P.pitch, kv[1]);
                }
#pragma unroll
                for (int r = 0; r < 2; ++r) {
                    const T* crow = sc + rbase + (r + 1) * (int)P.pitch - x;  // centre row, x = 0
                    // x edges from the neighbouring lanes, or shared memory at row/warp ends
                    T left = __shfl_up_sync(FULLM, cen[g][r][VN - 1], 1);
                    T right = __shfl_down_sync(FULLM, cen[g][r][0], 1);
                    if (lane == 0 || tgx[g] == 0) left = (PERIODIC && x == 0) ? crow[P.nx - 1] : crow[x - 1];
                    if (lane == 31 || tgx[g] == ngx - 1) right = (PERIODIC && x + VN >= P.nx) ? crow[0] : crow[x + VN];
                    const T* yl = r == 0 ? up : cen[g][0];
                    const T* yh = r == 0 ? cen[g][1] : dn;
                    T o[VN];
                    if constexpr (CONS) {
                        const T* krow = crow + P.u_elems;
                        T kleft = __shfl_up_sync(FULLM, kcn[g][r][VN - 1], 1);
                        T kright = __shfl_down_sync(FULLM, kcn[g][r][0], 1);
                        if (lane == 0 || tgx[g] == 0) kleft = (PERIODIC && x == 0) ? krow[P.nx - 1] : krow[x - 1];
                        if (lane == 31 || tgx[g] == ngx - 1)
                            kright = (PERIODIC && x + VN >= P.nx) ? krow[0] : krow[x + VN];
                        const T* kyl = r == 0 ? kup : kcn[g][0];
                        const T* kyh = r == 0 ? kcn[g][1] : kdn;
#pragma unroll
                        for (int j = 0; j < VN; ++j) {
                            const T xm = j == 0 ? left : cen[g][r][j - 1];
                            const T kxm = j == 0 ? kleft : kcn[g][r][j - 1];
                            T xp = j == VN - 1 ? right : cen[g][r][j + 1];
                            T kxp = j == VN - 1 ? kright : kcn[g][r][j + 1];
                            if (PERIODIC && wrap_in_group && x + j + 1 == P.nx) {
                                xp = crow[0];
                                kxp = krow[0];
                            }
                            o[j] = cons_point<T>(cen[g][r][j], kcn[g][r][j], xm, kxm, xp, kxp, yl[j], kyl[j], yh[j],
                                                 kyh[j], bel[g][r][j], kbl[g][r][j], abv[g][r][j], kab[g][r][j]);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < VN; ++j) {
                            const T xm = j == 0 ? left : cen[g][r][j - 1];
                            T xp = j == VN - 1 ? right : cen[g][r][j + 1];
                            if (PERIODIC && wrap_in_group && x + j + 1 == P.nx) xp = crow[0];
                            o[j] = point<T, KAPPA, SYM>(P, cen[g][r][j], xm, xp, yl[j], yh[j], bel[g][r][j],
                                                        abv[g][r][j], KAPPA ? kv[r][j] : T(0));
                        }
                    }
                    if (tact[g] && trow[g] + r < tye) {
                        T* op = oplane + (int64_t)(trow[g] + r) * P.pitch + x;
                        if (x + VN <= P.nx) {
                            stv(op, o);
                            if constexpr (RED) {
#pragma unroll
                                for (int j = 0; j < VN; j += 2) racc.put(make_float2(o[j], o[j + 1]));
                            }
                        } else {
                            for (int j = 0; j < VN && x + j < P.nx; ++j) {
                                op[j] = o[j];
                                if constexpr (RED) racc.put(make_float2(o[j], 0.f));
                            }
                        }
                    }
                }
#pragma unroll
                for (int r = 0; r < 2; ++r)
#pragma unroll
                    for (int j = 0; j < VN; ++j) {
                        bel[g][r][j] = cen[g][r][j];
                        cen[g][r][j] = abv[g][r][j];
                        if constexpr (CONS) {
                            kbl[g][r][j] = kcn[g][r][j];
                            kcn[g][r][j] = kab[g][r][j];
                        }
                    }
            }
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[slot_c]);  // plane i + 1
            if (i == zce - 1) release(i + 2);
            slot_c = slot_a;
            if (++slot_a == (uint32_t)P.NS) {
                slot_a = 0;
                par_a ^= 1u;
            }
        }
        gq = base + zce + 2;
    }
    if constexpr (!RED) {
        return;  // (the label below is RED's; this keeps it referenced in every instance)
        goto red_combine;
    }
red_combine:
    if constexpr (RED) {
        // the consumer warps only (the producer warp has left): named barrier 1
        double* wred = reinterpret_cast<double*>(empty + P.NS);  // 3 doubles per consumer warp
        double rs = ((double)racc.hs.x + (double)racc.ls.x) + ((double)racc.hs.y + (double)racc.ls.y);
        double rq = ((double)racc.hq.x + (double)racc.lq.x) + ((double)racc.hq.y + (double)racc.lq.y);
        double rm = (double)racc.m;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            rs += __shfl_down_sync(FULLM, rs, o);
            rq += __shfl_down_sync(FULLM, rq, o);
            rm = fmax(rm, __shfl_down_sync(FULLM, rm, o));
        }
        if (lane == 0) {
            wred[3 * warp + 0] = rs;
            wred[3 * warp + 1] = rq;
            wred[3 * warp + 2] = rm;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(NC) : "memory");
        if (threadIdx.x == 0) {
            double bs = 0.0, bq = 0.0, bm = 0.0;
            for (int w = 0; w < consumer_warps<CONS>(); ++w) {
                bs += wred[3 * w + 0];
                bq += wred[3 * w + 1];
                bm = fmax(bm, wred[3 * w + 2]);
            }
            P.red[3 * blockIdx.x + 0] = bs;
            P.red[3 * blockIdx.x + 1] = bq;
            P.red[3 * blockIdx.x + 2] = bm;
        }
    }
}

struct Cfg {
    int TY, ZC, NS, G;
};

int sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

constexpr size_t SMEM_BUDGET = 200 * 1024;

// Coefficient rows staged per plane: none, the tile rows, or (the
// conservative form) the tile rows with their y halo.
enum KMode { K_NONE = 0, K_TILE = 1, K_HALO = 2 };

size_t stage_bytes(const Geom& g, int TY, int kappa)
{
    const size_t krows = kappa == K_HALO ? (size_t)TY + 2 : (kappa == K_TILE ? (size_t)TY : 0);
    size_t e = (size_t)(TY + 2) * g.pitch + krows * g.pitch;
    e = (e * g.esize + 127) / 128 * 128;
    return e;
}

// Tile rows TY (even), z-chunk ZC, ring stages NS, tasks per thread G.
bool pick_cfg(const Geom& g, int kappa, Cfg* c)
{
    const int VN = 16 / g.esize;
    const int NC = consumer_warps<false>() * 32 * (kappa == K_HALO ? 3 : 4) / 4;
    const int ngx = (int)((g.nx + VN - 1) / VN);
    int TY = 2 * std::max(1, (NC + ngx - 1) / ngx);  // row pairs x groups ~ one task per thread
    TY = std::min(TY, 16);
    TY = (int)std::min<int64_t>(TY, (g.ny + 1) / 2 * 2);
    const char* env = std::getenv("ST_STAR1_CFG");  // "TY,ZC,NS" for tuning sweeps
    int eTY = 0, eZC = 0, eNS = 0;
    const bool use_env = env && std::sscanf(env, "%d,%d,%d", &eTY, &eZC, &eNS) == 3 && eTY >= 2 && eTY % 2 == 0 &&
                         eZC > 0 && eNS >= 4;
    if (use_env) TY = eTY;
    while (TY > 2 && stage_bytes(g, TY, kappa) * 4 > SMEM_BUDGET) TY -= 2;
    if (stage_bytes(g, TY, kappa) * 4 > SMEM_BUDGET) return false;
    const int tasks = (TY / 2) * ngx;
    const int G = (tasks + NC - 1) / NC;
    if (G > 2) return false;
    int NS = (int)std::min<size_t>(8, SMEM_BUDGET / stage_bytes(g, TY, kappa));
    const int nyt = (int)((g.ny + TY - 1) / TY);
    // z-chunk of at most 32 planes (each chunk stages 2 halo planes and
    // fills and drains its pipeline once): the one whose units spread most
    // evenly over the persistent CTAs, i.e. the smallest per-CTA path
    // ceil(units / SMs) x (ZC + 2) planes, the taller chunk on ties
    // (512^3 heat: 27 planes, 8 full waves, 3.5% faster than 32 planes and
    // 6.7 waves)
    int ZC = (int)std::min<int64_t>(32, g.nz);
    {
        const int64_t nsm = sm_count();
        int64_t best = -1;
        for (int zc = ZC; zc >= std::min(ZC, 8); --zc) {
            const int64_t units = (int64_t)nyt * ((g.nz + zc - 1) / zc);
            const int64_t cost = (units + nsm - 1) / nsm * (zc + 2);
            if (best < 0 || cost < best) {
                best = cost;
                ZC = zc;
            }
        }
    }
    if (use_env) {
        ZC = (int)std::min<int64_t>(eZC, g.nz);
        NS = std::min(eNS, (int)(SMEM_BUDGET / stage_bytes(g, TY, kappa)));
    }
    *c = Cfg{TY, ZC, NS, G};
    return true;
}

template <typename T, bool KAPPA, bool SYM, bool PERIODIC, bool CONS = false, bool RED = false>
cudaError_t launch_t(const Family& f, const SweepArgs& a, cudaStream_t s, double* red = nullptr, int red_cap = 0,
                     int* red_blocks = nullptr)
{
    const Geom& g = f.g;
    const int kmode = CONS ? K_HALO : (KAPPA ? K_TILE : K_NONE);
    Cfg c;
    if (!pick_cfg(g, kmode, &c)) return cudaErrorNotSupported;
    Star1Params P;
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
    P.ZC = c.ZC;
    P.NS = c.NS;
    P.nyt = (int)((g.ny + c.TY - 1) / c.TY);
    P.nzc = (int)((g.nz + c.ZC - 1) / c.ZC);
    P.units = P.nyt * P.nzc;
    P.u_elems = (uint32_t)((c.TY + 2) * g.pitch);
    P.stage_elems = (uint32_t)(stage_bytes(g, c.TY, kmode) / sizeof(T));
    const StarCoef& k = f.sc;
    P.wc = k.c_a;
    P.bc = k.c_b;
    P.wzm = k.a[0][0][0];
    P.wzp = k.a[0][1][0];
    P.wym = k.a[1][0][0];
    P.wyp = k.a[1][1][0];
    P.wxm = k.a[2][0][0];
    P.wxp = k.a[2][1][0];
    P.bzm = k.b[0][0][0];
    P.bzp = k.b[0][1][0];
    P.bym = k.b[1][0][0];
    P.byp = k.b[1][1][0];
    P.bxm = k.b[2][0][0];
    P.bxp = k.b[2][1][0];
    P.status = a.status;
    P.red = red;
    // RED: 3 doubles per consumer warp for the block's combination
    const size_t smem = (size_t)c.NS * P.stage_elems * sizeof(T) + 2 * sizeof(uint64_t) * c.NS +
                        (RED ? 3 * sizeof(double) * consumer_warps<CONS>() : 0);
    static bool attr_set[2] = {false, false};
    auto fn = c.G == 1 ? k_star1<T, KAPPA, SYM, PERIODIC, 1, CONS, RED> : k_star1<T, KAPPA, SYM, PERIODIC, 2, CONS, RED>;
    if (!attr_set[c.G - 1]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr_set[c.G - 1] = true;
    }
    const int grid = (int)std::min<int64_t>(P.units, sm_count());
    if (RED) {
        if (!red || grid > red_cap) return cudaErrorInvalidValue;
        if (red_blocks) *red_blocks = grid;
    }
    return launch_dependent(fn, dim3(grid), dim3(block_threads<CONS>()), smem, s, (const T*)a.in, (T*)a.out,
                            (const T*)a.kappa, P);
}

}  // namespace

bool star3d_supports(const FamilyDesc& d, int* variant, const char** name)
{
    if (d.g.ndim != 3 || d.levels != 1 || !d.star) return false;
    for (int k = 0; k < d.npts; ++k)
        for (int i = 0; i < 3; ++i)
            if (d.off[3 * k + i] > 1 || d.off[3 * k + i] < -1) return false;
    Cfg c;
    if (!pick_cfg(d.g, d.has_beta ? K_TILE : K_NONE, &c)) return false;
    *variant = 1;
    *name = d.has_beta ? "star3d_r1_bulk_kappa" : "star3d_r1_bulk";
    return true;
}

cudaError_t launch_star3d(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    const StarCoef& k = f.sc;
    const bool sym = k.a[0][0][0] == k.a[0][1][0] && k.a[0][0][0] == k.a[1][0][0] && k.a[0][0][0] == k.a[1][1][0] &&
                     k.a[0][0][0] == k.a[2][0][0] && k.a[0][0][0] == k.a[2][1][0] && k.b[0][0][0] == k.b[0][1][0] &&
                     k.b[0][0][0] == k.b[1][0][0] && k.b[0][0][0] == k.b[1][1][0] && k.b[0][0][0] == k.b[2][0][0] &&
                     k.b[0][0][0] == k.b[2][1][0];
    const bool dbl = f.g.esize == 8;
#define ST_DISPATCH(T, KA)                                                                                \
    (sym ? (f.periodic ? launch_t<T, KA, true, true>(f, a, s) : launch_t<T, KA, true, false>(f, a, s))  \
         : (f.periodic ? launch_t<T, KA, false, true>(f, a, s) : launch_t<T, KA, false, false>(f, a, s)))
    if (dbl) return f.has_beta ? ST_DISPATCH(double, true) : ST_DISPATCH(double, false);
    return f.has_beta ? ST_DISPATCH(float, true) : ST_DISPATCH(float, false);
#undef ST_DISPATCH
}

// The sweep fused with the reduction of the level it writes: FP32, constant
// symmetric weights (the 3D heat workloads).
bool star3d_reduce_supported(const Family& f)
{
    if (f.kind != FAM_STAR3D || f.g.esize != 4 || f.has_beta) return false;
    const StarCoef& k = f.sc;
    for (int ax = 0; ax < 3; ++ax)
        for (int sd = 0; sd < 2; ++sd)
            if (k.a[ax][sd][0] != k.a[0][0][0]) return false;
    return true;
}

cudaError_t launch_star3d_reduce(const Family& f, const SweepArgs& a, double* partials, int cap, double* out,
                                 cudaStream_t s)
{
    if (!star3d_reduce_supported(f)) return cudaErrorNotSupported;
    int nb = 0;
    cudaError_t e = f.periodic ? launch_t<float, false, true, true, false, true>(f, a, s, partials, cap, &nb)
                               : launch_t<float, false, true, false, false, true>(f, a, s, partials, cap, &nb);
    if (e != cudaSuccess) return e;
    return launch_reduce_final(partials, nb, out, s);
}

// The conservative face-averaged operator (3D) on the staged pipeline.
bool star3d_cons_supported(const Geom& g)
{
    Cfg c;
    return g.ndim == 3 && pick_cfg(g, K_HALO, &c);
}

cudaError_t launch_star3d_cons(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    if (f.g.esize == 8)
        return f.periodic ? launch_t<double, true, true, true, true>(f, a, s)
                          : launch_t<double, true, true, false, true>(f, a, s);
    return f.periodic ? launch_t<float, true, true, true, true>(f, a, s) : launch_t<float, true, true, false, true>(f, a, s);
}

}  // namespace st
