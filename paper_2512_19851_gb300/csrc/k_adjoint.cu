// Transpose (adjoint) sweep of the per-cell 7-point operator with K steps
// fused per pass, plus the coefficient gradient.
//
// Operator (symmetric star, one coefficient field):
//   w_centre(p) = ac + bc kappa_p,  w_neighbour(p) = an + bn kappa_p
// Transpose step (lambda_in = lambda_{t+1} -> lambda_out = lambda_t):
//   lambda_out[q] = w_c(q) lambda_in[q] + sum_{p nbr of q} w_n(p) lambda_in[p]
// Gradient term of that step:
//   g[q] = lambda_in[q] * (bc u_t[q] + bn sum_{p nbr of q} u_t[p])
//
// Design (HBM-bound; K levels per pass cut the lambda / kappa / gradient
// traffic by K):
//  * CTA tile = TY full rows, streamed through a chunk of z planes; staged per
//    input plane by 1D bulk copies into an mbarrier ring: lambda_{t+1} and
//    kappa with a K-row y halo, and the K states u_t .. u_{t-K+1} with a 1-row
//    halo.  For a Dirichlet boundary the copies are clipped to the ghost shell:
//    positions farther out are never read (see below).
//  * Time-skewed pipeline: at iteration j staged plane j has arrived and level
//    s (= lambda_{t+1-s}) is computed at plane j - s from level s-1 at planes
//    j-s-1 .. j-s+1; intermediate levels live in 3-plane shared rings.  Level
//    s is computed on TY + 2(K-s) rows (the shrinking halo).  Outside the
//    interior (Dirichlet) every level is 0 without reading anything: ghosts
//    are boundary data, not variables.  So no value more than one cell
//    outside the interior is ever read.
//  * The K gradient terms of a point arrive at K consecutive iterations; each
//    thread owns fixed interior points and sums them in a register ring, then
//    adds them to the gradient once per pass.  FP32 grids accumulate into a
//    float-float (hi, lo) scratch with error-free additions (the FP64 pipe of
//    this GPU runs at 1/64 of FP32); FP64 grids accumulate in FP64.
#include <algorithm>
#include <cstring>

#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

constexpr int A_CW = 16;  // consumer warps
constexpr int A_THREADS = (A_CW + 1) * 32;
constexpr int A_NC = A_CW * 32;
constexpr int A_KMAX = 2;
// Slots per intermediate ring: level s+1 reads planes pq-1..pq+1 of level s
// while the next iteration's level s writes plane pq+2; with four slots those
// never share a slot, so one consumer barrier per iteration (between the
// levels) suffices.
constexpr int LSLOTS = 4;

struct AdjParams {
    int64_t nz, ny, nx, pitch, plane, origin;
    int rz, r, xl;
    int TY, ZC, NS;
    int nyt, nzc, units;
    uint32_t stage_elems;                 // per staged plane
    uint32_t lam_off, kap_off, u_off[A_KMAX];  // element offsets inside a stage
    uint32_t g_off;                       // gradient accumulator tile (owned planes only)
    uint32_t ring_elems;                  // one plane of an intermediate level ring
    double ac, bc, an, bn;
    int* status;
};

template <typename T>
struct AV;
template <>
struct AV<float> {
    // two points per thread: twice the threads of four-wide groups for the
    // same tile, for latency hiding, at half the registers per thread
    static constexpr int N = 2;
    typedef float2 type;
};
template <>
struct AV<double> {
    static constexpr int N = 2;
    typedef double2 type;
};

template <typename T>
__device__ __forceinline__ void ald(const T* p, T (&v)[AV<T>::N])
{
    typename AV<T>::type t = *reinterpret_cast<const typename AV<T>::type*>(p);
    v[0] = t.x;
    v[1] = t.y;
}

template <typename T>
__device__ __forceinline__ void ast(T* p, const T (&v)[AV<T>::N])
{
    typename AV<T>::type t;
    t.x = v[0];
    t.y = v[1];
    *reinterpret_cast<typename AV<T>::type*>(p) = t;
}

__device__ __forceinline__ int64_t amin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t amax(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ void atimeout(int* status)
{
    if (status) atomicCAS(status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
}

// Barrier among the consumer warps only (the producer warp has left the
// block's main loop, so __syncthreads would wait for it).
__device__ __forceinline__ void consumer_bar()
{
    asm volatile("bar.sync 1, %0;" ::"r"(A_NC) : "memory");
}

__device__ __forceinline__ void ff_add(float& hi, float& lo, float x)
{
    const float s = hi + x;
    const float bb = s - hi;
    const float e = (hi - (s - bb)) + (x - bb);
    hi = s;
    lo += e;
}

template <typename T, int K, bool PERIODIC>
__global__ void __launch_bounds__(A_THREADS, 1)
k_adjoint(const T* __restrict__ lam_in, T* __restrict__ lam_out, const T* __restrict__ kappa,
          const T* __restrict__ ua, const T* __restrict__ ub, double* __restrict__ g64, float* __restrict__ ghi,
          float* __restrict__ glo, const __grid_constant__ AdjParams P)
{
    constexpr int VN = AV<T>::N;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T* ring = reinterpret_cast<T*>(smem_raw);
    T* lvl = ring + (size_t)P.NS * P.stage_elems;  // (K-1) rings of LSLOTS planes
    uint64_t* full = reinterpret_cast<uint64_t*>(lvl + (size_t)(K - 1) * LSLOTS * P.ring_elems);
    uint64_t* empty = full + P.NS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.NS; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], A_CW);
        }
        ptx::fence_barrier_init();
    }
    // zero the intermediate rings once (their ghost columns stay 0)
    for (size_t i = threadIdx.x; i < (size_t)(K - 1) * LSLOTS * P.ring_elems; i += blockDim.x) lvl[i] = T(0);
    __syncthreads();
    const uint32_t rowb = (uint32_t)(P.pitch * sizeof(T));

    if (warp == A_CW) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        uint32_t gq = 0;
        for (int un = blockIdx.x; un < P.units; un += gridDim.x) {
            const int yt = un % P.nyt, zc = un / P.nyt;
            const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
            const int tye = (int)amin(P.TY, P.ny - y0);
            const int zce = (int)amin(P.ZC, P.nz - z0);
            for (int q = 0; q < zce + 2 * K; ++q, ++gq) {
                const uint32_t s = gq % P.NS, k = gq / P.NS;
                if (k > 0 && !ptx::mbar_wait(&empty[s], (k - 1) & 1)) {
                    atimeout(P.status);
                    return;
                }
                const int64_t zi = z0 - K + q;  // interior plane index of this stage
                T* dst = ring + (size_t)s * P.stage_elems;
                // rows [y0 - h, y0 + tye + h): periodic wraps, Dirichlet clips to the ghost shell
                const bool zin = PERIODIC || (zi >= -P.rz && zi < P.nz + P.rz);
                auto rows_of = [&](int h, int64_t& lo, int64_t& hi) {
                    lo = y0 - h;
                    hi = y0 + tye + h;
                    if (!PERIODIC) {
                        lo = amax(lo, -P.r);
                        hi = amin(hi, P.ny + P.r);
                    }
                };
                uint32_t bytes = 0;
                // the gradient accumulators of the planes this unit owns
                const bool gtile = (g64 != nullptr || ghi != nullptr) && q >= K && q < zce + K;
                const uint32_t growb = (uint32_t)(P.pitch * 8);  // one double or two floats per point
                if (zin) {
                    int64_t lo, hi;
                    rows_of(K, lo, hi);
                    bytes += 2u * (uint32_t)(hi - lo) * rowb;
                    rows_of(1, lo, hi);
                    bytes += (uint32_t)K * (uint32_t)(hi - lo) * rowb;
                }
                if (gtile) bytes += (uint32_t)tye * growb;
                ptx::mbar_arrive_expect_tx(&full[s], bytes);
                if (gtile) {
                    const int64_t goff = P.origin + zi * P.plane + y0 * P.pitch - P.xl;  // row start
                    if (sizeof(T) == 8) {
                        ptx::bulk_g2s(dst + P.g_off, g64 + goff, (uint32_t)tye * growb / 1, &full[s]);
                    } else {
                        float* gd = reinterpret_cast<float*>(dst + P.g_off);
                        ptx::bulk_g2s(gd, ghi + goff, (uint32_t)tye * rowb, &full[s]);
                        ptx::bulk_g2s(gd + (size_t)P.TY * P.pitch, glo + goff, (uint32_t)tye * rowb, &full[s]);
                    }
                }
                if (!zin) continue;
                auto copy = [&](const T* a, T* d, int h) {
                    int64_t lo, hi;
                    rows_of(h, lo, hi);
                    T* dd = d + (size_t)(lo - (y0 - h)) * P.pitch;
                    if (!PERIODIC) {
                        const T* src = a + (zi + P.rz) * P.plane + (lo + P.r) * P.pitch;
                        ptx::bulk_g2s(dd, src, (uint32_t)(hi - lo) * rowb, &full[s]);
                    } else {
                        const int64_t zw = ((zi % P.nz) + P.nz) % P.nz;
                        const T* pl = a + (zw + P.rz) * P.plane + (int64_t)P.r * P.pitch;
                        int j = 0;
                        const int nrows = (int)(hi - lo);
                        while (j < nrows) {
                            int64_t row = lo + j;
                            row = ((row % P.ny) + P.ny) % P.ny;
                            const int run = (int)amin(nrows - j, P.ny - row);
                            ptx::bulk_g2s(dd + (size_t)j * P.pitch, pl + row * P.pitch, (uint32_t)run * rowb,
                                          &full[s]);
                            j += run;
                        }
                    }
                };
                copy(lam_in, dst + P.lam_off, K);
                copy(kappa, dst + P.kap_off, K);
                copy(ua, dst + P.u_off[0], 1);
                if (K > 1) copy(ub, dst + P.u_off[1], 1);
            }
        }
        for (uint32_t d = 0; d < (uint32_t)P.NS && d < gq; ++d) {
            const uint32_t g = gq - 1 - d;
            if (!ptx::mbar_wait(&full[g % P.NS], (g / P.NS) & 1)) atimeout(P.status);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ct = threadIdx.x;
    const int ngx = (int)((P.nx + VN - 1) / VN);
    const T ac = T(P.ac), bc = T(P.bc), an = T(P.an), bn = T(P.bn);
    bool dead = false;  // a bounded wait ran out (warp-uniform)
    uint32_t gq = 0;
    for (int un = blockIdx.x; un < P.units; un += gridDim.x) {
        const int yt = un % P.nyt, zc = un / P.nyt;
        const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
        const int tye = (int)amin(P.TY, P.ny - y0);
        const int zce = (int)amin(P.ZC, P.nz - z0);
        const uint32_t base = gq;
        // this thread's owned interior task (gradient ring) when ct < tye * ngx
        const bool own = ct < tye * ngx;
        // delay lines: dl[s-1][d] holds the level-s gradient term computed d
        // iterations ago (for plane j - s - d); plane j - K is flushed with the
        // terms dl[s-1][K-s], s = 1..K, added one at a time in step order so a
        // fused pass rounds exactly like K single-step passes
        T dl[K][K][VN];
#pragma unroll
        for (int s = 0; s < K; ++s)
#pragma unroll
            for (int d = 0; d < K; ++d)
#pragma unroll
                for (int e = 0; e < VN; ++e) dl[s][d][e] = T(0);

        // running slot and parity of staged plane j (no modulo per lookup);
        // stage(q) for a plane q <= j counts back from it
        uint32_t sj = base % P.NS, pj = (base / P.NS) & 1;
        int jcur = 0;
        auto slot_of = [&](int q) -> uint32_t {
            int sl = (int)sj - (jcur - q);
            while (sl < 0) sl += P.NS;
            return (uint32_t)sl;
        };
        auto stage = [&](int q) -> const T* { return ring + (size_t)slot_of(q) * P.stage_elems; };
        const int nq = zce + 2 * K;
        // task -> (row, x group) per level, fixed for the unit; tasks below
        // tye*ngx are the interior rows (same owner at every level, for the
        // gradient delay lines), the rest the level's halo rows
        int trr[K][2], tgx[K][2];
        bool tval[K][2];
#pragma unroll
        for (int s = 1; s <= K; ++s) {
            const int hs = K - s, rows_s = tye + 2 * hs;
#pragma unroll
            for (int ti = 0; ti < 2; ++ti) {
                const int t = ct + ti * A_NC;
                int rr = 0, gx = 0;
                tval[s - 1][ti] = t < rows_s * ngx;
                if (t < tye * ngx) {
                    rr = t / ngx;
                    gx = t - rr * ngx;
                } else if (tval[s - 1][ti]) {
                    const int h = t - tye * ngx;
                    const int hr = h / ngx;  // 0 .. 2hs-1
                    gx = h - hr * ngx;
                    rr = hr < hs ? -hs + hr : tye + (hr - hs);
                }
                trr[s - 1][ti] = rr;
                tgx[s - 1][ti] = gx;
            }
        }
        for (int j = 0; j < nq; ++j) {
            jcur = j;
            // A wait that runs out is recorded, and the warp carries on without
            // waiting: every consumer warp must keep reaching the named
            // barriers below, which have no time limit of their own.
            if (!dead) {
                if (!ptx::mbar_wait_warp(&full[sj], pj)) {
                    atimeout(P.status);
                    dead = true;
                }
            }
#pragma unroll
            for (int s = 1; s <= K; ++s) {
                const int pq = j - s;  // plane (stage index) of level s this iteration
                if (pq < s || pq > nq - 1 - s) continue;
                const int64_t zabs = z0 - K + pq;
                const int hs = K - s;                  // y halo of level s
                const int rows_s = tye + 2 * hs;
                const bool zout = !PERIODIC && (zabs < 0 || zabs >= P.nz);
                // sources of level s-1 at planes pq-1, pq, pq+1 (row 0 of level s-1 = y0 - (hs + 1))
                const T* src[3];
                int src_h;  // halo of the source arrays
                if (s == 1) {
#pragma unroll
                    for (int d = 0; d < 3; ++d) src[d] = stage(pq - 1 + d) + P.lam_off;
                    src_h = K;
                } else {
#pragma unroll
                    for (int d = 0; d < 3; ++d)
                        src[d] = lvl + (size_t)(s - 2) * LSLOTS * P.ring_elems +
                                 (size_t)((pq - 1 + d) % LSLOTS) * P.ring_elems;
                    src_h = K - s + 1;
                }
                const T* kap[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) kap[d] = stage(pq - 1 + d) + P.kap_off;
                const T* us[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) us[d] = stage(pq - 1 + d) + P.u_off[s - 1];
                T* dst = (s < K) ? lvl + (size_t)(s - 1) * LSLOTS * P.ring_elems + (size_t)(pq % LSLOTS) * P.ring_elems
                                 : nullptr;
#pragma unroll
                for (int ti = 0; ti < 2; ++ti) {
                    if (!tval[s - 1][ti]) continue;
                    const int t = ct + ti * A_NC;
                    const int rr = trr[s - 1][ti];
                    const int x = tgx[s - 1][ti] * VN;
                    const int64_t yabs = y0 + rr;
                    const bool outside = !PERIODIC && (zout || yabs < 0 || yabs >= P.ny);
                    T o[VN];
                    T gterm[VN];
                    if (outside) {
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            o[e] = T(0);
                            gterm[e] = T(0);
                        }
                    } else {
                        const int so = (rr + src_h) * (int)P.pitch + P.xl;   // source row, x = 0
                        const int ko = (rr + K) * (int)P.pitch + P.xl;       // kappa row
                        const int uo = (rr + 1) * (int)P.pitch + P.xl;       // state row
                        const int pt = (int)P.pitch;
                        T lc[VN], ly[VN], lyy[VN], lzm[VN], lzp[VN];
                        T kc[VN], ky[VN], kyy[VN], kzm[VN], kzp[VN];
                        ald(src[1] + so + x, lc);
                        ald(src[1] + so - pt + x, ly);
                        ald(src[1] + so + pt + x, lyy);
                        ald(src[0] + so + x, lzm);
                        ald(src[2] + so + x, lzp);
                        ald(kap[1] + ko + x, kc);
                        ald(kap[1] + ko - pt + x, ky);
                        ald(kap[1] + ko + pt + x, kyy);
                        ald(kap[0] + ko + x, kzm);
                        ald(kap[2] + ko + x, kzp);
                        const T* lrow = src[1] + so;
                        const T* krow = kap[1] + ko;
                        // x neighbours
                        T lxm[VN], lxp[VN], kxm[VN], kxp[VN];
#pragma unroll
                        const int nxi = (int)P.nx;
                        for (int e = 0; e < VN; ++e) {
                            int xm = x + e - 1, xp = x + e + 1;
                            if (PERIODIC) {
                                xm = xm < 0 ? xm + nxi : xm;
                                xp = xp >= nxi ? xp - nxi : xp;
                            }
                            lxm[e] = e > 0 ? lc[e - 1] : lrow[xm];
                            kxm[e] = e > 0 ? kc[e - 1] : krow[xm];
                            lxp[e] = (e < VN - 1 && !(PERIODIC && x + e + 1 == P.nx)) ? lc[e + 1] : lrow[xp];
                            kxp[e] = (e < VN - 1 && !(PERIODIC && x + e + 1 == P.nx)) ? kc[e + 1] : krow[xp];
                        }
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            // transposed step
                            T acc = fma(fma(bc, kc[e], ac), lc[e], T(0));
                            acc = fma(fma(bn, kxm[e], an), lxm[e], acc);
                            acc = fma(fma(bn, kxp[e], an), lxp[e], acc);
                            acc = fma(fma(bn, ky[e], an), ly[e], acc);
                            acc = fma(fma(bn, kyy[e], an), lyy[e], acc);
                            acc = fma(fma(bn, kzm[e], an), lzm[e], acc);
                            acc = fma(fma(bn, kzp[e], an), lzp[e], acc);
                            o[e] = acc;
                        }
                        // gradient term on interior rows of this unit's planes
                        if (rr >= 0 && rr < tye) {
                            T uc[VN], uy[VN], uyy[VN], uzm[VN], uzp[VN];
                            ald(us[1] + uo + x, uc);
                            ald(us[1] + uo - pt + x, uy);
                            ald(us[1] + uo + pt + x, uyy);
                            ald(us[0] + uo + x, uzm);
                            ald(us[2] + uo + x, uzp);
                            const T* urow = us[1] + uo;
#pragma unroll
                            for (int e = 0; e < VN; ++e) {
                                int xm = x + e - 1, xp = x + e + 1;
                                if (PERIODIC) {
                                    xm = xm < 0 ? xm + nxi : xm;
                                    xp = xp >= nxi ? xp - nxi : xp;
                                }
                                const T uxm = e > 0 ? uc[e - 1] : urow[xm];
                                const T uxp = (e < VN - 1 && !(PERIODIC && x + e + 1 == P.nx)) ? uc[e + 1] : urow[xp];
                                const T nb = ((((uxm + uxp) + uy[e]) + uyy[e]) + uzm[e]) + uzp[e];
                                gterm[e] = lc[e] * fma(bc, uc[e], bn * nb);
                            }
                        } else {
#pragma unroll
                            for (int e = 0; e < VN; ++e) gterm[e] = T(0);
                        }
                    }
                    if (s < K) {
                        T* rp = dst + (rr + hs) * (int)P.pitch + P.xl + x;
                        if (x + VN <= P.nx) {
                            ast(rp, o);
                        } else {
                            for (int e = 0; e < VN && x + e < P.nx; ++e) rp[e] = o[e];  // keep ghost columns 0
                        }
                    } else if (!zout && rr >= 0 && rr < tye) {
                        T* op = lam_out + P.origin + zabs * P.plane + (y0 + rr) * P.pitch + x;
                        if (x + VN <= P.nx) {
                            ast(op, o);
                        } else {
                            for (int e = 0; e < VN && x + e < P.nx; ++e) op[e] = o[e];
                        }
                    }
                    // delay line of level s: this term belongs to plane pq (owner threads only)
                    if (t < tye * ngx && own) {
#pragma unroll
                        for (int e = 0; e < VN; ++e) dl[s - 1][0][e] = gterm[e];
                    }
                }
                if (s < K) consumer_bar();  // level s is read by level s + 1 below
            }
            // plane j - K is complete for the owner: flush the K gradient terms once
            {
                const int pq = j - K;
                const int64_t zabs = z0 - K + pq;
                if (own && pq >= K && pq < zce + K && (sizeof(T) == 8 ? g64 != nullptr : ghi != nullptr)) {
                    const int rr = ct / ngx;
                    const int x = (ct - rr * ngx) * VN;
                    const int64_t off = P.origin + zabs * P.plane + (y0 + rr) * P.pitch + x;
                    // the K terms of plane pq, in step order (level 1 = the latest step);
                    // the old accumulator comes from the staged tile of plane pq
                    const T* gst = stage(pq) + P.g_off + rr * (int)P.pitch + P.xl + x;
                    if constexpr (sizeof(T) == 8) {
                        if (x + VN <= P.nx) {
                            double2 gv = *reinterpret_cast<const double2*>(gst);
#pragma unroll
                            for (int s = 1; s <= K; ++s) {
                                gv.x += (double)dl[s - 1][K - s][0];
                                gv.y += (double)dl[s - 1][K - s][1];
                            }
                            *reinterpret_cast<double2*>(g64 + off) = gv;
                        } else {
                            for (int e = 0; e < VN && x + e < P.nx; ++e) {
                                double gv = gst[e];
#pragma unroll
                                for (int s = 1; s <= K; ++s) gv += (double)dl[s - 1][K - s][e];
                                g64[off + e] = gv;
                            }
                        }
                    } else {
                        const float* hs = reinterpret_cast<const float*>(gst);
                        const float* ls = hs + (size_t)P.TY * P.pitch;
                        if (x + VN <= P.nx) {
                            float2 h = *reinterpret_cast<const float2*>(hs);
                            float2 l = *reinterpret_cast<const float2*>(ls);
#pragma unroll
                            for (int s = 1; s <= K; ++s) {
                                ff_add(h.x, l.x, (float)dl[s - 1][K - s][0]);
                                ff_add(h.y, l.y, (float)dl[s - 1][K - s][1]);
                            }
                            *reinterpret_cast<float2*>(ghi + off) = h;
                            *reinterpret_cast<float2*>(glo + off) = l;
                        } else {
                            for (int e = 0; e < VN && x + e < P.nx; ++e) {
                                float h = hs[e], l = ls[e];
#pragma unroll
                                for (int s = 1; s <= K; ++s) ff_add(h, l, (float)dl[s - 1][K - s][e]);
                                ghi[off + e] = h;
                                glo[off + e] = l;
                            }
                        }
                    }
                }
                // age every delay line by one iteration
#pragma unroll
                for (int s = 0; s < K; ++s)
#pragma unroll
                    for (int d = K - 1; d >= 1; --d)
#pragma unroll
                        for (int e = 0; e < VN; ++e) dl[s][d][e] = dl[s][d - 1][e];
#pragma unroll
                for (int s = 0; s < K; ++s)
#pragma unroll
                    for (int e = 0; e < VN; ++e) dl[s][0][e] = T(0);
            }
            // staged plane j-K-1 is no longer needed
            if (j - K - 1 >= 0) {
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&empty[slot_of(j - K - 1)]);
            }
            if (++sj == (uint32_t)P.NS) {
                sj = 0;
                pj ^= 1u;
            }
        }
        // release the planes still held (sj now belongs to plane nq)
        jcur = nq;
        for (int q = (nq - K - 1 > 0 ? nq - K - 1 : 0); q < nq; ++q) {
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[slot_of(q)]);
        }
        gq = base + nq;
    }
}

// gradient fold: grad[p] += hi[p] + lo[p] on the interior (FP32 grids)
__global__ void k_fold_ff(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ grad, Geom g)
{
    const int64_t rows = g.nz * g.ny;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const int64_t z = (uint32_t)row / (uint32_t)g.ny, y = row - z * g.ny;  // 32-bit division
        const int64_t base = g.origin + z * g.plane + y * g.pitch;
        for (int64_t x = threadIdx.x; x < g.nx; x += blockDim.x)
            grad[base + x] += (double)hi[base + x] + (double)lo[base + x];
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
    int K, TY, ZC, NS;
    size_t stage_bytes, ring_bytes;
};

bool adj_cfg(const Geom& g, int kmax, AdjCfg* c)
{
    const int VN = 2;  // AV<T>::N for both types
    const int ngx = (int)((g.nx + VN - 1) / VN);
    const int TY = (int)std::min<int64_t>(std::min(16, A_NC / std::max(1, ngx)), g.ny);
    if (TY < 1) return false;
    for (int K = kmax; K >= 1; --K) {
        if ((TY + 2 * (K - 1)) * ngx > 2 * A_NC) continue;  // at most two tasks per thread and level
        const size_t rows = 2 * (size_t)(TY + 2 * K) + (size_t)K * (TY + 2);
        // + the gradient accumulator tile: TY rows of 8 bytes per point
        const size_t sb = ((rows * g.pitch * g.esize + (size_t)TY * g.pitch * 8) + 127) / 128 * 128;
        const size_t rb = (K > 1) ? (size_t)(K - 1) * LSLOTS * ((size_t)(TY + 2 * (K - 1)) * g.pitch * g.esize) : 0;
        if (rb + (size_t)(K + 3) * sb + 256 > A_SMEM) continue;  // K+2 resident planes + 1 in flight
        const int NS = (int)std::min<size_t>(8, (A_SMEM - rb - 256) / sb);
        const int nyt = (int)((g.ny + TY - 1) / TY);
        const int64_t want = 6LL * adj_sm_count();
        const int64_t nzc = std::max<int64_t>(1, want / nyt);
        int ZC = (int)std::max<int64_t>(8, (g.nz + nzc - 1) / nzc);
        ZC = (int)std::min<int64_t>(ZC, g.nz);
        *c = AdjCfg{K, TY, ZC, NS, sb, rb};
        return true;
    }
    return false;
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
    P.ZC = c.ZC;
    P.NS = c.NS;
    P.nyt = (int)((g.ny + c.TY - 1) / c.TY);
    P.nzc = (int)((g.nz + c.ZC - 1) / c.ZC);
    P.units = P.nyt * P.nzc;
    P.stage_elems = (uint32_t)(c.stage_bytes / sizeof(T));
    P.lam_off = 0;
    P.kap_off = (uint32_t)((c.TY + 2 * K) * g.pitch);
    P.u_off[0] = 2 * P.kap_off;
    P.u_off[1] = P.u_off[0] + (uint32_t)((c.TY + 2) * g.pitch);
    P.g_off = P.u_off[0] + (uint32_t)(K * (c.TY + 2) * g.pitch);
    P.ring_elems = (uint32_t)((c.TY + 2 * (K - 1)) * g.pitch);
    const StarCoef& k = f.sc;
    P.ac = k.c_a;
    P.bc = k.c_b;
    P.an = k.a[0][0][0];
    P.bn = k.b[0][0][0];
    P.status = a.status;
    const size_t smem = c.ring_bytes + (size_t)c.NS * c.stage_bytes + 2 * sizeof(uint64_t) * c.NS;
    auto fn = k_adjoint<T, K, PERIODIC>;
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int grid = (int)std::min<int64_t>(P.units, adj_sm_count());
    fn<<<grid, A_THREADS, smem, s>>>((const T*)a.lam_in, (T*)a.lam_out, (const T*)a.kappa, (const T*)a.u,
                                     (const T*)a.u2, a.gk, a.ghi, a.glo, P);
    return cudaGetLastError();
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
    if (!adj_cfg(f.g, A_KMAX, &c)) return 0;
    return c.K;
}

cudaError_t launch_star3d_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s)
{
    if (star3d_adjoint_fuse(f) < a.steps) return cudaErrorNotSupported;
    AdjCfg c;
    if (!adj_cfg(f.g, a.steps, &c) || c.K != a.steps) return cudaErrorNotSupported;
    const bool dbl = f.g.esize == 8;
    if (a.steps == 2) {
        if (dbl) return f.periodic ? launch_adj_t<double, 2, true>(f, a, c, s) : launch_adj_t<double, 2, false>(f, a, c, s);
        return f.periodic ? launch_adj_t<float, 2, true>(f, a, c, s) : launch_adj_t<float, 2, false>(f, a, c, s);
    }
    if (dbl) return f.periodic ? launch_adj_t<double, 1, true>(f, a, c, s) : launch_adj_t<double, 1, false>(f, a, c, s);
    return f.periodic ? launch_adj_t<float, 1, true>(f, a, c, s) : launch_adj_t<float, 1, false>(f, a, c, s);
}

cudaError_t launch_fold_ff(const float* hi, const float* lo, double* grad, const Geom& g, cudaStream_t s)
{
    const int64_t rows = g.nz * g.ny;
    k_fold_ff<<<(unsigned)std::min<int64_t>(rows, 4096), 256, 0, s>>>(hi, lo, grad, g);
    return cudaGetLastError();
}

}  // namespace st
