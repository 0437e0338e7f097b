// Two sweeps of the constant-weight symmetric 7-point star per pass over HBM
// (temporal blocking; the 3D heat workloads), FP32.
//
//   u_{t+1}[p] = w_c u_t[p] + w_n * (sum of the six neighbours of p)
//
// evaluated exactly as the one-step kernel does (fma(w_c, c, w_n * nb) with
// nb = ((((x-1 + x+1) + y-1) + y+1) + z-1) + z+1), so a pass equals two
// single sweeps bit for bit; only u_t is read and u_{t+2} written, so a pass
// moves 8 bytes per point for two sweeps instead of 16.
//
// Design (the structure of the fused adjoint, without its coefficient field
// and gradient):
//  * A CTA owns TY full rows and streams them through a chunk of z planes; a
//    producer warp stages each plane of u_t with a 2-row y halo into a ring of
//    NS stages by 1D bulk copies completing on mbarriers.  Only the centre
//    plane and the plane above are read at a time; the rest are in flight.
//  * Time skew: at iteration j stage j has arrived, level 1 computes u_{t+1}
//    on the plane of stage j - 1 and level 2 computes u_{t+2} on the plane
//    below it.  Level 1 runs on the tile rows plus one halo row on each side
//    (halo warps) and publishes its rows in a 3-plane shared ring synchronised
//    by full/empty mbarriers; level 2 takes its outer y neighbours from the
//    ring and everything else from registers.
//  * Consumer threads own a pair of rows at one 16-byte x group: the plane
//    below lives in registers (z reuse), the pair shares its inner y
//    neighbours, x edges come from the neighbouring lanes by shuffles (from
//    shared memory at warp and row ends).
//  * Dirichlet: ghost cells keep the boundary value, so level 1 yields that
//    value outside the interior (by selection) and the ring's ghost columns
//    hold it.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

constexpr int P2_MAXCW = 16;                  // consumer warps at most
constexpr int P2_BLOCK = (P2_MAXCW + 1) * 32;  // + the producer warp
constexpr int P2_RING = 3;                    // planes in the level-1 ring
constexpr int VN = 4;                         // floats per 16-byte group

struct Pair2Params {
    int64_t nz, ny, nx, pitch, plane, origin;
    int rz, r, xl;
    int TY, NS, CW;
    int nyt, nzc, units;
    int ngx, npair, pair_warps;
    uint32_t stage_elems, ring_elems;  // a stage: TY + 4 rows; a ring plane: TY + 2 rows
    float wc, wn, bcv;                 // centre weight, neighbour weight, Dirichlet boundary value
    int* status;
};

__device__ __forceinline__ void vld(const float* p, float (&v)[VN])
{
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}

__device__ __forceinline__ int64_t pmin(int64_t a, int64_t b) { return a < b ? a : b; }
__device__ __forceinline__ int64_t pmax(int64_t a, int64_t b) { return a > b ? a : b; }

__device__ __forceinline__ void ptimeout(int* status)
{
    if (status) atomicCAS(status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
}

struct XG {
    int x, nx;
    int cl, cr;        // columns of the left neighbour of element 0 and the right one of element 3
    bool fixl, fixr;   // that neighbour is not held by the adjacent lane
    bool wig;          // periodic row end inside the group: element nx-1-x wraps to column 0
    bool xfull;        // the whole group is interior
};

// One output row group: fma(w_c, c, w_n * nb) with the one-step kernel's
// neighbour order.  `left`/`right` are the values at columns X.cl / X.cr
// when X.fixl / X.fixr; otherwise they come from the adjacent lanes.  All
// lanes of the warp must call it.
__device__ __forceinline__ void point4(const XG& X, float wc, float wn, const float (&v)[VN], const float (&ym)[VN],
                                       const float (&yp)[VN], const float (&zm)[VN], const float (&zp)[VN],
                                       float left, float right, float (&o)[VN])
{
    const float l = __shfl_up_sync(0xffffffffu, v[VN - 1], 1);
    const float r = __shfl_down_sync(0xffffffffu, v[0], 1);
    left = X.fixl ? left : l;
    right = X.fixr ? right : r;
#pragma unroll
    for (int e = 0; e < VN; ++e) {
        const float xm = e == 0 ? left : v[e - 1];
        float xp = e == VN - 1 ? right : v[e + 1];
        if (X.wig && X.x + e + 1 == X.nx) xp = right;
        const float nb = ((((xm + xp) + ym[e]) + yp[e]) + zm[e]) + zp[e];
        o[e] = fmaf(wc, v[e], wn * nb);
    }
}

__device__ __forceinline__ void store4(const XG& X, float* p, const float (&v)[VN])
{
    if (X.xfull) {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    } else {
        for (int e = 0; e < VN && X.x + e < X.nx; ++e) p[e] = v[e];
    }
}

template <bool PERIODIC>
__global__ void __launch_bounds__(P2_BLOCK, 1)
k_star2(const float* __restrict__ in, float* __restrict__ out, const __grid_constant__ Pair2Params P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* stg = reinterpret_cast<float*>(smem_raw);
    float* ring = stg + (size_t)P.NS * P.stage_elems;
    uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)P2_RING * P.ring_elems);
    uint64_t* empty = full + P.NS;
    uint64_t* rfull = empty + P.NS;      // a ring plane is written (one arrival per consumer warp)
    uint64_t* rempty = rfull + P2_RING;  // a ring plane is read
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < P.NS; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], P.CW);
        }
        for (int s = 0; s < P2_RING; ++s) {
            ptx::mbar_init(&rfull[s], P.CW);
            ptx::mbar_init(&rempty[s], P.CW);
        }
        ptx::fence_barrier_init();
    }
    // the ring's ghost columns hold the boundary value for good (only interior
    // columns are written)
    const float ghost = PERIODIC ? 0.f : P.bcv;
    for (size_t i = threadIdx.x; i < (size_t)P2_RING * P.ring_elems; i += blockDim.x) ring[i] = ghost;
    __syncthreads();
    ptx::griddep_wait();  // earlier kernels of the stream wrote our inputs / read our outputs
    ptx::griddep_trigger();
    const uint32_t rowb = (uint32_t)(P.pitch * sizeof(float));

    if (warp == P.CW) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        uint32_t gq = 0;
        for (int un = blockIdx.x; un < P.units; un += gridDim.x) {
            const int yt = un % P.nyt, zc = un / P.nyt;
            const int64_t y0 = (int64_t)yt * P.TY;
            const int tye = (int)pmin(P.TY, P.ny - y0);
            const int64_t z0 = (int64_t)zc * P.nz / P.nzc, z1 = (int64_t)(zc + 1) * P.nz / P.nzc;
            const int nq = (int)(z1 - z0) + 4;
            // rows [y0 - 2, y0 + tye + 2): periodic wraps, Dirichlet clips to the ghost shell
            int64_t lo = y0 - 2, hi = y0 + tye + 2;
            if (!PERIODIC) {
                lo = pmax(lo, -P.r);
                hi = pmin(hi, P.ny + P.r);
            }
            const uint32_t bytes = (uint32_t)(hi - lo) * rowb;
            for (int q = 0; q < nq; ++q, ++gq) {
                const uint32_t s = gq % P.NS, k = gq / P.NS;
                if (k > 0 && !ptx::mbar_wait(&empty[s], (k - 1) & 1)) {
                    ptimeout(P.status);
                    return;
                }
                const int64_t zi = z0 - 2 + q;
                const bool okz = PERIODIC || (zi >= -P.rz && zi < P.nz + P.rz);
                ptx::mbar_arrive_expect_tx(&full[s], okz ? bytes : 0u);
                if (!okz) continue;
                float* dd = stg + (size_t)s * P.stage_elems + (size_t)(lo - (y0 - 2)) * P.pitch;
                if (!PERIODIC) {
                    ptx::bulk_g2s(dd, in + (zi + P.rz) * P.plane + (lo + P.r) * P.pitch, bytes, &full[s]);
                } else {
                    const int64_t zw = ((zi % P.nz) + P.nz) % P.nz;
                    const float* pl = in + (zw + P.rz) * P.plane + (int64_t)P.r * P.pitch;
                    const int nrows = (int)(hi - lo);
                    int jr = 0;
                    while (jr < nrows) {
                        int64_t row = lo + jr;
                        row = ((row % P.ny) + P.ny) % P.ny;
                        const int run = (int)pmin(nrows - jr, P.ny - row);
                        ptx::bulk_g2s(dd + (size_t)jr * P.pitch, pl + row * P.pitch, (uint32_t)run * rowb, &full[s]);
                        jr += run;
                    }
                }
            }
        }
        for (uint32_t d = 0; d < (uint32_t)P.NS && d < gq; ++d) {
            const uint32_t g = gq - 1 - d;
            if (!ptx::mbar_wait(&full[g % P.NS], (g / P.NS) & 1)) ptimeout(P.status);
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
    } else {
        // both halo rows (above and below the tile) of one x group
        const int t = threadIdx.x - 32 * P.pair_warps;
        act = t < ngx;
        if (act) gx = t;
    }
    XG X;
    X.nx = (int)P.nx;
    X.x = gx * VN;
    X.fixl = lane == 0 || gx == 0;
    X.fixr = lane == 31 || gx == ngx - 1;
    X.wig = PERIODIC && X.x + VN > X.nx;
    X.cl = X.x > 0 ? X.x - 1 : (PERIODIC ? X.nx - 1 : -1);
    X.cr = X.x + VN >= X.nx ? (PERIODIC ? 0 : X.nx) : X.x + VN;
    X.xfull = X.x + VN <= X.nx;
    const int x = X.x;
    const float wc = P.wc, wn = P.wn;

    bool dead = false;
    uint32_t gq = 0, gr = 0;
    for (int un = blockIdx.x; un < P.units; un += gridDim.x) {
        const int yt = un % P.nyt, zc = un / P.nyt;
        const int64_t y0 = (int64_t)yt * P.TY;
        const int tye = (int)pmin(P.TY, P.ny - y0);
        const int64_t z0 = (int64_t)zc * P.nz / P.nzc, z1 = (int64_t)(zc + 1) * P.nz / P.nzc;
        const int nq = (int)(z1 - z0) + 4;
        const uint32_t base = gq, rbase = gr;
        uint32_t sj = base % P.NS, pj = (base / P.NS) & 1, sp = 0;
        const int rr0 = 2 * rp;
        // carried (registers, per owned row): u_t of the plane below the level-1
        // centre; u_{t+1} of the planes below and at the level-2 centre
        float u0p[2][VN], m1a[2][VN], m1b[2][VN], m1n[2][VN];
#pragma unroll
        for (int i = 0; i < 2; ++i)
#pragma unroll
            for (int e = 0; e < VN; ++e) u0p[i][e] = m1a[i][e] = m1b[i][e] = m1n[i][e] = 0.f;

        for (int j = 0; j < nq; ++j) {
            if (!dead && !ptx::mbar_wait_warp(&full[sj], pj)) {
                ptimeout(P.status);
                dead = true;
            }
            const float* S1 = stg + (size_t)sj * P.stage_elems + P.xl;  // plane above the level-1 centre
            const float* S0 = stg + (size_t)sp * P.stage_elems + P.xl;  // level-1 centre plane
            const int64_t c1 = z0 - 3 + j;                                // level-1 centre plane (j >= 2)
            const bool zout1 = !PERIODIC && (c1 < 0 || c1 >= P.nz);
            const uint32_t wn_ = rbase + (uint32_t)j - 2u, wslot = wn_ % P2_RING;
            if (j >= 2 && wn_ >= (uint32_t)P2_RING && !dead &&
                !ptx::mbar_wait_warp(&rempty[wslot], (wn_ / P2_RING - 1u) & 1u)) {
                ptimeout(P.status);
                dead = true;
            }
            float* RW = ring + (size_t)wslot * P.ring_elems + P.xl;  // ring plane written now (row -1 first)

            if (pairw) {
                // ------------------------------------------------ row pair, level 1
                const float* L = S0 + (rr0 + 1) * pitch;  // stage row of tile row rr0 - 1
                if (j == 1) {
#pragma unroll
                    for (int i = 0; i < 2; ++i) vld(L + (i + 1) * pitch + x, u0p[i]);
                } else if (j >= 2) {
                    float v[4][VN], vz[2][VN];
#pragma unroll
                    for (int i = 0; i < 4; ++i) vld(L + i * pitch + x, v[i]);
#pragma unroll
                    for (int i = 0; i < 2; ++i) vld(S1 + (rr0 + 2 + i) * pitch + x, vz[i]);
#pragma unroll
                    for (int i = 0; i < 2; ++i) {
                        const float* Lr = L + (i + 1) * pitch;
                        float left = 0.f, right = 0.f;
                        if (X.fixl) left = Lr[X.cl];
                        if (X.fixr) right = Lr[X.cr];
                        float o[VN];
                        point4(X, wc, wn, v[i + 1], v[i], v[i + 2], u0p[i], vz[i], left, right, o);
                        const bool out1 = zout1 || (!PERIODIC && y0 + rr0 + i >= P.ny);
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            float u1 = out1 ? P.bcv : o[e];
                            if (!PERIODIC && x + e >= X.nx) u1 = P.bcv;  // ghost column of a ragged group
                            m1n[i][e] = u1;
                            u0p[i][e] = v[i + 1][e];
                        }
                        if (act && rr0 + i < tye) store4(X, RW + (rr0 + 1 + i) * pitch + x, m1n[i]);
                    }
                }
            } else {
                // ------------------------------------------------ halo rows, level 1 only
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const int rh = i == 0 ? -1 : tye;
                    const float* L = S0 + (rh + 1) * pitch;  // stage row of tile row rh - 1
                    if (j == 1) {
                        vld(L + pitch + x, u0p[i]);
                    } else if (j >= 2) {
                        float v[3][VN], vz[VN];
#pragma unroll
                        for (int r3 = 0; r3 < 3; ++r3) vld(L + r3 * pitch + x, v[r3]);
                        vld(S1 + (rh + 2) * pitch + x, vz);
                        const float* Lr = L + pitch;
                        float left = 0.f, right = 0.f;
                        if (X.fixl) left = Lr[X.cl];
                        if (X.fixr) right = Lr[X.cr];
                        float o[VN];
                        point4(X, wc, wn, v[1], v[0], v[2], u0p[i], vz, left, right, o);
                        const int64_t yabs = y0 + rh;
                        const bool out1 = zout1 || (!PERIODIC && (yabs < 0 || yabs >= P.ny));
#pragma unroll
                        for (int e = 0; e < VN; ++e) {
                            o[e] = out1 ? P.bcv : o[e];
                            u0p[i][e] = v[1][e];
                        }
                        if (act) store4(X, RW + (rh + 1) * pitch + x, o);
                    }
                }
            }
            if (j >= 2) {  // this warp's rows of the ring plane are written
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&rfull[wslot]);
            }

            // ---------------------------------------------------- row pair, level 2
            const uint32_t rn = rbase + (uint32_t)j - 3u, rslot = rn % P2_RING;
            if (pairw && j >= 4) {
                if (!dead && !ptx::mbar_wait_warp(&rfull[rslot], (rn / P2_RING) & 1u)) {
                    ptimeout(P.status);
                    dead = true;
                }
                const int64_t c2 = c1 - 1;
                const float* M = ring + (size_t)rslot * P.ring_elems + P.xl + rr0 * pitch;  // ring row rr0 - 1
                float mup[VN], mdn[VN];
                vld(M + x, mup);
                vld(M + 3 * pitch + x, mdn);
#pragma unroll
                for (int i = 0; i < 2; ++i) {
                    const float* Mr = M + (i + 1) * pitch;
                    float left = 0.f, right = 0.f;
                    if (X.fixl) left = Mr[X.cl];
                    if (X.fixr) right = Mr[X.cr];
                    float o[VN];
                    point4(X, wc, wn, m1b[i], i == 0 ? mup : m1b[0], i == 0 ? m1b[1] : mdn, m1a[i], m1n[i], left,
                           right, o);
                    if (act && rr0 + i < tye)
                        store4(X, out + P.origin + c2 * P.plane + (y0 + rr0 + i) * P.pitch + x, o);
                }
            }
            if (pairw && j >= 2) {
#pragma unroll
                for (int i = 0; i < 2; ++i)
#pragma unroll
                    for (int e = 0; e < VN; ++e) {
                        m1a[i][e] = m1b[i][e];
                        m1b[i][e] = m1n[i][e];
                    }
            }
            if (j >= 3) {  // done with the previous ring plane (halo warps never read it)
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&rempty[rslot]);
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
            // the unit's last ring plane has no reader: release it as read
            ptx::mbar_arrive(&rempty[(rbase + (uint32_t)nq - 3u) % P2_RING]);
        }
        gq = base + nq;
        gr = rbase + (uint32_t)nq - 2u;
    }
}

int p2_sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

constexpr size_t P2_SMEM = 220 * 1024;

struct P2Cfg {
    int TY, NS, CW, pair_warps, npair, nzc;
    size_t stage_bytes, ring_bytes;
};

// Tallest even tile that one task per consumer thread covers (at most 16
// warps, halo tasks included) with at least 4 stages (2 in flight).
bool p2_cfg(const Geom& g, P2Cfg* c)
{
    if (g.esize != 4 || g.ndim != 3 || g.r != 1) return false;
    const int ngx = (int)((g.nx + VN - 1) / VN);
    const size_t rowb = (size_t)g.pitch * 4;
    int eTY = 0, eNS = 0, eNZC = 0;
    const char* env = std::getenv("ST_STAR2_CFG");  // "TY,NS,nzc" for tuning sweeps
    const bool use_env = env && std::sscanf(env, "%d,%d,%d", &eTY, &eNS, &eNZC) == 3 && eTY >= 2 && eTY % 2 == 0 &&
                         eNS >= 3 && eNZC >= 1;
    P2Cfg best{};
    bool have = false;
    for (int TY = 16; TY >= 2 && !have; TY -= 2) {
        if (use_env && TY != eTY) continue;
        if (TY > 2 && TY - 2 >= g.ny) continue;
        const int npair = (TY / 2) * ngx;
        const int pw = (npair + 31) / 32, hw = (ngx + 31) / 32;
        if (pw + hw > P2_MAXCW) continue;
        const size_t sb = ((size_t)(TY + 4) * rowb + 127) / 128 * 128;
        const size_t rb = (size_t)P2_RING * (TY + 2) * rowb;
        const size_t fixed = rb + 512;
        if (fixed + 4 * sb > P2_SMEM) continue;
        int NS = (int)std::min<size_t>(8, (P2_SMEM - fixed) / sb);
        if (use_env) NS = std::min(NS, eNS);
        best = P2Cfg{TY, NS, pw + hw, pw, npair, 1, sb, rb};
        have = true;
    }
    if (!have) return false;
    // z chunks: balance the per-CTA critical path against the 4 extra planes each chunk stages
    const int nyt = (int)((g.ny + best.TY - 1) / best.TY);
    const int64_t nsm = p2_sm_count();
    double bestcost = 1e300;
    for (int64_t nzc = 1; nzc <= g.nz; ++nzc) {
        const int64_t units = nyt * nzc;
        const int64_t zmax = (g.nz + nzc - 1) / nzc;
        const double waves = (double)((units + nsm - 1) / nsm);
        const double cost = std::max(waves * (double)(zmax + 4), (double)nyt * (double)(g.nz + 4 * nzc) / (double)nsm);
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

}  // namespace

bool star3d_pair_supported(const Family& f)
{
    if (f.kind != FAM_STAR3D || f.has_beta || f.levels != 1) return false;
    const StarCoef& k = f.sc;
    for (int ax = 0; ax < 3; ++ax)
        for (int sd = 0; sd < 2; ++sd)
            if (k.a[ax][sd][0] != k.a[0][0][0]) return false;
    P2Cfg c;
    return p2_cfg(f.g, &c);
}

cudaError_t launch_star3d_pair(const Family& f, const SweepArgs& a, double bc_value, cudaStream_t s)
{
    const Geom& g = f.g;
    P2Cfg c;
    if (!star3d_pair_supported(f) || !p2_cfg(g, &c)) return cudaErrorNotSupported;
    Pair2Params P;
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
    P.ngx = (int)((g.nx + VN - 1) / VN);
    P.npair = c.npair;
    P.pair_warps = c.pair_warps;
    P.stage_elems = (uint32_t)(c.stage_bytes / 4);
    P.ring_elems = (uint32_t)((c.TY + 2) * g.pitch);
    P.wc = (float)f.sc.c_a;
    P.wn = (float)f.sc.a[0][0][0];
    P.bcv = (float)bc_value;
    P.status = a.status;
    const size_t smem = c.ring_bytes + (size_t)c.NS * c.stage_bytes + sizeof(uint64_t) * (2 * c.NS + 2 * P2_RING);
    auto fn = f.periodic ? k_star2<true> : k_star2<false>;
    static bool attr[2] = {false, false};
    if (!attr[f.periodic ? 1 : 0]) {
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr[f.periodic ? 1 : 0] = true;
    }
    const int grid = (int)std::min<int64_t>(P.units, p2_sm_count());
    return launch_dependent(fn, dim3(grid), dim3((c.CW + 1) * 32), smem, s, (const float*)a.in, (float*)a.out, P);
}

}  // namespace st
