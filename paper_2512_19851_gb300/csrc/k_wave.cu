// 3D radius-4 star in the two-level (leapfrog) form with a per-cell factor:
//   u^{n+1}[p] = sum_k (alpha_k + beta_k m_p) u^n[p + o_k] - u^{n-1}[p] + s_n [p == src]
// (the acoustic wave workload: alpha = 2 at the centre, beta = 8th-order
// second-difference coefficients, m = (c dt / h)^2).  FP32.
//
// Design:
//  * CTA tile = TY full rows, streamed through a chunk of z planes.  Plane
//    tiles of u^n with a 4-row y halo are staged in shared memory by 1D bulk
//    copies (TMA) into an NS-stage mbarrier ring filled by a producer warp.
//  * z neighbours come from a per-thread register queue: each thread owns one
//    4-wide x group and keeps u^n at z-4..z+4 for it; a plane enters the queue
//    when it arrives (as z+4) and leaves it 9 planes later.  Only the centre
//    plane's x and y neighbours are read from shared memory, so the ring must
//    hold planes z..z+4 (5 stages) plus the ones in flight.
//  * m and u^{n-1} are needed only at the point: their plane tiles (TY rows,
//    no halo) travel through a second, short bulk-copy ring with its own
//    barriers, so no global load is ever waited on by the consumers.  u^{n+1}
//    overwrites u^{n-1} in place (every point's u^{n-1} is staged before the
//    point is written, and no other CTA reads it).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

constexpr int WR = 4;              // radius
constexpr int W_CWARPS = 16;       // consumer warps
constexpr int W_THREADS = (W_CWARPS + 1) * 32;
constexpr int W_NC = W_CWARPS * 32;

struct WaveParams {
    int64_t nz, ny, nx, pitch, plane, origin;
    int rz, r, xl;
    int TY, ZC, NS, NSM;  // u-ring and (m, u^{n-1})-ring stages
    int nyt, nzc, units;
    uint32_t stage_elems;    // u stage
    uint32_t mstage_elems;   // (m, u^{n-1}) stage: m rows then u^{n-1} rows
    // coefficients: alpha/beta of the centre and of distance j (symmetric star)
    float ac, bc;
    float aj[WR], bj[WR];
    // source
    int64_t sz, sy, sx;     // interior coordinates of the source, sz < 0: none
    const double* src_amp;  // device amplitudes
    int64_t step;           // step index of this launch
    int* status;
};

__device__ __forceinline__ int64_t wrapw(int64_t i, int64_t n)
{
    i = i < 0 ? i + n : i;
    return i >= n ? i - n : i;
}

__device__ __forceinline__ int64_t imin_w(int64_t a, int64_t b) { return a < b ? a : b; }

__device__ __forceinline__ void timeout(int* status)
{
    if (status) atomicCAS(status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
}

template <bool PERIODIC, bool ALPHA0>
__global__ void __launch_bounds__(W_THREADS, 1)
k_wave(const float* __restrict__ un, float* uprev_out, const float* __restrict__ m, const __grid_constant__ WaveParams P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    float* mring = ring + (size_t)P.NS * P.stage_elems;
    uint64_t* full = reinterpret_cast<uint64_t*>(mring + (size_t)P.NSM * P.mstage_elems);
    uint64_t* empty = full + P.NS;
    uint64_t* mfull = empty + P.NS;
    uint64_t* mempty = mfull + P.NSM;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.NS; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], W_CWARPS);
        }
        for (int s = 0; s < P.NSM; ++s) {
            ptx::mbar_init(&mfull[s], 1);
            ptx::mbar_init(&mempty[s], W_CWARPS);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();
    ptx::griddep_wait();  // earlier kernels of the stream wrote our inputs / read our outputs
    ptx::griddep_trigger();
    const uint32_t rowb = (uint32_t)(P.pitch * sizeof(float));
    const int H = 2 * WR;  // halo rows per tile

    if (warp == W_CWARPS) {
        // ------------------------------------------------------------ producer
        if (lane != 0) return;
        uint32_t gq = 0, gm = 0;
        for (int u = blockIdx.x; u < P.units; u += gridDim.x) {
            const int yt = u % P.nyt, zc = u / P.nyt;
            const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
            const int tye = (int)imin_w(P.TY, P.ny - y0);
            const int zce = (int)imin_w(P.ZC, P.nz - z0);
            auto issue_u = [&](int q) -> bool {  // u^n plane z0 - 4 + q with a 4-row halo
                const uint32_t s = gq % P.NS, k = gq / P.NS;
                if (k > 0 && !ptx::mbar_wait(&empty[s], (k - 1) & 1)) return false;
                const int64_t zi = z0 - WR + q;
                float* dst = ring + (size_t)s * P.stage_elems;
                ptx::mbar_arrive_expect_tx(&full[s], (uint32_t)(tye + H) * rowb);
                if (!PERIODIC) {
                    const float* src = un + (zi + P.rz) * P.plane + (y0 - WR + P.r) * P.pitch;
                    ptx::bulk_g2s(dst, src, (uint32_t)(tye + H) * rowb, &full[s]);
                } else {
                    const float* pl = un + (((zi % P.nz) + P.nz) % P.nz + P.rz) * P.plane + (int64_t)P.r * P.pitch;
                    int j = 0;
                    while (j < tye + H) {
                        int64_t row = y0 - WR + j;
                        row = ((row % P.ny) + P.ny) % P.ny;
                        const int run = (int)imin_w(tye + H - j, P.ny - row);
                        ptx::bulk_g2s(dst + (size_t)j * P.pitch, pl + row * P.pitch, (uint32_t)run * rowb, &full[s]);
                        j += run;
                    }
                }
                ++gq;
                return true;
            };
            auto issue_m = [&](int i) -> bool {  // m and u^{n-1} of output plane z0 + i
                const uint32_t s = gm % P.NSM, k = gm / P.NSM;
                if (k > 0 && !ptx::mbar_wait(&mempty[s], (k - 1) & 1)) return false;
                const int64_t off = (z0 + i + P.rz) * P.plane + (y0 + P.r) * P.pitch;
                float* dst = mring + (size_t)s * P.mstage_elems;
                ptx::mbar_arrive_expect_tx(&mfull[s], 2u * (uint32_t)tye * rowb);
                ptx::bulk_g2s(dst, m + off, (uint32_t)tye * rowb, &mfull[s]);
                ptx::bulk_g2s(dst + (size_t)P.TY * P.pitch, uprev_out + off, (uint32_t)tye * rowb, &mfull[s]);
                ++gm;
                return true;
            };
            bool ok = true;
            for (int q = 0; q < 2 * WR && ok; ++q) ok = issue_u(q);
            for (int i = 0; i < zce && ok; ++i) ok = issue_m(i) && issue_u(i + 2 * WR);
            if (!ok) {
                timeout(P.status);
                return;
            }
        }
        for (uint32_t d = 0; d < (uint32_t)P.NS && d < gq; ++d) {
            const uint32_t g = gq - 1 - d;
            if (!ptx::mbar_wait(&full[g % P.NS], (g / P.NS) & 1)) timeout(P.status);
        }
        for (uint32_t d = 0; d < (uint32_t)P.NSM && d < gm; ++d) {
            const uint32_t g = gm - 1 - d;
            if (!ptx::mbar_wait(&mfull[g % P.NSM], (g / P.NSM) & 1)) timeout(P.status);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ct = threadIdx.x;
    const int ngx = (int)((P.nx + 3) / 4);
    const float bj[WR] = {P.bj[0], P.bj[1], P.bj[2], P.bj[3]};
    const float aj[WR] = {P.aj[0], P.aj[1], P.aj[2], P.aj[3]};
    // Shared memory addressed by 32-bit indices in 16-byte units: stage s of
    // the u ring starts at s * st4, stage s of the (m, u^{n-1}) ring at
    // mr4 + s * mst4 (every stage, row and group start is 16-byte aligned).
    const float4* S4 = reinterpret_cast<const float4*>(smem_raw);
    const uint32_t st4 = P.stage_elems / 4u, mst4 = P.mstage_elems / 4u;
    const uint32_t mr4 = (uint32_t)P.NS * st4;
    const uint32_t pitch4 = (uint32_t)P.pitch / 4u;
    uint32_t gq = 0, gm = 0;
    for (int u = blockIdx.x; u < P.units; u += gridDim.x) {
        const int yt = u % P.nyt, zc = u / P.nyt;
        const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
        const int tye = (int)imin_w(P.TY, P.ny - y0);
        const int zce = (int)imin_w(P.ZC, P.nz - z0);
        const uint32_t base = gq, mbase = gm;
        const bool active = ct < tye * ngx;
        const int row = active ? ct / ngx : 0;
        const int x = active ? (ct - row * ngx) * 4 : 0;
        const bool full4 = x + 4 <= P.nx;
        // A Dirichlet row's ghost columns (4 of them, and the pitch padding)
        // follow it in the staged copy, so 16-byte loads of a ragged last group
        // stay inside the row and its in-range points see the right
        // neighbours; only a periodic ragged group must gather wrapped ones.
        const bool fast = full4 || !PERIODIC;
        const int64_t gofs = P.origin + (y0 + row) * P.pitch + x;  // + z * plane
        const bool src_here = active && P.sz >= 0 && P.sy == y0 + row && P.sx >= x && P.sx < x + 4;
        // this thread's group in a u stage (its centre row) and in an (m, u^{n-1}) stage
        const uint32_t t4 = (uint32_t)((P.xl + (row + WR) * P.pitch + x) / 4);
        const uint32_t m4 = (uint32_t)((P.xl + row * P.pitch + x) / 4);
        const uint32_t prev4 = (uint32_t)(P.TY * P.pitch / 4);  // u^{n-1} rows follow the m rows
        // z queue: before output plane i, q[0 .. 7] hold the group at planes
        // i .. i + 7 of the chunk (z - 4 .. z + 3 of the output); the step
        // for a window w (= q or q + 1) takes plane i + 8 into w[8]
        float4 q[2 * WR + 2];

        auto wait_plane = [&](int qq) -> bool {
            const uint32_t g = base + qq;
            return ptx::mbar_wait_warp(&full[g % P.NS], (g / P.NS) & 1);
        };
        // plane q is a centre (output z0 + q - 4) for q in [4, zce + 4); all
        // other planes of the chunk only feed the z queues
        auto is_centre = [&](int qq) -> bool { return qq >= WR && qq < zce + WR; };
        // prime: planes z0-4 .. z0+3 (q = 0..7)
#pragma unroll
        for (int qq = 0; qq < 2 * WR; ++qq) {
            if (!wait_plane(qq)) {
                timeout(P.status);
                return;
            }
            q[qq] = active ? S4[((base + qq) % P.NS) * st4 + t4] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (!is_centre(qq)) {
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&empty[(base + qq) % P.NS]);
            }
        }
        // running ring slots (no modulo per plane): the centre plane i + 4,
        // the incoming plane i + 8 with its phase parity, and the (m, u^{n-1})
        // stage of output i with its parity
        uint32_t s_c = (base + WR) % P.NS, s_n = (base + 2 * WR) % P.NS, p_n = ((base + 2 * WR) / P.NS) & 1;
        uint32_t s_m = mbase % P.NSM, p_m = (mbase / P.NSM) & 1;
        // one output plane i from window w; false when a wait ran out
        auto step = [&](float4* w, int i) -> bool {
            if (!ptx::mbar_wait_warp(&full[s_n], p_n) || !ptx::mbar_wait_warp(&mfull[s_m], p_m)) {
                timeout(P.status);
                return false;
            }
            if (active) w[2 * WR] = S4[s_n * st4 + t4];
            if (!is_centre(i + 2 * WR)) {
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&empty[s_n]);
            }
            if (active) {
                const uint32_t mb = mr4 + s_m * mst4 + m4;
                const float4 mv = S4[mb];
                const float4 pv = S4[mb + prev4];
                const uint32_t cb = s_c * st4 + t4;  // centre plane, own group of the centre row
                const float c[4] = {w[WR].x, w[WR].y, w[WR].z, w[WR].w};
                // running sums per point: lb = sum_k beta_k u_k, la = sum_{k != 0} alpha_k u_k
                float lb[4], la[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    lb[e] = P.bc * c[e];
                    la[e] = 0.f;
                }
                // coefficient of distance j by register selects (j may be a loop
                // variable: indexing a local array with it would go to local memory)
                auto cb_ = [&](int j) { return j == 1 ? bj[0] : (j == 2 ? bj[1] : (j == 3 ? bj[2] : bj[3])); };
                auto ca_ = [&](int j) { return j == 1 ? aj[0] : (j == 2 ? aj[1] : (j == 3 ? aj[2] : aj[3])); };
                auto add_pair = [&](int j, int e, float s2) {  // the two neighbours at distance j
                    lb[e] = fmaf(cb_(j), s2, lb[e]);
                    if (!ALPHA0) la[e] = fmaf(ca_(j), s2, la[e]);
                };
#pragma unroll
                for (int j = 1; j <= WR; ++j) {  // z neighbours from the register queue
                    const float4 zl = w[WR - j], zh = w[WR + j];
                    add_pair(j, 0, zl.x + zh.x);
                    add_pair(j, 1, zl.y + zh.y);
                    add_pair(j, 2, zl.z + zh.z);
                    add_pair(j, 3, zl.w + zh.w);
                }
                if (fast) {
#pragma unroll
                    for (int j = 1; j <= WR; ++j) {  // y neighbours
                        const float4 yl = S4[cb - j * pitch4];
                        const float4 yh = S4[cb + j * pitch4];
                        add_pair(j, 0, yl.x + yh.x);
                        add_pair(j, 1, yl.y + yh.y);
                        add_pair(j, 2, yl.z + yh.z);
                        add_pair(j, 3, yl.w + yh.w);
                    }
                    // x window: 4 left, the group, 4 right (16-byte groups of the
                    // row); a periodic window that wraps is gathered element-wise
                    float4 L, R;
                    const float* rc = reinterpret_cast<const float*>(S4 + cb) - x;  // column 0 of the centre row
                    if (PERIODIC && x == 0)
                        L = make_float4(rc[wrapw(x - 4, P.nx)], rc[wrapw(x - 3, P.nx)], rc[wrapw(x - 2, P.nx)],
                                        rc[wrapw(x - 1, P.nx)]);
                    else
                        L = S4[cb - 1];
                    if (PERIODIC && x + 8 > P.nx)
                        R = make_float4(rc[wrapw(x + 4, P.nx)], rc[wrapw(x + 5, P.nx)], rc[wrapw(x + 6, P.nx)],
                                        rc[wrapw(x + 7, P.nx)]);
                    else
                        R = S4[cb + 1];
                    const float wx[12] = {L.x, L.y, L.z, L.w, c[0], c[1], c[2], c[3], R.x, R.y, R.z, R.w};
#pragma unroll
                    for (int j = 1; j <= WR; ++j)
#pragma unroll
                        for (int e = 0; e < 4; ++e) add_pair(j, e, wx[4 + e - j] + wx[4 + e + j]);
                } else {
                    const float* rc = reinterpret_cast<const float*>(S4 + cb) - x;  // column 0 of the centre row
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int64_t xe = x + e;
                        if (xe >= P.nx) break;
#pragma unroll
                        for (int j = 1; j <= WR; ++j) {
                            const float yl = rc[xe - j * P.pitch], yh = rc[xe + j * P.pitch];
                            const int64_t xm = PERIODIC ? wrapw(xe - j, P.nx) : xe - j;
                            const int64_t xp = PERIODIC ? wrapw(xe + j, P.nx) : xe + j;
                            add_pair(j, e, yl + yh);
                            add_pair(j, e, rc[xm] + rc[xp]);
                        }
                    }
                }
                const float mm[4] = {mv.x, mv.y, mv.z, mv.w};
                const float pp[4] = {pv.x, pv.y, pv.z, pv.w};
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) o[e] = fmaf(mm[e], lb[e], fmaf(P.ac, c[e], -pp[e]) + la[e]);
                const int64_t z = z0 + i;
                if (src_here && P.sz == z) {
                    const float amp = (float)P.src_amp[P.step];
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (P.sx - x == e) o[e] += amp;
                }
                float* op = uprev_out + gofs + z * P.plane;
                if (full4) {
                    *reinterpret_cast<float4*>(op) = make_float4(o[0], o[1], o[2], o[3]);
                } else {
                    for (int e = 0; e < 4 && x + e < P.nx; ++e) op[e] = o[e];
                }
            }
            __syncwarp();
            if (lane == 0) {
                ptx::mbar_arrive(&empty[s_c]);  // centre plane i + 4
                ptx::mbar_arrive(&mempty[s_m]);
            }
            s_c = (s_c + 1 == (uint32_t)P.NS) ? 0 : s_c + 1;
            if (++s_n == (uint32_t)P.NS) {
                s_n = 0;
                p_n ^= 1u;
            }
            if (++s_m == (uint32_t)P.NSM) {
                s_m = 0;
                p_m ^= 1u;
            }
            return true;
        };
        if constexpr (PERIODIC) {
            // one plane per iteration (the wrapped gathers leave no registers
            // for a second window)
            for (int i = 0; i < zce; ++i) {
                if (!step(q, i)) return;
#pragma unroll
                for (int d = 0; d < 2 * WR; ++d) q[d] = q[d + 1];
            }
        } else {
            // two output planes per iteration: the queue moves by two planes
            // (8 float4 moves per two planes instead of per plane)
            int i = 0;
            for (; i + 2 <= zce; i += 2) {
                if (!step(q, i) || !step(q + 1, i + 1)) return;
#pragma unroll
                for (int d = 0; d < 2 * WR; ++d) q[d] = q[d + 2];
            }
            if (i < zce && !step(q, i)) return;
        }
        gq = base + zce + 2 * WR;
        gm = mbase + zce;
    }
}

int wave_sm_count()
{
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 148;
    }
    return n;
}

constexpr size_t W_SMEM = 226 * 1024;  // of the 227 KB a block may use

// The u ring holds planes z..z+4 plus two in flight (7 stages); the (m, u^{n-1})
// ring carries half of the bytes read and gets the rest of shared memory (2 to
// 6 stages): with only 2 its stream is latency-bound.
bool wave_cfg(const Geom& g, int* TY, int* ZC, int* NS, int* NSM, size_t* stage_bytes, size_t* mstage_bytes)
{
    if (g.esize != 4) return false;
    const int ngx = (int)((g.nx + 3) / 4);
    int ty = (int)std::min<int64_t>(g.ny, W_NC / std::max(1, ngx));
    if (ty < 1) return false;  // a row wider than 4 * 512 points
    for (; ty >= 1; --ty) {
        const size_t sb = ((size_t)(ty + 2 * WR) * g.pitch * 4 + 127) / 128 * 128;
        const size_t mb = ((size_t)2 * ty * g.pitch * 4 + 127) / 128 * 128;
        const size_t fixed = 7 * sb + 256;
        if (fixed + mb * 2 <= W_SMEM) {
            *TY = ty;
            *NS = 7;
            *NSM = (int)std::min<size_t>(6, (W_SMEM - fixed) / mb);
            *stage_bytes = sb;
            *mstage_bytes = mb;
            break;
        }
    }
    if (ty < 1) return false;
    int eNS = 0, eNSM = 0, eZC = 0;  // "NS,NSM,ZC" for tuning sweeps
    const char* env = std::getenv("ST_WAVE_CFG");
    const bool use_env = env && std::sscanf(env, "%d,%d,%d", &eNS, &eNSM, &eZC) == 3 && eNS >= 5 && eNSM >= 2 &&
                         eZC >= 1 &&
                         (size_t)eNS * *stage_bytes + (size_t)eNSM * *mstage_bytes + 256 <=
                             227 * 1024 - 16 * (eNS + eNSM);
    if (use_env) {
        *NS = eNS;
        *NSM = eNSM;
    }
    const int nyt = (int)((g.ny + *TY - 1) / *TY);
    const int64_t want = 6LL * wave_sm_count();
    const int64_t nzc = std::max<int64_t>(1, want / nyt);
    int zc = (int)std::max<int64_t>(16, (g.nz + nzc - 1) / nzc);
    if (use_env) zc = eZC;
    *ZC = (int)std::min<int64_t>(zc, g.nz);
    return true;
}

}  // namespace

bool wave_supports(const FamilyDesc& d)
{
    if (d.g.ndim != 3 || d.levels != 2 || !d.star || d.g.esize != 4) return false;
    // star of radius exactly 4 whose weights depend only on the distance
    double a[WR + 1] = {}, b[WR + 1] = {};
    bool seen[3][2][WR] = {};
    bool centre = false;
    for (int k = 0; k < d.npts; ++k) {
        const int32_t* o = d.off + 3 * k;
        const int ax = o[0] ? 0 : (o[1] ? 1 : (o[2] ? 2 : -1));
        const double al = d.alpha[k], be = d.has_beta ? d.beta[k] : 0.0;
        if (ax < 0) {
            if (centre) return false;
            centre = true;
            a[0] = al;
            b[0] = be;
            continue;
        }
        const int v = o[ax], j = v < 0 ? -v : v;
        if (j > WR || seen[ax][v > 0][j - 1]) return false;
        seen[ax][v > 0][j - 1] = true;
        if (ax == 0 && v > 0) {
            a[j] = al;
            b[j] = be;
        }
    }
    for (int ax = 0; ax < 3; ++ax)
        for (int s = 0; s < 2; ++s)
            for (int j = 0; j < WR; ++j)
                if (!seen[ax][s][j]) return false;
    // every neighbour at distance j must carry the same (alpha, beta)
    for (int k = 0; k < d.npts; ++k) {
        const int32_t* o = d.off + 3 * k;
        const int ax = o[0] ? 0 : (o[1] ? 1 : (o[2] ? 2 : -1));
        if (ax < 0) continue;
        const int j = o[ax] < 0 ? -o[ax] : o[ax];
        if (d.alpha[k] != a[j] || (d.has_beta ? d.beta[k] : 0.0) != b[j]) return false;
    }
    if (!d.has_beta) return false;
    int TY, ZC, NS, NSM;
    size_t sb, mb;
    return wave_cfg(d.g, &TY, &ZC, &NS, &NSM, &sb, &mb);
}

cudaError_t launch_wave(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    const Geom& g = f.g;
    int TY, ZC, NS, NSM;
    size_t sb, mb;
    if (!wave_cfg(g, &TY, &ZC, &NS, &NSM, &sb, &mb)) return cudaErrorNotSupported;
    WaveParams P;
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
    P.TY = TY;
    P.ZC = ZC;
    P.NS = NS;
    P.NSM = NSM;
    P.mstage_elems = (uint32_t)(mb / 4);
    P.nyt = (int)((g.ny + TY - 1) / TY);
    P.nzc = (int)((g.nz + ZC - 1) / ZC);
    P.units = P.nyt * P.nzc;
    P.stage_elems = (uint32_t)(sb / 4);
    const StarCoef& c = f.sc;
    P.ac = (float)c.c_a;
    P.bc = (float)c.c_b;
    for (int j = 0; j < WR; ++j) {
        P.aj[j] = (float)c.a[0][1][j];
        P.bj[j] = (float)c.b[0][1][j];
    }
    P.sz = -1;
    if (a.src >= 0 && a.step >= 0 && a.step < a.src_count) {
        int64_t rel = a.src - g.origin;
        P.sz = rel / g.plane;
        rel -= P.sz * g.plane;
        P.sy = rel / g.pitch;
        P.sx = rel - P.sy * g.pitch;  // rel is measured from the interior origin
        P.src_amp = a.src_amp;
        P.step = a.step;
    }
    P.status = a.status;
    const size_t smem = (size_t)NS * sb + (size_t)NSM * mb + 2 * sizeof(uint64_t) * (NS + NSM);
    const bool alpha0 = P.aj[0] == 0.f && P.aj[1] == 0.f && P.aj[2] == 0.f && P.aj[3] == 0.f;
    typedef void (*WFn)(const float*, float*, const float*, const WaveParams);
    static const WFn table[2][2] = {{k_wave<false, false>, k_wave<false, true>}, {k_wave<true, false>, k_wave<true, true>}};
    static bool attr[2][2] = {{false, false}, {false, false}};
    const int pi = f.periodic ? 1 : 0, ai = alpha0 ? 1 : 0;
    if (!attr[pi][ai]) {
        cudaError_t e = cudaFuncSetAttribute(table[pi][ai], cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr[pi][ai] = true;
    }
    const int grid = (int)std::min<int64_t>(P.units, wave_sm_count());
    return launch_dependent(table[pi][ai], dim3(grid), dim3(W_THREADS), smem, s, (const float*)a.in, (float*)a.out,
                            (const float*)a.kappa, P);
}

}  // namespace st
