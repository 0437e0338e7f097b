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
//  * m and u^{n-1} are needed only at the point: they are loaded from global
//    memory two planes ahead into registers.  u^{n+1} overwrites u^{n-1} in
//    place (each point reads its own u^{n-1} before writing it).
#include <algorithm>
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
    int TY, ZC, NS;
    int nyt, nzc, units;
    uint32_t stage_elems;
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

template <bool PERIODIC>
__global__ void __launch_bounds__(W_THREADS, 1)
k_wave(const float* __restrict__ un, float* uprev_out, const float* __restrict__ m, const __grid_constant__ WaveParams P)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)P.NS * P.stage_elems * sizeof(float));
    uint64_t* empty = full + P.NS;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.NS; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], W_CWARPS);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();
    const uint32_t rowb = (uint32_t)(P.pitch * sizeof(float));
    const int H = 2 * WR;  // halo rows per tile

    if (warp == W_CWARPS) {
        if (lane != 0) return;
        uint32_t gq = 0;
        for (int u = blockIdx.x; u < P.units; u += gridDim.x) {
            const int yt = u % P.nyt, zc = u / P.nyt;
            const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
            const int tye = (int)imin_w(P.TY, P.ny - y0);
            const int zce = (int)imin_w(P.ZC, P.nz - z0);
            for (int q = 0; q < zce + 2 * WR; ++q, ++gq) {
                const uint32_t s = gq % P.NS, k = gq / P.NS;
                if (k > 0 && !ptx::mbar_wait(&empty[s], (k - 1) & 1)) {
                    timeout(P.status);
                    return;
                }
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
            }
        }
        for (uint32_t d = 0; d < (uint32_t)P.NS && d < gq; ++d) {
            const uint32_t g = gq - 1 - d;
            if (!ptx::mbar_wait(&full[g % P.NS], (g / P.NS) & 1)) timeout(P.status);
        }
        return;
    }

    // ---------------------------------------------------------------- consumers
    const int ct = threadIdx.x;
    const int ngx = (int)((P.nx + 3) / 4);
    uint32_t gq = 0;
    for (int u = blockIdx.x; u < P.units; u += gridDim.x) {
        const int yt = u % P.nyt, zc = u / P.nyt;
        const int64_t y0 = (int64_t)yt * P.TY, z0 = (int64_t)zc * P.ZC;
        const int tye = (int)imin_w(P.TY, P.ny - y0);
        const int zce = (int)imin_w(P.ZC, P.nz - z0);
        const uint32_t base = gq;
        const bool active = ct < tye * ngx;
        const int row = active ? ct / ngx : 0;
        const int x = active ? (ct - row * ngx) * 4 : 0;
        const bool full4 = x + 4 <= P.nx;
        const int64_t gofs = P.origin + (y0 + row) * P.pitch + x;  // + z * plane
        float4 q[2 * WR + 1];
        float4 m0, m1, p0, p1;  // m and u^{n-1} of the next two output planes

        auto stage_of = [&](int qq) -> const float* {
            return ring + (size_t)((base + qq) % P.NS) * P.stage_elems + P.xl;
        };
        auto wait_plane = [&](int qq) -> bool {
            const uint32_t g = base + qq;
            return ptx::mbar_wait_warp(&full[g % P.NS], (g / P.NS) & 1);
        };
        auto release = [&](int qq) {
            __syncwarp();
            if (lane == 0) ptx::mbar_arrive(&empty[(base + qq) % P.NS]);
        };
        // plane q is a centre (output z0 + q - 4) for q in [4, zce + 4); all
        // other planes of the chunk only feed the z queues
        auto is_centre = [&](int qq) -> bool { return qq >= WR && qq < zce + WR; };
        auto read_q = [&](int qq) -> float4 {
            const float* rp = stage_of(qq) + (int64_t)(row + WR) * P.pitch;
            if (full4) return *reinterpret_cast<const float4*>(rp + x);
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (x + 0 < P.nx) v.x = rp[x + 0];
            if (x + 1 < P.nx) v.y = rp[x + 1];
            if (x + 2 < P.nx) v.z = rp[x + 2];
            return v;
        };
        auto load_g = [&](const float* arr, int64_t zz) -> float4 {
            const float* p = arr + gofs + zz * P.plane;
            if (full4) return __ldg(reinterpret_cast<const float4*>(p));
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (x + 0 < P.nx) v.x = p[0];
            if (x + 1 < P.nx) v.y = p[1];
            if (x + 2 < P.nx) v.z = p[2];
            return v;
        };
        // prime: queue planes z0-4 .. z0+3 (q = 0..7)
        for (int qq = 0; qq < 2 * WR; ++qq) {
            if (!wait_plane(qq)) {
                timeout(P.status);
                return;
            }
            q[qq + 1] = active ? read_q(qq) : make_float4(0.f, 0.f, 0.f, 0.f);
            if (!is_centre(qq)) release(qq);
        }
        m0 = m1 = p0 = p1 = make_float4(0.f, 0.f, 0.f, 0.f);
        if (active) {
            m0 = load_g(m, z0);
            p0 = load_g(uprev_out, z0);
            if (zce > 1) {
                m1 = load_g(m, z0 + 1);
                p1 = load_g(uprev_out, z0 + 1);
            }
        }
        for (int i = 0; i < zce; ++i) {
            // shift the queue and take plane z+4 (q = i + 8)
#pragma unroll
            for (int d = 0; d < 2 * WR; ++d) q[d] = q[d + 1];
            if (!wait_plane(i + 2 * WR)) {
                timeout(P.status);
                return;
            }
            if (active) q[2 * WR] = read_q(i + 2 * WR);
            if (!is_centre(i + 2 * WR)) release(i + 2 * WR);
            const float4 mv = m0, pv = p0;
            m0 = m1;
            p0 = p1;
            if (active && i + 2 < zce) {
                m1 = load_g(m, z0 + i + 2);
                p1 = load_g(uprev_out, z0 + i + 2);
            }
            if (active) {
                const float* cp = stage_of(i + WR);  // centre plane, x origin applied
                const float* rc = cp + (int64_t)(row + WR) * P.pitch;
                float c[4] = {q[WR].x, q[WR].y, q[WR].z, q[WR].w};
                // distance sums S_j over the six neighbours at distance j
                float S[WR][4];
#pragma unroll
                for (int j = 1; j <= WR; ++j) {
                    const float4 zl = q[WR - j], zh = q[WR + j];
                    S[j - 1][0] = zl.x + zh.x;
                    S[j - 1][1] = zl.y + zh.y;
                    S[j - 1][2] = zl.z + zh.z;
                    S[j - 1][3] = zl.w + zh.w;
                }
                if (full4) {
#pragma unroll
                    for (int j = 1; j <= WR; ++j) {
                        const float4 yl = *reinterpret_cast<const float4*>(rc - j * P.pitch + x);
                        const float4 yh = *reinterpret_cast<const float4*>(rc + j * P.pitch + x);
                        S[j - 1][0] += yl.x + yh.x;
                        S[j - 1][1] += yl.y + yh.y;
                        S[j - 1][2] += yl.z + yh.z;
                        S[j - 1][3] += yl.w + yh.w;
                    }
                    // x window: 4 left, the group, 4 right
                    // vector loads only at multiples of 4 from the row start (16-byte
                    // aligned); a periodic window that wraps is gathered element-wise
                    float4 L, R;
                    if (PERIODIC && x == 0)
                        L = make_float4(rc[wrapw(x - 4, P.nx)], rc[wrapw(x - 3, P.nx)], rc[wrapw(x - 2, P.nx)],
                                        rc[wrapw(x - 1, P.nx)]);
                    else
                        L = *reinterpret_cast<const float4*>(rc + x - 4);
                    if (PERIODIC && x + 8 > P.nx)
                        R = make_float4(rc[wrapw(x + 4, P.nx)], rc[wrapw(x + 5, P.nx)], rc[wrapw(x + 6, P.nx)],
                                        rc[wrapw(x + 7, P.nx)]);
                    else
                        R = *reinterpret_cast<const float4*>(rc + x + 4);
                    const float w[12] = {L.x, L.y, L.z, L.w, c[0], c[1], c[2], c[3], R.x, R.y, R.z, R.w};
#pragma unroll
                    for (int j = 1; j <= WR; ++j)
#pragma unroll
                        for (int e = 0; e < 4; ++e) S[j - 1][e] += w[4 + e - j] + w[4 + e + j];
                } else {
                    for (int e = 0; e < 4; ++e) {
                        const int64_t xe = x + e;
                        if (xe >= P.nx) break;
#pragma unroll
                        for (int j = 1; j <= WR; ++j) {
                            const float yl = rc[xe - j * P.pitch], yh = rc[xe + j * P.pitch];
                            const int64_t xm = PERIODIC ? wrapw(xe - j, P.nx) : xe - j;
                            const int64_t xp = PERIODIC ? wrapw(xe + j, P.nx) : xe + j;
                            S[j - 1][e] += yl + yh + rc[xm] + rc[xp];
                        }
                    }
                }
                const float mm[4] = {mv.x, mv.y, mv.z, mv.w};
                const float pp[4] = {pv.x, pv.y, pv.z, pv.w};
                float o[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    float lap = P.bj[0] * S[0][e];
                    lap = fmaf(P.bj[1], S[1][e], lap);
                    lap = fmaf(P.bj[2], S[2][e], lap);
                    lap = fmaf(P.bj[3], S[3][e], lap);
                    lap = fmaf(P.bc, c[e], lap);                      // beta part: sum_k beta_k u_k
                    float acc = fmaf(P.ac, c[e], -pp[e]);             // alpha part (centre only) - u^{n-1}
                    float alo = P.aj[0] * S[0][e];
                    alo = fmaf(P.aj[1], S[1][e], alo);
                    alo = fmaf(P.aj[2], S[2][e], alo);
                    alo = fmaf(P.aj[3], S[3][e], alo);
                    acc += alo;
                    o[e] = fmaf(mm[e], lap, acc);
                }
                const int64_t z = z0 + i;
                if (P.sz == z && P.sy == y0 + row && P.sx >= x && P.sx < x + 4) {
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
            release(i + WR);
        }
        gq = base + zce + 2 * WR;
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

constexpr size_t W_SMEM = 210 * 1024;

bool wave_cfg(const Geom& g, int* TY, int* ZC, int* NS, size_t* stage_bytes)
{
    if (g.esize != 4) return false;
    const int ngx = (int)((g.nx + 3) / 4);
    int ty = std::min<int64_t>(g.ny, W_NC / std::max(1, ngx));
    if (ty < 1) return false;  // a row wider than 4 * 512 points
    for (; ty >= 1; --ty) {
        const size_t sb = ((size_t)(ty + 2 * WR) * g.pitch * 4 + 127) / 128 * 128;
        if (sb * 8 + 128 <= W_SMEM) {
            *TY = ty;
            *NS = 8;
            *stage_bytes = sb;
            break;
        }
    }
    if (ty < 1) return false;
    const int nyt = (int)((g.ny + *TY - 1) / *TY);
    const int64_t want = 6LL * wave_sm_count();
    const int64_t nzc = std::max<int64_t>(1, want / nyt);
    int zc = (int)std::max<int64_t>(16, (g.nz + nzc - 1) / nzc);
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
    int TY, ZC, NS;
    size_t sb;
    return wave_cfg(d.g, &TY, &ZC, &NS, &sb);
}

cudaError_t launch_wave(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    const Geom& g = f.g;
    int TY, ZC, NS;
    size_t sb;
    if (!wave_cfg(g, &TY, &ZC, &NS, &sb)) return cudaErrorNotSupported;
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
    const size_t smem = (size_t)NS * sb + 2 * sizeof(uint64_t) * NS;
    static bool attr[2] = {false, false};
    const int pi = f.periodic ? 1 : 0;
    if (!attr[pi]) {
        cudaError_t e = cudaFuncSetAttribute(f.periodic ? k_wave<true> : k_wave<false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        if (e != cudaSuccess) return e;
        attr[pi] = true;
    }
    const int grid = (int)std::min<int64_t>(P.units, wave_sm_count());
    if (f.periodic)
        k_wave<true><<<grid, W_THREADS, smem, s>>>((const float*)a.in, (float*)a.out, (const float*)a.kappa, P);
    else
        k_wave<false><<<grid, W_THREADS, smem, s>>>((const float*)a.in, (float*)a.out, (const float*)a.kappa, P);
    return cudaGetLastError();
}

}  // namespace st
