// One-thread-per-point kernels: the general form of the update (any offsets,
// constant or per-cell weights, one or two time levels), its transpose, the
// ghost fill of a Dirichlet boundary and the double-precision reductions.
//
// The sweep kernel has the shape of the kernels the paper's backend generates
// (Sec. III-C "Code generation": each thread computes one element of the
// output slice, the grid covers the whole slice).  It is the fallback for any
// stencil the specialised families do not cover and the "plain launch"
// baseline of the batched workload.
#include "common.cuh"
#include "ptx.cuh"

namespace st {

namespace {

template <typename T>
__device__ __forceinline__ T alpha_of(const GenParams& P, int k)
{
    if constexpr (sizeof(T) == 4) return P.alpha_f[k];
    else return P.alpha[k];
}

template <typename T>
__device__ __forceinline__ T beta_of(const GenParams& P, int k)
{
    if constexpr (sizeof(T) == 4) return P.beta_f[k];
    else return P.beta[k];
}

__device__ __forceinline__ int64_t wrap1(int64_t i, int64_t n)
{
    // |offset| < n is validated on the host, so one correction suffices
    i = (i < 0) ? i + n : i;
    return (i >= n) ? i - n : i;
}

template <typename T>
__global__ void __launch_bounds__(256)
k_sweep_generic(const T* __restrict__ in, T* out, const T* prev, const T* __restrict__ kappa,
                const __grid_constant__ GenParams P)
{
    ptx::griddep_wait();  // the previous sweep wrote `in` and read `out`
    ptx::griddep_trigger();
    const int64_t x = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * 8 + threadIdx.y;
    const int64_t z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int64_t p = P.origin + z * P.plane + y * P.pitch + x;
    const T kap = P.has_kappa ? kappa[p] : T(0);
    T acc = T(0);
    for (int k = 0; k < P.npts; ++k) {
        T v;
        if (P.periodic) {
            const int64_t zz = wrap1(z + P.dz[k], P.nz);
            const int64_t yy = wrap1(y + P.dy[k], P.ny);
            const int64_t xx = wrap1(x + P.dx[k], P.nx);
            v = in[P.origin + zz * P.plane + yy * P.pitch + xx];
        } else {
            v = in[p + P.lin[k]];
        }
        T w = alpha_of<T>(P, k);
        if (P.has_kappa) w = fma(beta_of<T>(P, k), kap, w);
        acc = fma(w, v, acc);
    }
    if (P.leapfrog) acc = acc - prev[p];
    if (p == P.src && P.step >= 0 && P.step < P.src_count) acc = acc + T(P.src_amp[P.step]);
    out[p] = acc;
}

// Transpose step: lambda_t[q] = sum_k w_k(q - o_k) lambda_{t+1}[q - o_k], and the
// coefficient gradient gk[q] += lambda_{t+1}[q] * sum_k beta_k u_t[q + o_k].
// Dirichlet: q - o_k may be a ghost cell; lambda's ghosts are zero and the
// coefficient field's ghosts finite, so those terms vanish.
template <typename T>
__global__ void __launch_bounds__(256)
k_adjoint_generic(const T* __restrict__ u, const T* __restrict__ lam, T* __restrict__ lout,
                  const T* __restrict__ kappa, double* __restrict__ gk,
                  const __grid_constant__ GenParams P)
{
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int64_t x = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * 8 + threadIdx.y;
    const int64_t z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    const int64_t q = P.origin + z * P.plane + y * P.pitch + x;
    T acc = T(0);
    T s = T(0);
    for (int k = 0; k < P.npts; ++k) {
        int64_t pm, pp;
        if (P.periodic) {
            pm = P.origin + wrap1(z - P.dz[k], P.nz) * P.plane + wrap1(y - P.dy[k], P.ny) * P.pitch +
                 wrap1(x - P.dx[k], P.nx);
            pp = P.origin + wrap1(z + P.dz[k], P.nz) * P.plane + wrap1(y + P.dy[k], P.ny) * P.pitch +
                 wrap1(x + P.dx[k], P.nx);
        } else {
            pm = q - P.lin[k];
            pp = q + P.lin[k];
        }
        T w = alpha_of<T>(P, k);
        if (P.has_kappa) w = fma(beta_of<T>(P, k), kappa[pm], w);
        acc = fma(w, lam[pm], acc);
        if (gk) s = fma(beta_of<T>(P, k), u[pp], s);
    }
    lout[q] = acc;
    if (gk) gk[q] += (double)lam[q] * (double)s;
}

// Transposed step of the zero-flux sweep (constant weights).  The sweep
// reads, for interior p and offset k, the cell mirror(p + o_k) (mirror per
// axis: -1 - i below the interior, 2n - 1 - i above), so its transpose
// gathers at q
//   lambda_t[q] = sum_k w_k sum over the cells g with mirror(g) = q of
//                 lambda_{t+1}[g - o_k]   (g - o_k interior),
// where per axis g takes q itself and, within r of a face, q's reflection
// across it (axes without ghosts, z in 2D, have only q).  Offsets in order,
// pre-images in a fixed order.
template <typename T>
__global__ void __launch_bounds__(256)
k_adjoint_neumann(const T* __restrict__ lam, T* __restrict__ lout, const __grid_constant__ GenParams P, int r, int rz)
{
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int64_t x = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * 8 + threadIdx.y;
    const int64_t z = blockIdx.z;
    if (x >= P.nx || y >= P.ny) return;
    // pre-images of q per axis (at most three)
    int64_t cz[3], cy[3], cx[3];
    int nzc = 0, nyc = 0, nxc = 0;
    auto pre = [](int64_t q, int64_t n, int rr, int64_t (&c)[3], int& m) {
        c[m++] = q;
        if (q <= rr - 1) c[m++] = -1 - q;
        if (q >= n - rr) c[m++] = 2 * n - 1 - q;
    };
    pre(z, P.nz, rz, cz, nzc);
    pre(y, P.ny, r, cy, nyc);
    pre(x, P.nx, r, cx, nxc);
    T acc = T(0);
    for (int k = 0; k < P.npts; ++k) {
        const T w = alpha_of<T>(P, k);
        for (int a = 0; a < nzc; ++a) {
            const int64_t pz = cz[a] - P.dz[k];
            if (pz < 0 || pz >= P.nz) continue;
            for (int b = 0; b < nyc; ++b) {
                const int64_t py = cy[b] - P.dy[k];
                if (py < 0 || py >= P.ny) continue;
                for (int c = 0; c < nxc; ++c) {
                    const int64_t px = cx[c] - P.dx[k];
                    if (px < 0 || px >= P.nx) continue;
                    acc = fma(w, lam[P.origin + pz * P.plane + py * P.pitch + px], acc);
                }
            }
        }
    }
    lout[P.origin + z * P.plane + y * P.pitch + x] = acc;
}

// Write `value` into every cell of a padded buffer that is not interior: the
// whole rows of the z ghost planes and of the y ghost rows, then the lead and
// tail columns of the interior rows.  Flat grid-stride loops over those cells
// only, so the cost follows the ghost shell, not the row count.
template <typename T>
__global__ void __launch_bounds__(256) k_fill_ghosts(T* __restrict__ buf, Geom g, T value)
{
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t zrows = 2 * g.rz * g.pny;  // rows of the z ghost planes
    const int64_t yrows = g.nz * 2 * g.r;    // y ghost rows of the interior planes
    const int64_t full = (zrows + yrows) * g.pitch;
    for (int64_t i = tid; i < full; i += nthr) {
        const int64_t row = i / g.pitch, x = i - row * g.pitch;
        int64_t pz, py;
        if (row < zrows) {
            const int64_t zp = row / g.pny;
            py = row - zp * g.pny;
            pz = zp < g.rz ? zp : zp + g.nz;
        } else {
            const int64_t k = row - zrows;
            const int64_t zi = k / (2 * g.r), yk = k - zi * 2 * g.r;
            pz = g.rz + zi;
            py = yk < g.r ? yk : yk + g.ny;
        }
        buf[pz * g.plane + py * g.pitch + x] = value;
    }
    const int64_t side = g.pitch - g.nx;  // lead [0, xl) and tail [xl + nx, pitch) of a row
    const int64_t nside = g.nz * g.ny * side;
    for (int64_t i = tid; i < nside; i += nthr) {
        const int64_t row = i / side, c = i - row * side;
        const int64_t zi = row / g.ny, yi = row - zi * g.ny;
        const int64_t x = c < g.xl ? c : g.nx + c;
        buf[(g.rz + zi) * g.plane + (g.r + yi) * g.pitch + x] = value;
    }
}

// Zero-flux (Neumann) boundary: every ghost cell within the ghost width takes
// the value of its mirror image across the boundary face, axis by axis
// (interior index i < 0 reads -1 - i, i >= n reads 2n - 1 - i).  Mirror images
// are interior cells, which this kernel never writes, so the order of the
// writes does not matter.  The same shell walk as k_fill_ghosts; padding
// columns beyond the ghost width are left alone.
__device__ __forceinline__ int64_t mirror(int64_t i, int64_t n) { return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i); }

template <typename T>
__global__ void __launch_bounds__(256) k_mirror_ghosts(T* __restrict__ buf, Geom g)
{
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t zrows = 2 * g.rz * g.pny;
    const int64_t yrows = g.nz * 2 * g.r;
    const int64_t w = g.nx + 2 * g.r;        // columns [xl - r, xl + nx + r)
    const int64_t full = (zrows + yrows) * w;
    auto src = [&](int64_t pz, int64_t py, int64_t x) {
        const int64_t zi = mirror(pz - g.rz, g.nz), yi = mirror(py - g.r, g.ny), xi = mirror(x - g.xl, g.nx);
        return buf[(g.rz + zi) * g.plane + (g.r + yi) * g.pitch + g.xl + xi];
    };
    for (int64_t i = tid; i < full; i += nthr) {
        const int64_t row = i / w, x = g.xl - g.r + (i - row * w);
        int64_t pz, py;
        if (row < zrows) {
            const int64_t zp = row / g.pny;
            py = row - zp * g.pny;
            pz = zp < g.rz ? zp : zp + g.nz;
        } else {
            const int64_t k = row - zrows;
            const int64_t zi = k / (2 * g.r), yk = k - zi * 2 * g.r;
            pz = g.rz + zi;
            py = yk < g.r ? yk : yk + g.ny;
        }
        buf[pz * g.plane + py * g.pitch + x] = src(pz, py, x);
    }
    const int64_t side = 2 * g.r;  // ghost columns of an interior row
    const int64_t nside = g.nz * g.ny * side;
    for (int64_t i = tid; i < nside; i += nthr) {
        const int64_t row = i / side, c = i - row * side;
        const int64_t zi = row / g.ny, yi = row - zi * g.ny;
        const int64_t x = c < g.r ? g.xl - g.r + c : g.xl + g.nx + (c - g.r);
        buf[(g.rz + zi) * g.plane + (g.r + yi) * g.pitch + x] = src(g.rz + zi, g.r + yi, x);
    }
}

// Deterministic block reduction of (sum, sum of squares, max) in double.
struct Red3 {
    double s, q, m;
};

__device__ __forceinline__ Red3 warp_red(Red3 v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.s += __shfl_down_sync(0xffffffffu, v.s, o);
        v.q += __shfl_down_sync(0xffffffffu, v.q, o);
        v.m = fmax(v.m, __shfl_down_sync(0xffffffffu, v.m, o));
    }
    return v;
}

__device__ Red3 block_red(Red3 v)
{
    __shared__ double sh[3][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = warp_red(v);
    if (lane == 0) {
        sh[0][wid] = v.s;
        sh[1][wid] = v.q;
        sh[2][wid] = v.m;
    }
    __syncthreads();
    const int nw = blockDim.x >> 5;
    Red3 w{0.0, 0.0, 0.0};
    if (wid == 0) {
        if (lane < nw) w = Red3{sh[0][lane], sh[1][lane], sh[2][lane]};
        w = warp_red(w);
    }
    __syncthreads();
    return w;  // valid in thread 0
}

// Compensated single-precision accumulator (hi + lo carries ~48 bits): the
// per-element work of an FP32 reduction stays on the FP32 pipe, because the
// FP64 rate of this GPU is 1/64 of FP32.  Error-free transformations:
// TwoSum (Knuth) for additions, fma for the exact product error.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e)
{
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// The sum and the sum of squares are two independent compensated pairs that
// take the same operations, so they run side by side in packed FP32x2
// instructions (one instruction per pair; each lane rounds exactly as the
// scalar operation would).  a - b is formed as fma(b, -1, a), which rounds
// a - b once, as a subtraction does.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// (hi, lo) += x + xlo for both pairs at once: lane 0 is the sum, lane 1 the
// sum of squares.  TwoSum of hi and x, then lo += err + xlo.
__device__ __forceinline__ void f2_add2(float2& hi, float2& lo, float2 x, float2 xlo)
{
    const float2 s = p_add(hi, x);
    const float2 bb = p_sub(s, hi);
    const float2 e = p_add(p_sub(hi, p_sub(s, bb)), p_sub(x, bb));
    hi = s;
    lo = p_add(lo, p_add(e, xlo));
}

// Per-element accumulation: FP32 inputs use the compensated float pair,
// FP64 inputs plain double.
struct AccF {
    float2 H{0.f, 0.f}, L{0.f, 0.f};  // (sum, sum of squares): high and low parts
    // max |d| kept exactly in single precision: |d| = |dh| + sign(dh) dl with
    // |dl| at most half the float spacing around dh, so ordering by |dh| first
    // and sign(dh) dl second orders the exact |d| (a rounding interval never
    // reaches past the gap to the next float)
    float mA = 0.f, mS = 0.f;
    __device__ __forceinline__ float add(float av, float bv)
    {
        float dh, dl;
        two_sum(av, -bv, dh, dl);  // d = dh + dl exactly
        const float p = dh * dh;
        const float pe = fmaf(dh, dh, -p);  // dh^2 = p + pe exactly
        f2_add2(H, L, make_float2(dh, p), make_float2(dl, pe + 2.f * dh * dl));
        const float A = fabsf(dh);
        const float sg = dh < 0.f ? -dl : dl;
        const bool gt = A > mA || (A == mA && sg > mS);
        mA = gt ? A : mA;
        mS = gt ? sg : mS;
        return dh;
    }
    // the same with b = 0 (then d = a exactly, dl = 0): fewer operations, the
    // same results
    __device__ __forceinline__ float add1(float av)
    {
        const float p = av * av;
        f2_add2(H, L, make_float2(av, p), make_float2(0.f, fmaf(av, av, -p)));
        mA = fmaxf(mA, fabsf(av));
        return av;
    }
    __device__ __forceinline__ Red3 result() const
    {
        return Red3{(double)H.x + (double)L.x, (double)H.y + (double)L.y, (double)mA + (double)mS};
    }
};

struct AccD {
    Red3 r{0.0, 0.0, 0.0};
    __device__ __forceinline__ double add(double av, double bv)
    {
        const double d = av - bv;
        r.s += d;
        r.q = fma(d, d, r.q);
        r.m = fmax(r.m, fabs(d));
        return d;
    }
    __device__ __forceinline__ double add1(double av) { return add(av, 0.0); }
    __device__ __forceinline__ Red3 result() const { return r; }
};

template <typename T>
struct VecOf;
template <>
struct VecOf<float> {
    typedef float4 V;
    typedef AccF Acc;
    static constexpr int N = 4;
};
template <>
struct VecOf<double> {
    typedef double2 V;
    typedef AccD Acc;
    static constexpr int N = 2;
};

// mode 0: d = a - b (b may be null); mode 1: also lam_out = d on the interior.
// Each warp walks whole interior rows; each lane loads 16-byte vectors, four
// per trip, so several loads are in flight (interior rows start 16-byte
// aligned).  The grid is sized to the blocks that are resident at once
// (reduce_blocks), so there is no partial second wave.  partials[3*block +
// {0,1,2}].
template <typename T, bool HAS_B>
__global__ void __launch_bounds__(256, HAS_B ? 3 : 4)
k_reduce_partial(const T* __restrict__ a, const T* __restrict__ b, Geom g, double* __restrict__ partials,
                 int mode, T* __restrict__ lam_out)
{
    typedef typename VecOf<T>::V V;
    constexpr int N = VecOf<T>::N;
    constexpr int U = 4;  // vectors per lane per trip
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t rows = g.nz * g.ny;
    const int64_t wstride = (int64_t)gridDim.x * (blockDim.x >> 5);
    const int64_t nxv = g.nx / N * N;  // vector part of a row
    typename VecOf<T>::Acc acc;
    // (z, y) of the warp's row, advanced by the stride's whole planes and
    // remaining rows (no division inside the loop)
    const int64_t row0 = (int64_t)blockIdx.x * (blockDim.x >> 5) + warp;
    int64_t z = row0 / g.ny, y = row0 - z * g.ny;
    const int64_t sz = wstride / g.ny, sy = wstride - sz * g.ny;
    for (int64_t row = row0; row < rows; row += wstride) {
        const int64_t base = g.origin + z * g.plane + y * g.pitch;
        z += sz;
        y += sy;
        if (y >= g.ny) {
            y -= g.ny;
            ++z;
        }
        const T* ra = a + base;
        const T* rb = HAS_B ? b + base : nullptr;
        for (int64_t x0 = (int64_t)lane * N; x0 < nxv; x0 += (int64_t)32 * N * U) {
            V va[U], vb[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t x = x0 + (int64_t)u * 32 * N;
                if (x < nxv) {
                    va[u] = *reinterpret_cast<const V*>(ra + x);
                    if (HAS_B) vb[u] = *reinterpret_cast<const V*>(rb + x);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int64_t x = x0 + (int64_t)u * 32 * N;
                if (x >= nxv) break;
                const T* pa = reinterpret_cast<const T*>(&va[u]);
                const T* pb = reinterpret_cast<const T*>(&vb[u]);
                T dv[N];
#pragma unroll
                for (int e = 0; e < N; ++e) dv[e] = HAS_B ? acc.add(pa[e], pb[e]) : acc.add1(pa[e]);
                if (mode == 1) *reinterpret_cast<V*>(lam_out + base + x) = *reinterpret_cast<const V*>(dv);
            }
        }
        for (int64_t x = nxv + lane; x < g.nx; x += 32) {  // ragged tail
            const T d = HAS_B ? acc.add(ra[x], rb[x]) : acc.add1(ra[x]);
            if (mode == 1) lam_out[base + x] = d;
        }
    }
    Red3 r = block_red(acc.result());
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = r.s;
        partials[3 * blockIdx.x + 1] = r.q;
        partials[3 * blockIdx.x + 2] = r.m;
    }
}

__global__ void __launch_bounds__(256)
k_reduce_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out, int mode)
{
    Red3 acc{0.0, 0.0, 0.0};
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) {
        acc.s += partials[3 * i + 0];
        acc.q += partials[3 * i + 1];
        acc.m = fmax(acc.m, partials[3 * i + 2]);
    }
    acc = block_red(acc);
    if (threadIdx.x == 0) {
        if (mode == 1) {
            out[0] = 0.5 * acc.q;
        } else {
            out[0] = acc.s;
            out[1] = acc.q;
            out[2] = acc.m;
        }
    }
}

// Dense interior <-> padded layout (dir 0: dense -> padded, 1: padded -> dense).
// One block per interior row.
// 16-byte groups of V elements, for rows whose length is a multiple of V and a
// 16-byte aligned dense buffer (the padded interior rows always are).
template <typename T, typename V>
__global__ void __launch_bounds__(256) k_pack_v(T* __restrict__ dense, T* __restrict__ padded, Geom g, int dir)
{
    // one flat grid-stride loop over (row, group) so that every thread has
    // work whatever the row length (this kernel may stream host memory);
    // the caller guarantees fewer than 2^31 groups, so indices are 32-bit
    constexpr int VE = sizeof(V) / sizeof(T);
    const uint32_t ny32 = (uint32_t)g.ny;
    const uint32_t nv = (uint32_t)(g.nx / VE);
    const uint32_t total = (uint32_t)(g.nz * g.ny) * nv;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
        const uint32_t row = i / nv;
        const uint32_t xv = i - row * nv;
        const uint32_t z = row / ny32, y = row - z * ny32;
        V* pr = reinterpret_cast<V*>(padded + g.origin + (int64_t)z * g.plane + (int64_t)y * g.pitch) + xv;
        V* dr = reinterpret_cast<V*>(dense + (int64_t)row * g.nx) + xv;
        if (dir == 0)
            *pr = *dr;
        else
            *dr = *pr;
    }
}

template <typename T>
__global__ void __launch_bounds__(256) k_pack(T* __restrict__ dense, T* __restrict__ padded, Geom g, int dir)
{
    const int64_t rows = g.nz * g.ny;
    const uint32_t ny32 = (uint32_t)g.ny;
    for (int64_t row = blockIdx.x; row < rows; row += gridDim.x) {
        const uint32_t z = (uint32_t)row / ny32, y = (uint32_t)row - z * ny32;
        T* pr = padded + g.origin + (int64_t)z * g.plane + (int64_t)y * g.pitch;
        T* dr = dense + row * g.nx;
        if (dir == 0)
            for (int64_t x = threadIdx.x; x < g.nx; x += blockDim.x) pr[x] = dr[x];
        else
            for (int64_t x = threadIdx.x; x < g.nx; x += blockDim.x) dr[x] = pr[x];
    }
}

dim3 point_grid(const GenParams& P)
{
    return dim3((unsigned)((P.nx + 31) / 32), (unsigned)((P.ny + 7) / 8), (unsigned)P.nz);
}

}  // namespace

void gen_params_floats(GenParams& P)
{
    for (int k = 0; k < ST_MAX_POINTS; ++k) {
        P.alpha_f[k] = (float)P.alpha[k];
        P.beta_f[k] = (float)P.beta[k];
    }
}

cudaError_t launch_generic_sweep(int esize, const void* in, void* out, const void* prev,
                                 const void* kappa, const GenParams& P, cudaStream_t s)
{
    if (P.nz * P.ny * P.nx == 0) return cudaSuccess;
    const dim3 grid = point_grid(P), block(32, 8);
    if (esize == 8)
        return launch_dependent(k_sweep_generic<double>, grid, block, 0, s, (const double*)in, (double*)out,
                                (const double*)prev, (const double*)kappa, P);
    return launch_dependent(k_sweep_generic<float>, grid, block, 0, s, (const float*)in, (float*)out,
                            (const float*)prev, (const float*)kappa, P);
}

cudaError_t launch_generic_adjoint(int esize, const void* u_t, const void* lam_in, void* lam_out,
                                   const void* kappa, double* gk, const GenParams& P,
                                   cudaStream_t s)
{
    if (P.nz * P.ny * P.nx == 0) return cudaSuccess;
    const dim3 grid = point_grid(P), block(32, 8);
    if (esize == 8)
        return launch_dependent(k_adjoint_generic<double>, grid, block, 0, s, (const double*)u_t,
                                (const double*)lam_in, (double*)lam_out, (const double*)kappa, gk, P);
    return launch_dependent(k_adjoint_generic<float>, grid, block, 0, s, (const float*)u_t, (const float*)lam_in,
                            (float*)lam_out, (const float*)kappa, gk, P);
}

cudaError_t launch_neumann_adjoint(int esize, const void* lam_in, void* lam_out, const GenParams& P, int r, int rz,
                                   cudaStream_t s)
{
    if (P.nz * P.ny * P.nx == 0) return cudaSuccess;
    const dim3 grid = point_grid(P), block(32, 8);
    if (esize == 8)
        return launch_dependent(k_adjoint_neumann<double>, grid, block, 0, s, (const double*)lam_in, (double*)lam_out,
                                P, r, rz);
    return launch_dependent(k_adjoint_neumann<float>, grid, block, 0, s, (const float*)lam_in, (float*)lam_out, P, r,
                            rz);
}

cudaError_t launch_pack(int esize, void* dense, void* padded, const Geom& g, int dir, cudaStream_t s)
{
    const int64_t rows = g.nz * g.ny;
    const unsigned blocks = (unsigned)(rows < 65535 * 8 ? rows : 65535 * 8);
    const bool vec = ((g.nx * esize) % 16 == 0) && (((uintptr_t)dense & 15u) == 0) &&
                     g.npoints * esize / 16 < ((int64_t)1 << 31);
    const unsigned vblocks = 152 * 16;  // grid-stride: a few waves of 256-thread blocks
    if (esize == 8) {
        if (vec)
            k_pack_v<double, double2><<<vblocks, 256, 0, s>>>((double*)dense, (double*)padded, g, dir);
        else
            k_pack<double><<<blocks, 256, 0, s>>>((double*)dense, (double*)padded, g, dir);
    } else {
        if (vec)
            k_pack_v<float, float4><<<vblocks, 256, 0, s>>>((float*)dense, (float*)padded, g, dir);
        else
            k_pack<float><<<blocks, 256, 0, s>>>((float*)dense, (float*)padded, g, dir);
    }
    return cudaGetLastError();
}

cudaError_t launch_fill_ghosts(int esize, void* buf, const Geom& g, double value, cudaStream_t s)
{
    const int64_t cells = (2 * g.rz * g.pny + g.nz * 2 * g.r) * g.pitch + g.nz * g.ny * (g.pitch - g.nx);
    const int64_t want = (cells + 255) / 256;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 8));
    if (esize == 8)
        return launch_dependent(k_fill_ghosts<double>, dim3(blocks), dim3(256), 0, s, (double*)buf, g, value);
    return launch_dependent(k_fill_ghosts<float>, dim3(blocks), dim3(256), 0, s, (float*)buf, g, (float)value);
}

cudaError_t launch_mirror_ghosts(int esize, void* buf, const Geom& g, cudaStream_t s)
{
    const int64_t cells = (2 * g.rz * g.pny + g.nz * 2 * g.r) * (g.nx + 2 * g.r) + g.nz * g.ny * 2 * g.r;
    const int64_t want = (cells + 255) / 256;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>(want, 152 * 8));
    if (esize == 8)
        return launch_dependent(k_mirror_ghosts<double>, dim3(blocks), dim3(256), 0, s, (double*)buf, g);
    return launch_dependent(k_mirror_ghosts<float>, dim3(blocks), dim3(256), 0, s, (float*)buf, g);
}

namespace {
// Blocks of one reduction kernel instance resident at once on this GPU.
int resident_blocks(const void* fn)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
    }
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0) != cudaSuccess || occ <= 0) {
        (void)cudaGetLastError();
        occ = 1;
    }
    return nsm * occ;
}

int64_t blocks_by_rows(const Geom& g) { return std::max<int64_t>(1, (g.nz * g.ny + 7) / 8); }
}  // namespace

int reduce_blocks(const Geom& g, int max_blocks)
{
    static int resident = 0;  // the most blocks any reduction kernel instance keeps resident
    if (resident == 0)
        for (const void* f : {(const void*)k_reduce_partial<float, true>, (const void*)k_reduce_partial<float, false>,
                              (const void*)k_reduce_partial<double, true>, (const void*)k_reduce_partial<double, false>})
            resident = std::max(resident, resident_blocks(f));
    return (int)std::min<int64_t>(std::min<int64_t>(resident, max_blocks), blocks_by_rows(g));
}

cudaError_t launch_reduce(int esize, const void* a, const void* b, const Geom& g, double* partials,
                          int nblocks, double* out, int mode, void* lam_out, cudaStream_t s)
{
    // the grid: the blocks of this kernel instance that are resident at once
    // (no partial second wave), within the caller's partials
    static int res[2][2] = {{0, 0}, {0, 0}};
    const int di = esize == 8, bi = b != nullptr;
    if (res[di][bi] == 0) {
        const void* fns[2][2] = {{(const void*)k_reduce_partial<float, false>, (const void*)k_reduce_partial<float, true>},
                                 {(const void*)k_reduce_partial<double, false>, (const void*)k_reduce_partial<double, true>}};
        res[di][bi] = resident_blocks(fns[di][bi]);
    }
    nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(nblocks, res[di][bi]), blocks_by_rows(g)));
    if (esize == 8) {
        if (b)
            k_reduce_partial<double, true><<<nblocks, 256, 0, s>>>((const double*)a, (const double*)b, g, partials,
                                                                   mode, (double*)lam_out);
        else
            k_reduce_partial<double, false><<<nblocks, 256, 0, s>>>((const double*)a, nullptr, g, partials, mode,
                                                                    (double*)lam_out);
    } else {
        if (b)
            k_reduce_partial<float, true><<<nblocks, 256, 0, s>>>((const float*)a, (const float*)b, g, partials,
                                                                  mode, (float*)lam_out);
        else
            k_reduce_partial<float, false><<<nblocks, 256, 0, s>>>((const float*)a, nullptr, g, partials, mode,
                                                                   (float*)lam_out);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_reduce_final<<<1, 256, 0, s>>>(partials, nblocks, out, mode);
    return cudaGetLastError();
}

}  // namespace st
