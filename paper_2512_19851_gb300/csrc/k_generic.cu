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

// FP32 reductions accumulate in compensated single precision (hi + lo
// carries about 48 bits): the per-element work stays on the FP32 pipe,
// because the FP64 rate of this GPU is 1/64 of FP32.  Error-free
// transformations: TwoSum (Knuth) for additions, fma for the exact product
// error.  They run in packed FP32x2 instructions (each lane rounds exactly as
// the scalar operation would); a - b is formed as fma(b, -1, a), which rounds
// a - b once, as a subtraction does.
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }

// FP64 reductions: plain double accumulation (three FP64 operations per
// element; the FP64 pipe, not the loads, sets their pace).
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
struct VecOf<double> {
    typedef double2 V;
    typedef AccD Acc;
    static constexpr int N = 2;
};

// FP64 fields (k_reduce_ring takes FP32).
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

// FP32 reductions through a shared-memory ring filled by bulk copies.  Two
// persistent blocks per SM: lane 0 of the last warp of a block copies work
// items into an NS-stage ring, RR_CW consumer warps accumulate the interior
// elements of each stage.  The bytes in flight per SM are set by the rings
// (several stages), not by the consumers' registers, which is what a plain
// load loop runs short of.
//
// A work item is either a run of whole padded rows of one plane (rpi rows,
// ghost columns included: they share the DRAM sectors of the interior's first
// and last elements, so copying them adds no traffic) or, when a padded row
// is longer than a stage, one segment of an interior row.  Consumer warp w
// takes rows w, w + RR_CW, ... of a row item, or the w-th slice of a segment;
// its lanes walk 16-byte vectors of the row.
struct RedRing {
    int64_t nz, ny, nx, pitch, plane, origin, xl, r, rz;
    int se;        // elements per array per stage (a multiple of 4)
    int ns;        // stages
    int rpi;       // rows per item; 0: row segments of se elements
    int nseg;      // segments per interior row (segment items)
    int64_t ipp;   // items per plane (row items)
    int64_t items;
    int mode;      // 1: also lam_out = a - b on the interior
    int all_whole; // every item is whole (rpi divides ny, or se divides nx)
    int* status;   // set to ST_ERR_DEVICE_TIMEOUT when a wait runs out
};
constexpr int RR_CW = 16;  // consumer warps per block

// Position of a work item as (plane z, b, c): row items b = item in the plane,
// c = 0; segment items b = row in the plane, c = segment.  A block visits
// items blockIdx.x, blockIdx.x + gridDim.x, ...; the walk advances (z, b, c)
// by the grid size in mixed radix (nb, nc) without dividing per item (all
// three fit in 32 bits: nz <= 65535, ny <= 2^24).
struct ItemWalk {
    int z, b, c;
    int nz, nb, nc;
    int dz, db, dc;
    __device__ __forceinline__ void init(const RedRing& P)
    {
        nb = (int)(P.rpi > 0 ? P.ipp : P.ny);
        nc = P.rpi > 0 ? 1 : P.nseg;
        nz = (int)P.nz;
        const int64_t it = blockIdx.x, G = gridDim.x;
        c = (int)(it % nc);
        b = (int)((it / nc) % nb);
        z = (int)(it / nc / nb);
        dc = (int)(G % nc);
        db = (int)((G / nc) % nb);
        dz = (int)(G / nc / nb);
    }
    // The item the walk's position stands for: positions run backwards
    // through memory (the last item first), so that a reduction launched
    // right after a sweep starts on the part of the field the sweep wrote
    // last, which is still in L2.
    __device__ __forceinline__ ItemWalk item() const
    {
        ItemWalk r = *this;
        r.z = nz - 1 - z;
        r.b = nb - 1 - b;
        r.c = nc - 1 - c;
        return r;
    }
    __device__ __forceinline__ void next()
    {
        c += dc;
        const int carry = c >= nc;
        c -= carry ? nc : 0;
        b += db + carry;
        z += dz;
        if (b >= nb) {
            b -= nb;
            ++z;
        }
    }
};

struct RedItem {
    int64_t gsrc;    // element index of the first copied element
    int64_t gbase;   // element index of interior x = x0 of the item's first row
    uint32_t bytes;  // bytes per array
    int nrows, sstride, sx0, nxe;
};

// The layout fields an item needs, copied out of the kernel parameters once
// so that they live in registers (a parameter struct read through a
// reference each item costs a memory access per field).
struct RedGeo {
    int64_t plane, pitch, origin;
    int ny, nx, rpi, se, xl, r, rz;
};

__device__ __forceinline__ RedItem red_item(const RedGeo& G, const ItemWalk& w)
{
    RedItem I;
    if (G.rpi > 0) {
        const int64_t y0 = (int64_t)w.b * G.rpi;
        I.nrows = (int)(G.ny - y0 < G.rpi ? G.ny - y0 : G.rpi);
        I.gsrc = ((int64_t)w.z + G.rz) * G.plane + (y0 + G.r) * G.pitch;
        I.gbase = I.gsrc + G.xl;
        I.bytes = (uint32_t)(I.nrows * G.pitch * 4);
        I.sstride = (int)G.pitch;
        I.sx0 = G.xl;
        I.nxe = G.nx;
    } else {
        const int64_t x0 = (int64_t)w.c * G.se;
        I.nxe = (int)(G.nx - x0 < G.se ? G.nx - x0 : G.se);
        I.gsrc = G.origin + (int64_t)w.z * G.plane + (int64_t)w.b * G.pitch + x0;
        I.gbase = I.gsrc;
        I.bytes = (uint32_t)(((I.nxe + 3) & ~3) * 4);
        I.nrows = 1;
        I.sstride = 0;
        I.sx0 = 0;
    }
    return I;
}

// How the consumer warps share an item of nrows rows of nxe elements: wpr
// warps per row (rows fewer than warps, or one long segment), warp w takes
// slice w % wpr of rows w / wpr, w / wpr + jstep, ...; its lanes walk the
// 16-byte vectors [vb, ve) of the slice.
struct WarpShare {
    int j0, jstep, vb, ve, nfull, rem, slice, active;
    __device__ __forceinline__ void set(int nrows, int nxe, int warp)
    {
        nfull = nxe >> 2;
        rem = nxe - 4 * nfull;
        const int wpr = RR_CW / min(nrows, RR_CW);
        jstep = RR_CW / wpr;
        slice = warp % wpr;
        j0 = warp / wpr;
        active = warp < wpr * jstep;
        const int q = (nfull + wpr - 1) / wpr;
        vb = slice * q;
        ve = min(nfull, vb + q);
    }
};

// Compensated accumulation of two interleaved element streams: the even and
// the odd elements of a row each have their own (hi, lo) pairs for the sum
// and the sum of squares, so one packed FP32x2 instruction advances both
// (a quarter fewer instructions per element than one stream carrying the sum
// and the sum of squares side by side).  TwoSum for the additions, fma for
// the exact square error.
struct AccP {
    float2 Hs{0.f, 0.f}, Ls{0.f, 0.f}, Hq{0.f, 0.f}, Lq{0.f, 0.f};
    // max |d| kept exactly in single precision: |d| = |dh| + sign(dh) dl with
    // |dl| at most half the float spacing around dh, so ordering by |dh| first
    // and sign(dh) dl second orders the exact |d| (a rounding interval never
    // reaches past the gap to the next float)
    float mA = 0.f, mS = 0.f;
    // hi + lo += x + xlo
    __device__ __forceinline__ static void add(float2& hi, float2& lo, float2 x, float2 xlo)
    {
        const float2 s = p_add(hi, x);
        const float2 bb = p_sub(s, hi);
        const float2 e = p_add(p_sub(hi, p_sub(s, bb)), p_sub(x, bb));
        hi = s;
        lo = p_add(lo, p_add(e, xlo));
    }
    // hi + lo += x (no low part)
    __device__ __forceinline__ static void add0(float2& hi, float2& lo, float2 x)
    {
        const float2 s = p_add(hi, x);
        const float2 bb = p_sub(s, hi);
        const float2 e = p_add(p_sub(hi, p_sub(s, bb)), p_sub(x, bb));
        hi = s;
        lo = p_add(lo, e);
    }
    // two elements of a (b = 0)
    __device__ __forceinline__ void put1(float2 x)
    {
        const float2 p = __fmul2_rn(x, x);
        const float2 pe = __ffma2_rn(x, x, make_float2(-p.x, -p.y));  // x^2 = p + pe exactly
        add0(Hs, Ls, x);
        add(Hq, Lq, p, pe);
        mA = fmaxf(mA, fmaxf(fabsf(x.x), fabsf(x.y)));
    }
    // two elements of a - b; returns the rounded differences
    __device__ __forceinline__ float2 put2(float2 a, float2 b)
    {
        // d = dh + dl exactly (TwoSum of a and -b)
        const float2 dh = p_sub(a, b);
        const float2 bb = p_sub(dh, a);
        const float2 dl = p_sub(p_sub(a, p_sub(dh, bb)), p_add(b, bb));
        const float2 p = __fmul2_rn(dh, dh);
        float2 pe = __ffma2_rn(dh, dh, make_float2(-p.x, -p.y));
        pe = __ffma2_rn(p_add(dh, dh), dl, pe);  // d^2 = p + pe + dl^2 (dl^2 below the pair's precision)
        add(Hs, Ls, dh, dl);
        add(Hq, Lq, p, pe);
        max1(dh.x, dl.x);
        max1(dh.y, dl.y);
        return dh;
    }
    __device__ __forceinline__ void max1(float dh, float dl)
    {
        const float A = fabsf(dh);
        const float sg = dh < 0.f ? -dl : dl;
        const bool gt = A > mA || (A == mA && sg > mS);
        mA = gt ? A : mA;
        mS = gt ? sg : mS;
    }
    // one element (a row's ragged end)
    __device__ __forceinline__ float put_one(float a, float b, bool has_b)
    {
        if (has_b) return put2(make_float2(a, 0.f), make_float2(b, 0.f)).x;
        put1(make_float2(a, 0.f));
        return a;
    }
};

// A compensated single-precision value hi + lo and its sum (TwoSum of the
// high parts, the low parts added): the block's partial sums are combined in
// single precision, and converted to double once per block, because every
// FP64 instruction runs on this GPU's narrow FP64 pipe.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    return FF{s, (a.lo + b.lo) + e};
}

// The block's (sum, sum of squares, max |d|) from every thread's AccP;
// valid in thread 0.
__device__ Red3 block_red_ff(const AccP& acc)
{
    __shared__ float sh[6][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    FF S = ff_add(FF{acc.Hs.x, acc.Ls.x}, FF{acc.Hs.y, acc.Ls.y});
    FF Q = ff_add(FF{acc.Hq.x, acc.Lq.x}, FF{acc.Hq.y, acc.Lq.y});
    float mA = acc.mA, mS = acc.mS;
    auto fold = [&](int o) {
        const FF S2{__shfl_down_sync(0xffffffffu, S.hi, o), __shfl_down_sync(0xffffffffu, S.lo, o)};
        const FF Q2{__shfl_down_sync(0xffffffffu, Q.hi, o), __shfl_down_sync(0xffffffffu, Q.lo, o)};
        const float A2 = __shfl_down_sync(0xffffffffu, mA, o), B2 = __shfl_down_sync(0xffffffffu, mS, o);
        S = ff_add(S, S2);
        Q = ff_add(Q, Q2);
        const bool gt = A2 > mA || (A2 == mA && B2 > mS);
        mA = gt ? A2 : mA;
        mS = gt ? B2 : mS;
    };
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fold(o);
    if (lane == 0) {
        sh[0][wid] = S.hi;
        sh[1][wid] = S.lo;
        sh[2][wid] = Q.hi;
        sh[3][wid] = Q.lo;
        sh[4][wid] = mA;
        sh[5][wid] = mS;
    }
    __syncthreads();
    Red3 r{0.0, 0.0, 0.0};
    if (wid == 0) {
        const int nw = blockDim.x >> 5;
        const bool in = lane < nw;
        S = FF{in ? sh[0][lane] : 0.f, in ? sh[1][lane] : 0.f};
        Q = FF{in ? sh[2][lane] : 0.f, in ? sh[3][lane] : 0.f};
        mA = in ? sh[4][lane] : 0.f;
        mS = in ? sh[5][lane] : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fold(o);
        r = Red3{(double)S.hi + (double)S.lo, (double)Q.hi + (double)Q.lo, (double)mA + (double)mS};
    }
    return r;
}

// One 16-byte vector v of a staged row (a at ra, b at ra + bofs): accumulate
// a - b (or a) and, in mode 1, store the differences at lo.
template <bool HAS_B>
__device__ __forceinline__ void red_vec(AccP& acc, const float* ra, int bofs, int v, bool mode1, float* lo)
{
    const float4 x = *reinterpret_cast<const float4*>(ra + 4 * v);
    if (HAS_B) {
        const float4 y = *reinterpret_cast<const float4*>(ra + bofs + 4 * v);
        const float2 d0 = acc.put2(make_float2(x.x, x.y), make_float2(y.x, y.y));
        const float2 d1 = acc.put2(make_float2(x.z, x.w), make_float2(y.z, y.w));
        if (mode1) *reinterpret_cast<float4*>(lo + 4 * v) = make_float4(d0.x, d0.y, d1.x, d1.y);
    } else {
        acc.put1(make_float2(x.x, x.y));
        acc.put1(make_float2(x.z, x.w));
    }
}

// One element x of a row's ragged end.
template <bool HAS_B>
__device__ __forceinline__ void red_tail(AccP& acc, const float* ra, int bofs, int x, bool mode1, float* lo)
{
    const float d = acc.put_one(ra[x], HAS_B ? ra[bofs + x] : 0.f, HAS_B);
    if (mode1) lo[x] = d;
}

// A partial item (a plane's last rows, a row's last segment), out of line so
// that its bookkeeping does not take registers from the whole-item loop.
template <bool HAS_B>
__device__ __noinline__ AccP red_partial(AccP acc, const RedGeo G, const ItemWalk w, const float* stg, int warp,
                                         int lane, bool mode1, float* lam_out)
{
    const RedItem I = red_item(G, w);
    stg += I.sx0;
    WarpShare sh;
    sh.set(I.nrows, I.nxe, warp);
    for (int j = sh.j0; sh.active && j < I.nrows; j += sh.jstep) {
        const float* ra = stg + j * I.sstride;
        float* lo = lam_out + I.gbase + (int64_t)j * G.pitch;
        for (int v = sh.vb + lane; v < sh.ve; v += 32) red_vec<HAS_B>(acc, ra, G.se, v, mode1, lo);
        // the row's ragged end (fewer than 4 elements), by the row's first slice
        if (sh.rem > 0 && sh.slice == 0 && lane < sh.rem) red_tail<HAS_B>(acc, ra, G.se, 4 * sh.nfull + lane, mode1, lo);
    }
    return acc;
}

template <bool HAS_B>
__global__ void __launch_bounds__((RR_CW + 1) * 32, 2)
k_reduce_ring(const float* __restrict__ a, const float* __restrict__ b, const __grid_constant__ RedRing P,
              double* __restrict__ partials, float* __restrict__ lam_out)
{
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float* ring = reinterpret_cast<float*>(smem_raw);
    const int stage_f = (HAS_B ? 2 : 1) * P.se;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem_raw + (size_t)P.ns * stage_f * sizeof(float));
    uint64_t* empty = full + P.ns;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < P.ns; ++s) {
            ptx::mbar_init(&full[s], 1);
            ptx::mbar_init(&empty[s], RR_CW);
        }
        ptx::fence_barrier_init();
    }
    __syncthreads();
    ptx::griddep_wait();  // earlier kernels of the stream wrote the inputs
    ptx::griddep_trigger();

    const RedGeo G{P.plane, P.pitch, P.origin, (int)P.ny, (int)P.nx, P.rpi, P.se, (int)P.xl, (int)P.r, (int)P.rz};
    // items of this block: blockIdx.x, blockIdx.x + gridDim.x, ...
    const int my_items = P.items > blockIdx.x ? (int)((P.items - blockIdx.x + gridDim.x - 1) / gridDim.x) : 0;
    const int ns = P.ns;
    const bool mode1 = HAS_B && P.mode == 1;  // the residual's lambda (needs b)
    AccP acc;
    if (warp == RR_CW) {
        // ------------------------------------------------------------ producer
        if (lane == 0) {
            uint32_t gq = 0;
            ItemWalk w;
            w.init(P);
            uint32_t s = 0, k = 0;  // ring slot and its use count
            for (int it = 0; it < my_items; ++it, ++gq, w.next()) {
                if (k > 0 && !ptx::mbar_wait(&empty[s], (k - 1) & 1)) {
                    if (P.status) atomicCAS(P.status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
                    break;
                }
                const RedItem I = red_item(G, w.item());
                float* dst = ring + (size_t)s * stage_f;
                ptx::mbar_arrive_expect_tx(&full[s], (HAS_B ? 2u : 1u) * I.bytes);
                ptx::bulk_g2s(dst, a + I.gsrc, I.bytes, &full[s]);
                if (HAS_B) ptx::bulk_g2s(dst + G.se, b + I.gsrc, I.bytes, &full[s]);
                if (++s == (uint32_t)ns) {
                    s = 0;
                    ++k;
                }
            }
            // every issued copy lands before the block leaves
            for (uint32_t d = 0; d < (uint32_t)ns && d < gq; ++d) {
                const uint32_t g = gq - 1 - d;
                if (!ptx::mbar_wait(&full[g % ns], (g / ns) & 1) && P.status)
                    atomicCAS(P.status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
            }
        }
        __syncwarp();
    } else {
        // ---------------------------------------------------------- consumers
        // a whole item (all but a plane's last row item when rpi does not
        // divide ny, all but a row's last segment when se does not divide
        // nx): b < lim_b and c < lim_c.  Each warp holds at most one of its
        // rows (see WarpShare); this thread's part of it is fixed.
        WarpShare fs;
        const int full_rows = G.rpi > 0 ? G.rpi : 1;
        fs.set(full_rows, G.rpi > 0 ? G.nx : G.se, warp);
        const int lim_b = G.rpi > 0 ? G.ny / G.rpi : G.ny;
        const int lim_c = G.rpi > 0 ? 1 : G.nx / G.se;
        const bool f_act = fs.active && fs.j0 < full_rows;
        const int f_off = (G.rpi > 0 ? G.xl + fs.j0 * (int)G.pitch : 0);
        const int f_ve = fs.ve;
        const bool f_tail = f_act && fs.rem > 0 && fs.slice == 0 && lane < fs.rem;
        const int f_tx = 4 * fs.nfull + lane;
        auto whole = [&](const float* stg, float* lo) {
            const float* ra = stg + f_off;
            for (int v = fs.vb + lane; v < f_ve; v += 32) red_vec<HAS_B>(acc, ra, G.se, v, mode1, lo);
            if (f_tail) red_tail<HAS_B>(acc, ra, G.se, f_tx, mode1, lo);
        };
        uint32_t s = 0, par = 0;  // ring slot and the parity of its phase
        if (P.all_whole && !mode1) {
            // every item whole and nothing to store: no item positions needed
            for (int it = 0; it < my_items; ++it) {
                if (!ptx::mbar_wait_warp(&full[s], par)) {
                    if (lane == 0 && P.status) atomicCAS(P.status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
                    break;
                }
                if (f_act) whole(ring + (size_t)s * stage_f, nullptr);
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&empty[s]);
                if (++s == (uint32_t)ns) {
                    s = 0;
                    par ^= 1u;
                }
            }
        } else {
            ItemWalk w;
            w.init(P);
            for (int it = 0; it < my_items; ++it, w.next()) {
                if (!ptx::mbar_wait_warp(&full[s], par)) {
                    if (lane == 0 && P.status) atomicCAS(P.status, 0, (int)ST_ERR_DEVICE_TIMEOUT);
                    break;
                }
                const float* stg = ring + (size_t)s * stage_f;
                const ItemWalk at = w.item();
                if (at.b < lim_b && at.c < lim_c) {
                    // the item's position is needed only for mode 1's stores
                    if (f_act)
                        whole(stg, mode1 ? lam_out + red_item(G, at).gbase + (int64_t)fs.j0 * G.pitch : nullptr);
                } else {
                    acc = red_partial<HAS_B>(acc, G, at, stg, warp, lane, mode1, lam_out);
                }
                __syncwarp();
                if (lane == 0) ptx::mbar_arrive(&empty[s]);
                if (++s == (uint32_t)ns) {
                    s = 0;
                    par ^= 1u;
                }
            }
        }
    }
    const Red3 r = block_red_ff(acc);
    if (threadIdx.x == 0) {
        partials[3 * blockIdx.x + 0] = r.s;
        partials[3 * blockIdx.x + 1] = r.q;
        partials[3 * blockIdx.x + 2] = r.m;
    }
}

__global__ void __launch_bounds__(256)
k_reduce_final(const double* __restrict__ partials, int nblocks, double* __restrict__ out, int mode)
{
    ptx::griddep_wait();  // the partial kernel's results
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
int sm_count()
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm <= 0) nsm = 148;
    }
    return nsm;
}

// Blocks of one reduction kernel instance resident at once on this GPU.
int resident_blocks(const void* fn)
{
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 256, 0) != cudaSuccess || occ <= 0) {
        (void)cudaGetLastError();
        occ = 1;
    }
    return sm_count() * occ;
}

int64_t blocks_by_rows(const Geom& g) { return std::max<int64_t>(1, (g.nz * g.ny + 7) / 8); }
}  // namespace

int reduce_blocks(const Geom& g, int max_blocks)
{
    static int resident = 0;  // the most blocks any reduction kernel instance keeps resident
    if (resident == 0)
        for (const void* f : {(const void*)k_reduce_partial<double, true>, (const void*)k_reduce_partial<double, false>})
            resident = std::max(resident, resident_blocks(f));
    return (int)std::min<int64_t>(std::min<int64_t>(resident, max_blocks), blocks_by_rows(g));
}

namespace {
// Stage and ring sizes of k_reduce_ring: 36 KB per stage (one array of 9216
// floats, or two of 4608), three stages per block, two blocks per SM.
constexpr int RR_STAGE = 9216;
constexpr int RR_NS = 3;

cudaError_t launch_reduce_ring(const float* a, const float* b, const Geom& g, double* partials, int nblocks,
                               int mode, float* lam_out, int* status, cudaStream_t s, int* used_blocks)
{
    RedRing P{};
    P.nz = g.nz;
    P.ny = g.ny;
    P.nx = g.nx;
    P.pitch = g.pitch;
    P.plane = g.plane;
    P.origin = g.origin;
    P.xl = g.xl;
    P.r = g.r;
    P.rz = g.rz;
    P.se = b ? RR_STAGE / 2 : RR_STAGE;
    P.ns = RR_NS;
    if (g.pitch <= P.se) {
        P.rpi = (int)std::min<int64_t>(RR_CW, P.se / g.pitch);
        P.nseg = 1;
        P.ipp = (g.ny + P.rpi - 1) / P.rpi;
        P.items = g.nz * P.ipp;
    } else {
        P.rpi = 0;
        P.nseg = (int)((g.nx + P.se - 1) / P.se);
        P.ipp = 0;
        P.items = g.nz * g.ny * P.nseg;
    }
    P.mode = mode;
    P.all_whole = P.rpi > 0 ? (g.ny % P.rpi == 0) : (g.nx % P.se == 0);
    P.status = status;
    const size_t smem = (size_t)RR_NS * RR_STAGE * sizeof(float) + 2 * (size_t)RR_NS * sizeof(uint64_t);
    static int per_sm[2] = {0, 0};
    const int bi = b != nullptr;
    if (per_sm[bi] == 0) {
        const void* fn = bi ? (const void*)k_reduce_ring<true> : (const void*)k_reduce_ring<false>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        int occ = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, (RR_CW + 1) * 32, smem);
        if (e != cudaSuccess) return e;
        per_sm[bi] = std::max(1, occ);
    }
    const int nb = (int)std::max<int64_t>(
        1, std::min<int64_t>(std::min(nblocks, per_sm[bi] * sm_count()), P.items));
    *used_blocks = nb;
    const dim3 block((RR_CW + 1) * 32);
    if (b) return launch_dependent(k_reduce_ring<true>, dim3(nb), block, smem, s, a, b, P, partials, lam_out);
    return launch_dependent(k_reduce_ring<false>, dim3(nb), block, smem, s, a, (const float*)nullptr, P, partials,
                            lam_out);
}
}  // namespace

cudaError_t launch_reduce(int esize, const void* a, const void* b, const Geom& g, double* partials,
                          int nblocks, double* out, int mode, void* lam_out, int* status, cudaStream_t s)
{
    if (esize == 4) {
        // FP32: the ring-staged kernel, two blocks per SM (at most nblocks)
        int nb = 1;
        cudaError_t e = launch_reduce_ring((const float*)a, (const float*)b, g, partials, nblocks, mode,
                                           (float*)lam_out, status, s, &nb);
        if (e != cudaSuccess) return e;
        return launch_dependent(k_reduce_final, dim3(1), dim3(256), 0, s, (const double*)partials, nb, out, mode);
    }
    // FP64 (bound by the FP64 pipe, not by loads): the blocks of this kernel
    // instance that are resident at once (no partial second wave), within the
    // caller's partials
    static int res[2] = {0, 0};
    const int bi = b != nullptr;
    if (res[bi] == 0)
        res[bi] = resident_blocks(bi ? (const void*)k_reduce_partial<double, true>
                                     : (const void*)k_reduce_partial<double, false>);
    nblocks = (int)std::max<int64_t>(1, std::min<int64_t>(std::min(nblocks, res[bi]), blocks_by_rows(g)));
    if (b)
        k_reduce_partial<double, true><<<nblocks, 256, 0, s>>>((const double*)a, (const double*)b, g, partials, mode,
                                                               (double*)lam_out);
    else
        k_reduce_partial<double, false><<<nblocks, 256, 0, s>>>((const double*)a, nullptr, g, partials, mode,
                                                                (double*)lam_out);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_dependent(k_reduce_final, dim3(1), dim3(256), 0, s, (const double*)partials, nblocks, out, mode);
}

// dev_out = the combination of nblocks (sum, sum of squares, max) partials
// (the second kernel of a reduction whose first pass ran elsewhere).
cudaError_t launch_reduce_final(const double* partials, int nblocks, double* out, cudaStream_t s)
{
    return launch_dependent(k_reduce_final, dim3(1), dim3(256), 0, s, partials, nblocks, out, 0);
}

}  // namespace st
