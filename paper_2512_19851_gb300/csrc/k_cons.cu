// Per-cell diffusion in conservative (face-averaged) form, its transpose and
// the coefficient gradient: the paper's per-point stencil update
// u_{t+1}[p] = sum_k w_k(p) u_t[p + o_k] (Sec. III-A) with weights built from
// face coefficients, so that a periodic grid conserves the sum of u for any
// coefficient field:
//
//   u'[p] = u[p] + sum over the axis neighbours q of p of k_pq (u[q] - u[p]),
//   k_pq  = (kappa[p] + kappa[q]) / 2 for an interior (or wrapped) q,
//   k_pq  = kappa[p] for a Dirichlet ghost q (whose u holds the boundary value).
//
// The matrix of the map is symmetric (k_pq = k_qp), so one transposed step
// is the same sweep applied to lambda, whose ghost cells are 0.  The
// gradient term of a step at p gathers the derivatives of every face term
// that holds kappa[p]:
//   g[p] += sum over interior q of (u[q] - u[p]) (lambda[p] - lambda[q]) / 2
//         + sum over ghost q    of (u[q] - u[p]) lambda[p].
//
// Each thread marches up a column of planes (z reuse in registers), its
// in-plane neighbours coming through L1/L2, so DRAM sees about one read of u
// and kappa and one write per point.
#include "families.cuh"
#include "ptx.cuh"

namespace st {

namespace {

constexpr int CZ = 16;  // planes a thread marches through

__device__ __forceinline__ int64_t wrapc(int64_t i, int64_t n) { return i < 0 ? i + n : (i >= n ? i - n : i); }

// Thread (x, y) of a 32 x 8 block marches up CZ planes of its column, keeping
// the column's values at z - 1, z and z + 1 in registers (z reuse); its
// in-plane neighbours come from L1/L2, where the neighbouring threads' own
// centre loads put them.  Neighbour order in every sum: -z, +z, -y, +y, -x,
// +x.  Dirichlet: a ghost neighbour's u is the ghost cell (the boundary
// value) and its face takes kappa[p]; periodic: indices wrap.
struct Col {
    int64_t xm, xp, ym, yp;  // offsets of the in-plane neighbours from the column
    bool ixm, ixp, iym, iyp; // interior?
};

template <bool PER>
__device__ __forceinline__ Col make_col(const GenParams& P, int64_t y, int64_t x)
{
    Col c;
    if (PER) {
        c.xm = wrapc(x - 1, P.nx) - x;
        c.xp = wrapc(x + 1, P.nx) - x;
        c.ym = (wrapc(y - 1, P.ny) - y) * P.pitch;
        c.yp = (wrapc(y + 1, P.ny) - y) * P.pitch;
        c.ixm = c.ixp = c.iym = c.iyp = true;
    } else {
        c.xm = -1;
        c.xp = 1;
        c.ym = -P.pitch;
        c.yp = P.pitch;
        c.ixm = x > 0;
        c.ixp = x + 1 < P.nx;
        c.iym = y > 0;
        c.iyp = y + 1 < P.ny;
    }
    return c;
}

// linear index of plane z of the column (wrapped when periodic; Dirichlet
// planes -1 and nz are the ghost planes)
template <bool PER>
__device__ __forceinline__ int64_t plane_at(const GenParams& P, int64_t col, int64_t z)
{
    return col + (PER ? wrapc(z, P.nz) : z) * P.plane;
}

template <typename T>
__device__ __forceinline__ T face(bool inside, T kp, T kq)
{
    return inside ? (kp + kq) * T(0.5) : kp;
}

template <typename T, bool PER, bool THREE>
__global__ void __launch_bounds__(256) k_cons_sweep(const T* __restrict__ in, T* __restrict__ out,
                                                    const T* __restrict__ kap, const __grid_constant__ GenParams P)
{
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int64_t x = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int64_t z0 = (int64_t)blockIdx.z * CZ, z1 = z0 + CZ < P.nz ? z0 + CZ : P.nz;
    const Col c = make_col<PER>(P, y, x);
    const int64_t col = P.origin + y * P.pitch + x;
    T um = T(0), km = T(0), uc, kc;
    int64_t pc = plane_at<PER>(P, col, z0);
    uc = in[pc];
    kc = kap[pc];
    if (THREE) {
        const int64_t pm = plane_at<PER>(P, col, z0 - 1);
        um = in[pm];
        km = (PER || z0 > 0) ? kap[pm] : kc;
    }
    for (int64_t z = z0; z < z1; ++z) {
        T up = T(0), kq = T(0);
        bool izp = true, izm = true;
        if (THREE) {
            const int64_t pp = plane_at<PER>(P, col, z + 1);
            up = in[pp];
            izp = PER || z + 1 < P.nz;
            izm = PER || z > 0;
            kq = izp ? kap[pp] : kc;
        }
        T acc = T(0);
        if (THREE) {
            acc = fma(face(izm, kc, km), um - uc, acc);
            acc = fma(face(izp, kc, kq), up - uc, acc);
        }
        acc = fma(face(c.iym, kc, c.iym ? kap[pc + c.ym] : kc), in[pc + c.ym] - uc, acc);
        acc = fma(face(c.iyp, kc, c.iyp ? kap[pc + c.yp] : kc), in[pc + c.yp] - uc, acc);
        acc = fma(face(c.ixm, kc, c.ixm ? kap[pc + c.xm] : kc), in[pc + c.xm] - uc, acc);
        acc = fma(face(c.ixp, kc, c.ixp ? kap[pc + c.xp] : kc), in[pc + c.xp] - uc, acc);
        out[pc] = uc + acc;
        um = uc;
        km = kc;
        uc = up;
        kc = kq;
        pc += P.plane;
        if (PER && THREE && z + 1 == P.nz) pc -= P.nz * P.plane;
    }
}

// The transposed step (the same sweep on lambda, whose ghosts are 0) fused
// with the gradient term of the step, both gathered at p:
//   g[p] = sum over interior q of (u[q] - u[p]) (lambda[p] - lambda[q]) / 2
//        + sum over ghost q    of (u[q] - u[p]) lambda[p].
// The term goes to the FP64 gradient as a reduction performed at L2 (the
// thread never waits on the accumulator; a load-add-store exposed the DRAM
// latency every plane: 308 vs 181 us per reverse step at 256^3); each point
// has one thread, so its terms still arrive in step order.  (Loads of plane
// z + 2 issued before plane z is computed made both kernels slower: 87 vs
// 63 us per forward step.)
template <typename T, bool PER, bool THREE>
__global__ void __launch_bounds__(256) k_cons_adjoint(const T* __restrict__ u, const T* __restrict__ lam,
                                                      T* __restrict__ lout, const T* __restrict__ kap,
                                                      double* __restrict__ gk, const __grid_constant__ GenParams P)
{
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int64_t x = (int64_t)blockIdx.x * 32 + threadIdx.x;
    const int64_t y = (int64_t)blockIdx.y * 8 + threadIdx.y;
    if (x >= P.nx || y >= P.ny) return;
    const int64_t z0 = (int64_t)blockIdx.z * CZ, z1 = z0 + CZ < P.nz ? z0 + CZ : P.nz;
    const Col c = make_col<PER>(P, y, x);
    const int64_t col = P.origin + y * P.pitch + x;
    const bool grad = gk != nullptr;
    int64_t pc = plane_at<PER>(P, col, z0);
    T lc = lam[pc], kc = kap[pc], uc = u[pc];
    T lm = T(0), km = T(0), um = T(0);
    if (THREE) {
        const int64_t pm = plane_at<PER>(P, col, z0 - 1);
        const bool in_m = PER || z0 > 0;
        lm = in_m ? lam[pm] : T(0);
        km = in_m ? kap[pm] : kc;
        um = u[pm];
    }
    for (int64_t z = z0; z < z1; ++z) {
        T lq = T(0), kq = kc, uq = T(0);
        bool izp = true, izm = true;
        if (THREE) {
            const int64_t pp = plane_at<PER>(P, col, z + 1);
            izp = PER || z + 1 < P.nz;
            izm = PER || z > 0;
            lq = izp ? lam[pp] : T(0);
            kq = izp ? kap[pp] : kc;
            uq = u[pp];
        }
        T acc = T(0), g = T(0);
        auto term = [&](bool inside, T kn, T ln, T un) {
            acc = fma(face(inside, kc, kn), ln - lc, acc);
            if (grad) {
                const T du = un - uc;
                g += inside ? T(0.5) * du * (lc - ln) : du * lc;
            }
        };
        if (THREE) {
            term(izm, km, lm, um);
            term(izp, kq, lq, uq);
        }
        term(c.iym, c.iym ? kap[pc + c.ym] : kc, c.iym ? lam[pc + c.ym] : T(0), u[pc + c.ym]);
        term(c.iyp, c.iyp ? kap[pc + c.yp] : kc, c.iyp ? lam[pc + c.yp] : T(0), u[pc + c.yp]);
        term(c.ixm, c.ixm ? kap[pc + c.xm] : kc, c.ixm ? lam[pc + c.xm] : T(0), u[pc + c.xm]);
        term(c.ixp, c.ixp ? kap[pc + c.xp] : kc, c.ixp ? lam[pc + c.xp] : T(0), u[pc + c.xp]);
        lout[pc] = lc + acc;
        if (grad) atomicAdd(gk + pc, (double)g);
        lm = lc;
        km = kc;
        um = uc;
        lc = lq;
        kc = kq;
        uc = uq;
        pc += P.plane;
        if (PER && THREE && z + 1 == P.nz) pc -= P.nz * P.plane;
    }
}

// The coefficient gradient of up to GMAX transposed steps in one pass, for
// the reverse pass whose transposed steps run as the forward sweep on lambda
// (the matrix is symmetric): pair k holds the state u_t and lambda_{t+1} of
// one step.  A 32 x 8 block walks GCZ planes; for each plane it brings the
// plane of every pair (tile and a one-cell halo, both fields) into a 4-plane
// shared ring by asynchronous element copies, the next plane's copies in
// flight while the current plane is computed, so a thread keeps up to
// 2 GMAX copies per plane going instead of waiting for one plane at a time.
// Each point adds the pairs' terms (k_cons_adjoint's step term, its face
// products chained by fma) in pair order, in the grid's precision (a sum of
// at most a few terms, each already rounded to that precision), and sends
// the sum to the FP64 gradient as one L2 reduction per launch instead of one
// per step: the accumulation over the run stays in FP64.
constexpr int GMAX = 8;   // pairs per launch
constexpr int GCZ = 32;   // planes per block
constexpr int GTX = 32, GTY = 8, GHY = GTY + 2;
// A staged row holds the tile's 32 columns and one 16-byte group on each
// side (the x halo is its inner element): GW(T) elements, copied as 16-byte
// groups from a 16-byte aligned start (interior rows start 16-byte aligned
// and x0 is a multiple of 32).
template <typename T>
__host__ __device__ constexpr int gvn() { return 16 / (int)sizeof(T); }
template <typename T>
__host__ __device__ constexpr int gw() { return GTX + 2 * gvn<T>(); }
template <typename T>
__host__ __device__ constexpr int gplane() { return GHY * gw<T>(); }

template <typename T>
struct GradPairs {
    const T* u[GMAX];
    const T* lam[GMAX];
    int n;
};

template <typename T>
constexpr size_t grad_smem(int n) { return (size_t)4 * n * 2 * gplane<T>() * sizeof(T); }

template <typename T, bool PER>
__global__ void __launch_bounds__(GTX * GTY) k_cons_grad(const __grid_constant__ GradPairs<T> G,
                                                         double* __restrict__ gk,
                                                         const __grid_constant__ GenParams P, int64_t xend)
{
    constexpr int VN = gvn<T>(), W = gw<T>(), HP = gplane<T>(), NCH = W / VN;  // 16-byte groups per row
    extern __shared__ __align__(16) unsigned char graw[];
    T* ring = reinterpret_cast<T*>(graw);  // [slot 4][pair GMAX][field 2][HP]
    ptx::griddep_wait();
    ptx::griddep_trigger();
    const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * GTX + tx;
    const int64_t x0 = (int64_t)blockIdx.x * GTX, y0 = (int64_t)blockIdx.y * GTY;
    const int64_t x = x0 + tx, y = y0 + ty;
    const int64_t z0 = (int64_t)blockIdx.z * GCZ;
    const int nzc = (int)(P.nz - z0 < GCZ ? P.nz - z0 : GCZ);
    const int n = G.n;
    const bool own = x < P.nx && y < P.ny;
    const bool ixm = PER || x > 0, ixp = PER || x + 1 < P.nx, iym = PER || y > 0, iyp = PER || y + 1 < P.ny;
    auto at = [&](int slot, int k, int f) { return ring + ((size_t)(slot * n + k) * 2 + f) * HP; };
    // This thread's 16-byte group of a staged plane (at most one: GHY * NCH
    // <= the block's threads), fixed for the whole block: staged row hy,
    // group hc, i.e. grid row y0 - 1 + hy and columns x0 - VN + VN hc ...
    // Periodic: a group that crosses the row's wrap is copied element-wise
    // (gidx = -1 marks it); Dirichlet: groups outside the padded row, and rows
    // past the ghost row, are not copied.
    const int hy = tid / NCH, hc = tid - hy * NCH;
    bool cp = tid < GHY * NCH;
    int64_t yy = y0 - 1 + hy;
    const int64_t gx = x0 - VN + (int64_t)VN * hc;  // first column of the group
    bool whole = true;                               // the group copies in one 16-byte piece
    if (cp) {
        if (PER) {
            yy = wrapc(yy, P.ny);
            whole = gx >= 0 && gx + VN <= P.nx;
        } else {
            cp = yy <= P.ny && gx + VN <= xend;  // xend: columns from x = 0 to the padded row's end
        }
    }
    const int so = hy * W + hc * VN;  // shared offset of the group in a plane
    auto issue = [&](int64_t z) {
        if (cp && z <= z0 + nzc) {
            const int slot = (int)((z - z0 + 1) & 3);
            const int64_t zz = PER ? wrapc(z, P.nz) : z;
            const int64_t row = P.origin + zz * P.plane + yy * P.pitch;
            if (whole) {
                for (int k = 0; k < n; ++k) {
                    ptx::cp_async_16(at(slot, k, 0) + so, G.u[k] + row + gx);
                    ptx::cp_async_16(at(slot, k, 1) + so, G.lam[k] + row + gx);
                }
            } else {
                for (int e = 0; e < VN; ++e) {
                    const int64_t xx = wrapc(gx + e, P.nx);
                    for (int k = 0; k < n; ++k) {
                        ptx::cp_async_elem<sizeof(T)>(at(slot, k, 0) + so + e, G.u[k] + row + xx);
                        ptx::cp_async_elem<sizeof(T)>(at(slot, k, 1) + so + e, G.lam[k] + row + xx);
                    }
                }
            }
        }
        ptx::cp_async_commit();
    };
    issue(z0 - 1);
    issue(z0);
    issue(z0 + 1);
    const int c = (ty + 1) * W + tx + VN;
    for (int zi = 0; zi < nzc; ++zi) {
        const int64_t z = z0 + zi;
        issue(z + 2);                    // in flight while plane z is computed
        ptx::cp_async_wait_group<1>();  // planes up to z + 1 have landed
        __syncthreads();
        if (own) {
            // slot bases of planes z - 1, z, z + 1; pair k's fields at
            // offsets 2 k HP (u) and 2 k HP + HP (lambda)
            const T* Rm = ring + (size_t)(zi & 3) * n * 2 * HP;
            const T* Rc = ring + (size_t)((zi + 1) & 3) * n * 2 * HP;
            const T* Rp = ring + (size_t)((zi + 2) & 3) * n * 2 * HP;
            const bool izm = PER || z > 0, izp = PER || z + 1 < P.nz;
            // a face's term (u_q - u_p) w with w = A lambda_p - B lambda_q:
            // interior face A = B = 1/2, ghost face A = 1, B = 0 (the same
            // values as the fused kernel's 1/2 du (lambda_p - lambda_q) and
            // du lambda_p: the halving is exact)
            const T Azm = izm ? T(0.5) : T(1), Bzm = izm ? T(0.5) : T(0);
            const T Azp = izp ? T(0.5) : T(1), Bzp = izp ? T(0.5) : T(0);
            const T Aym = iym ? T(0.5) : T(1), Bym = iym ? T(0.5) : T(0);
            const T Ayp = iyp ? T(0.5) : T(1), Byp = iyp ? T(0.5) : T(0);
            const T Axm = ixm ? T(0.5) : T(1), Bxm = ixm ? T(0.5) : T(0);
            const T Axp = ixp ? T(0.5) : T(1), Bxp = ixp ? T(0.5) : T(0);
            T acc = T(0);  // the pairs' sum (each term is rounded in T already)
            for (int k = 0, o = c; k < n; ++k, o += 2 * HP) {
                const T uc = Rc[o], lc = Rc[o + HP];
                T g = (Rm[o] - uc) * fma(-Bzm, Rm[o + HP], Azm * lc);
                g = fma(Rp[o] - uc, fma(-Bzp, Rp[o + HP], Azp * lc), g);
                g = fma(Rc[o - W] - uc, fma(-Bym, Rc[o - W + HP], Aym * lc), g);
                g = fma(Rc[o + W] - uc, fma(-Byp, Rc[o + W + HP], Ayp * lc), g);
                g = fma(Rc[o - 1] - uc, fma(-Bxm, Rc[o - 1 + HP], Axm * lc), g);
                g = fma(Rc[o + 1] - uc, fma(-Bxp, Rc[o + 1 + HP], Axp * lc), g);
                acc += g;
            }
            atomicAdd(gk + P.origin + z * P.plane + y * P.pitch + x, (double)acc);
        }
        __syncthreads();  // before plane z + 3 reuses plane z - 1's slot
    }
    ptx::cp_async_wait_all();
}

dim3 cons_grid(const GenParams& P)
{
    return dim3((unsigned)((P.nx + 31) / 32), (unsigned)((P.ny + 7) / 8), (unsigned)((P.nz + CZ - 1) / CZ));
}

template <typename T>
cudaError_t sweep_t(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    const GenParams& P = f.gp;
    const dim3 g = cons_grid(P), b(32, 8);
    const T* in = (const T*)a.in;
    const T* k = (const T*)a.kappa;
    T* o = (T*)a.out;
    const bool three = f.g.ndim == 3;
    if (f.periodic)
        return three ? launch_dependent(k_cons_sweep<T, true, true>, g, b, 0, s, in, o, k, P)
                     : launch_dependent(k_cons_sweep<T, true, false>, g, b, 0, s, in, o, k, P);
    return three ? launch_dependent(k_cons_sweep<T, false, true>, g, b, 0, s, in, o, k, P)
                 : launch_dependent(k_cons_sweep<T, false, false>, g, b, 0, s, in, o, k, P);
}

template <typename T>
cudaError_t adjoint_t(const Family& f, const AdjointArgs& a, cudaStream_t s)
{
    const GenParams& P = f.gp;
    const dim3 g = cons_grid(P), b(32, 8);
    const T* u = (const T*)a.u;
    const T* l = (const T*)a.lam_in;
    const T* k = (const T*)a.kappa;
    T* o = (T*)a.lam_out;
    const bool three = f.g.ndim == 3;
    if (f.periodic)
        return three ? launch_dependent(k_cons_adjoint<T, true, true>, g, b, 0, s, u, l, o, k, a.gk, P)
                     : launch_dependent(k_cons_adjoint<T, true, false>, g, b, 0, s, u, l, o, k, a.gk, P);
    return three ? launch_dependent(k_cons_adjoint<T, false, true>, g, b, 0, s, u, l, o, k, a.gk, P)
                 : launch_dependent(k_cons_adjoint<T, false, false>, g, b, 0, s, u, l, o, k, a.gk, P);
}

}  // namespace

cudaError_t launch_cons_sweep(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    const GenParams& P = f.gp;
    if (P.nz * P.ny * P.nx == 0) return cudaSuccess;
    if (f.variant == 1) return launch_star3d_cons(f, a, s);
    return f.g.esize == 8 ? sweep_t<double>(f, a, s) : sweep_t<float>(f, a, s);
}

cudaError_t launch_cons_grad(const Family& f, const void* const* u, const void* const* lam, int n, double* gk,
                             cudaStream_t s)
{
    const GenParams& P = f.gp;
    if (P.nz * P.ny * P.nx == 0 || n <= 0) return cudaSuccess;
    if (f.g.ndim != 3 || n > GMAX) return cudaErrorInvalidValue;
    const dim3 g((unsigned)((P.nx + GTX - 1) / GTX), (unsigned)((P.ny + GTY - 1) / GTY),
                 (unsigned)((P.nz + GCZ - 1) / GCZ)),
        b(GTX, GTY);
    auto go = [&](auto zero) -> cudaError_t {
        using T = decltype(zero);
        GradPairs<T> G{};
        G.n = n;
        for (int k = 0; k < n; ++k) {
            G.u[k] = static_cast<const T*>(u[k]);
            G.lam[k] = static_cast<const T*>(lam[k]);
        }
        const size_t smem = grad_smem<T>(n);
        auto fn = f.periodic ? k_cons_grad<T, true> : k_cons_grad<T, false>;
        cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)grad_smem<T>(GMAX));
        if (e != cudaSuccess) return e;
        return launch_dependent(fn, g, b, smem, s, G, gk, P, (int64_t)(f.g.pitch - f.g.xl));
    };
    return f.g.esize == 8 ? go(0.0) : go(0.f);
}

// Pairs per launch for the reverse pass: up to 5 keeps three blocks of
// 64 KB (FP32) resident per SM.
int cons_grad_max_pairs() { return 5; }

cudaError_t launch_cons_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s)
{
    if (a.steps != 1) return cudaErrorInvalidValue;
    const GenParams& P = f.gp;
    if (P.nz * P.ny * P.nx == 0) return cudaSuccess;
    return f.g.esize == 8 ? adjoint_t<double>(f, a, s) : adjoint_t<float>(f, a, s);
}

}  // namespace st
