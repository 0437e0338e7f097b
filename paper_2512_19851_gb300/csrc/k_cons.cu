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

cudaError_t launch_cons_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s)
{
    if (a.steps != 1) return cudaErrorInvalidValue;
    const GenParams& P = f.gp;
    if (P.nz * P.ny * P.nx == 0) return cudaSuccess;
    return f.g.esize == 8 ? adjoint_t<double>(f, a, s) : adjoint_t<float>(f, a, s);
}

}  // namespace st
