/*
 * Plain CPU oracle for the stencil sweeps of "An Adaptive Distributed Stencil
 * Abstraction for GPUs" (CharmStencil).  TEST INFRASTRUCTURE ONLY: it is
 * linked by the tests, by the package's smoke check and by the CPU-baseline
 * leg of the benchmark, never by the product path.  It shares no code, header
 * or constant with the CUDA library.
 *
 * Every routine is the plain definition written out with loops, in a fixed
 * and stated summation order, compiled with -ffp-contract=off so that no
 * multiply-add is fused.  The same source is compiled twice: with REAL=double
 * (the reference results) and with REAL=float (used only to measure how far a
 * single-precision evaluation of the same definition drifts).
 *
 * Arrays are dense interiors in C order: index (z, y, x), x fastest.  A 2D
 * grid is passed as nz = 1; a neighbour offset is (dz, dy, dx).  Points
 * outside the interior are the ghost region: with a Dirichlet boundary they
 * read the constant bc_value (the paper's boundary ring written once by slice
 * assignment and never updated, Example 1 in Sec. III-A); with a periodic
 * boundary the index wraps modulo the extent.
 *
 * OpenMP is used only across the slowest axis of gather loops (no reduction
 * inside), so a threaded run is bitwise identical to a serial one.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef REAL
#define REAL double
#endif

#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_CAT2(a, b) a##b
#define ORC_CAT(a, b) ORC_CAT2(a, b)
#ifndef ORC_SUFFIX
#define ORC_SUFFIX _f64
#endif
#define ORC(name) ORC_CAT(name, ORC_SUFFIX)

static int64_t orc_wrap(int64_t i, int64_t n)
{
    while (i < 0) i += n;
    while (i >= n) i -= n;
    return i;
}

/* Value of field f at (z, y, x), which may lie outside the interior. */
static REAL orc_read(const REAL* f, int64_t nz, int64_t ny, int64_t nx,
                     int64_t z, int64_t y, int64_t x, int periodic, REAL bc_value)
{
    if (periodic) {
        z = orc_wrap(z, nz);
        y = orc_wrap(y, ny);
        x = orc_wrap(x, nx);
    } else if (z < 0 || z >= nz || y < 0 || y >= ny || x < 0 || x >= nx) {
        return bc_value;
    }
    return f[(z * ny + y) * nx + x];
}

static int orc_inside(int64_t nz, int64_t ny, int64_t nx, int64_t z, int64_t y, int64_t x)
{
    return z >= 0 && z < nz && y >= 0 && y < ny && x >= 0 && x < nx;
}

static void orc_threads(int nthreads)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

/*
 * Constant-weight stencil sweep (the update of Example 1, Sec. III-A, in its
 * general form u_{t+1}[p] = sum_k w_k u_t[p + o_k]): for every interior point
 * the weighted neighbour values are added in the order the offsets are given,
 * starting from zero, into a second array (the paper's two-array, Jacobi form:
 * the output is never read in the same step).  After each step the arrays
 * swap roles, as `u1, u2 = u2, u1` does in Example 1.  On return u holds
 * u_nsteps; tmp is scratch of the same size.
 */
void ORC(orc_sweep_const)(int64_t nz, int64_t ny, int64_t nx, int npts,
                          const int32_t* off, const double* w, int periodic,
                          double bc_value, int nsteps, REAL* u, REAL* tmp, int nthreads)
{
    REAL* src = u;
    REAL* dst = tmp;
    REAL wr[64];
    REAL bc = (REAL)bc_value;
    int64_t n = nz * ny * nx;
    for (int k = 0; k < npts && k < 64; ++k) wr[k] = (REAL)w[k];
    orc_threads(nthreads);
    for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    REAL acc = (REAL)0;
                    for (int k = 0; k < npts; ++k) {
                        REAL v = orc_read(src, nz, ny, nx, z + off[3 * k], y + off[3 * k + 1],
                                          x + off[3 * k + 2], periodic, bc);
                        acc = acc + wr[k] * v;
                    }
                    dst[(z * ny + y) * nx + x] = acc;
                }
        REAL* t = src;
        src = dst;
        dst = t;
    }
    if (src != u) memcpy(u, src, (size_t)n * sizeof(REAL));
}

/*
 * Variable-coefficient 7-point diffusion with one diffusivity per cell:
 *   u_{t+1}[p] = (1 - 6 kappa_p) u_t[p] + kappa_p (u[x-1] + u[x+1] + u[y-1]
 *                + u[y+1] + u[z-1] + u[z+1]),
 * the neighbours added in that order.  If states is not NULL, u_0 .. u_nsteps
 * are stored there, one dense interior after another.
 */
void ORC(orc_varcoef7)(int64_t nz, int64_t ny, int64_t nx, const REAL* kappa, int periodic,
                       double bc_value, int nsteps, REAL* u, REAL* tmp, REAL* states,
                       int nthreads)
{
    REAL* src = u;
    REAL* dst = tmp;
    REAL bc = (REAL)bc_value;
    int64_t n = nz * ny * nx;
    orc_threads(nthreads);
    if (states) memcpy(states, u, (size_t)n * sizeof(REAL));
    for (int s = 0; s < nsteps; ++s) {
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    int64_t p = (z * ny + y) * nx + x;
                    REAL nb = orc_read(src, nz, ny, nx, z, y, x - 1, periodic, bc);
                    nb = nb + orc_read(src, nz, ny, nx, z, y, x + 1, periodic, bc);
                    nb = nb + orc_read(src, nz, ny, nx, z, y - 1, x, periodic, bc);
                    nb = nb + orc_read(src, nz, ny, nx, z, y + 1, x, periodic, bc);
                    nb = nb + orc_read(src, nz, ny, nx, z - 1, y, x, periodic, bc);
                    nb = nb + orc_read(src, nz, ny, nx, z + 1, y, x, periodic, bc);
                    REAL k = kappa[p];
                    dst[p] = ((REAL)1 - (REAL)6 * k) * src[p] + k * nb;
                }
        if (states) memcpy(states + (int64_t)(s + 1) * n, dst, (size_t)n * sizeof(REAL));
        REAL* t = src;
        src = dst;
        dst = t;
    }
    if (src != u) memcpy(u, src, (size_t)n * sizeof(REAL));
}

/*
 * Adjoint (transpose) of orc_varcoef7 over one run of nsteps steps.
 * states holds u_0 .. u_{nsteps-1}; lam holds lambda_nsteps on entry and
 * lambda_0 on return; gk receives  += sum_t lambda_{t+1}[p] * du_{t+1}[p]/dkappa_p
 * where du_{t+1}[p]/dkappa_p = (sum of the 6 neighbours of u_t) - 6 u_t[p]
 * (ghost neighbours read bc_value).
 *
 * lambda_t = S^T lambda_{t+1} is evaluated by SCATTER, the literal transpose:
 * every interior p sends w_k(p) lambda_{t+1}[p] to the point p + o_k it read
 * in the forward step, if that point is a variable (interior; wrapped when
 * periodic).  Ghost cells are boundary data, not variables, and receive
 * nothing.  To keep the scatter race-free under OpenMP the z-planes are
 * visited in three passes (z = 0, 3, 6, ...; then 1, 4, ...; then 2, 5, ...),
 * so each target plane has one writer per pass and the order of the partial
 * sums does not depend on the thread count.  With a periodic boundary and an
 * extent nz that is not a multiple of three, the first and last planes of one
 * pass would share a target plane, so that case runs serially.
 */
void ORC(orc_varcoef7_adjoint)(int64_t nz, int64_t ny, int64_t nx, const REAL* kappa,
                               int periodic, double bc_value, int nsteps, const REAL* states,
                               REAL* lam, REAL* lam_tmp, REAL* gk, int nthreads)
{
    REAL bc = (REAL)bc_value;
    int64_t n = nz * ny * nx;
    REAL* lin = lam;    /* lambda_{t+1} */
    REAL* lout = lam_tmp; /* lambda_t   */
    static const int dz6[6] = {0, 0, 0, 0, -1, 1};
    static const int dy6[6] = {0, 0, -1, 1, 0, 0};
    static const int dx6[6] = {-1, 1, 0, 0, 0, 0};
    int serial = periodic && (nz % 3) != 0;
    orc_threads(nthreads);
    for (int t = nsteps - 1; t >= 0; --t) {
        const REAL* ut = states + (int64_t)t * n;
        memset(lout, 0, (size_t)n * sizeof(REAL));
        for (int pass = 0; pass < 3; ++pass) {
#pragma omp parallel for schedule(static) if (!serial)
            for (int64_t z = pass; z < nz; z += 3)
                for (int64_t y = 0; y < ny; ++y)
                    for (int64_t x = 0; x < nx; ++x) {
                        int64_t p = (z * ny + y) * nx + x;
                        REAL lp = lin[p];
                        REAL k = kappa[p];
                        /* centre weight 1 - 6 kappa_p */
                        lout[p] = lout[p] + ((REAL)1 - (REAL)6 * k) * lp;
                        /* neighbour weights kappa_p */
                        REAL nb = (REAL)0;
                        for (int j = 0; j < 6; ++j) {
                            int64_t qz = z + dz6[j], qy = y + dy6[j], qx = x + dx6[j];
                            nb = nb + orc_read(ut, nz, ny, nx, qz, qy, qx, periodic, bc);
                            if (periodic) {
                                qz = orc_wrap(qz, nz);
                                qy = orc_wrap(qy, ny);
                                qx = orc_wrap(qx, nx);
                            } else if (!orc_inside(nz, ny, nx, qz, qy, qx)) {
                                continue;
                            }
                            int64_t q = (qz * ny + qy) * nx + qx;
                            lout[q] = lout[q] + k * lp;
                        }
                        gk[p] = gk[p] + lp * (nb - (REAL)6 * ut[p]);
                    }
        }
        REAL* tt = lin;
        lin = lout;
        lout = tt;
    }
    if (lin != lam) memcpy(lam, lin, (size_t)n * sizeof(REAL));
}

/*
 * Leapfrog acoustic wave step with a radius-4 star Laplacian:
 *   u^{n+1}[p] = 2 u^n[p] - u^{n-1}[p] + m_p * L u^n[p] + s_n [p == src]
 *   L u[p] = sum over axes (z, y, x) of ( a_0 u[p] + sum_{j=1..4} a_j (u[p + j e] + u[p - j e]) )
 * a[0..4] are the stencil coefficients (already divided by h^2 or folded
 * into m), m_p the per-cell factor (c_p dt / h)^2, s_n the source amplitude
 * of step n added at the single interior cell src (src < 0: no source).
 * On entry un = u^0, unm1 = u^{-1}; on return un = u^nsteps, unm1 =
 * u^{nsteps-1}.  The new level overwrites the oldest one (each point of
 * u^{n+1} needs only its own point of u^{n-1}).
 */
void ORC(orc_wave25)(int64_t nz, int64_t ny, int64_t nx, const double* a, const REAL* m,
                     int periodic, double bc_value, int64_t src, const double* s, int nsteps,
                     REAL* un, REAL* unm1, int nthreads)
{
    REAL* cur = un;
    REAL* old = unm1;
    REAL bc = (REAL)bc_value;
    REAL ar[5];
    int64_t n = nz * ny * nx;
    for (int j = 0; j < 5; ++j) ar[j] = (REAL)a[j];
    orc_threads(nthreads);
    for (int st = 0; st < nsteps; ++st) {
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    int64_t p = (z * ny + y) * nx + x;
                    REAL c = cur[p];
                    REAL lz = ar[0] * c, ly = ar[0] * c, lx = ar[0] * c;
                    for (int j = 1; j <= 4; ++j) {
                        lz = lz + ar[j] * (orc_read(cur, nz, ny, nx, z + j, y, x, periodic, bc) +
                                           orc_read(cur, nz, ny, nx, z - j, y, x, periodic, bc));
                        ly = ly + ar[j] * (orc_read(cur, nz, ny, nx, z, y + j, x, periodic, bc) +
                                           orc_read(cur, nz, ny, nx, z, y - j, x, periodic, bc));
                        lx = lx + ar[j] * (orc_read(cur, nz, ny, nx, z, y, x + j, periodic, bc) +
                                           orc_read(cur, nz, ny, nx, z, y, x - j, periodic, bc));
                    }
                    REAL lap = lz + ly + lx;
                    REAL v = (REAL)2 * c - old[p] + m[p] * lap;
                    if (p == src) v = v + (REAL)s[st];
                    old[p] = v;
                }
        REAL* t = cur;
        cur = old;
        old = t;
    }
    if (cur != un) {
        /* odd step count: levels ended up swapped */
        for (int64_t i = 0; i < n; ++i) {
            REAL t = un[i];
            un[i] = unm1[i];
            unm1[i] = t;
        }
    }
}

/*
 * Reductions over n values of a - b (b may be NULL: b = 0), accumulated in
 * double precision in index order:
 *   out[0] = sum (a - b), out[1] = sum (a - b)^2, out[2] = max |a - b|.
 */
void ORC(orc_reduce)(int64_t n, const REAL* a, const REAL* b, double* out)
{
    double s = 0.0, q = 0.0, mx = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double d = (double)a[i] - (b ? (double)b[i] : 0.0);
        s = s + d;
        q = q + d * d;
        double ad = d < 0 ? -d : d;
        if (ad > mx) mx = ad;
    }
    out[0] = s;
    out[1] = q;
    out[2] = mx;
}
