// Family selection and dispatch.
#include <cstring>

#include "families.cuh"

namespace st {

static GenParams make_gen_params(const FamilyDesc& d)
{
    GenParams P;
    std::memset(&P, 0, sizeof(P));
    const Geom& g = d.g;
    P.nz = g.nz;
    P.ny = g.ny;
    P.nx = g.nx;
    P.pitch = g.pitch;
    P.plane = g.plane;
    P.origin = g.origin;
    P.npts = d.npts;
    P.periodic = d.periodic ? 1 : 0;
    P.leapfrog = d.levels == 2 ? 1 : 0;
    P.has_kappa = d.has_beta ? 1 : 0;
    P.src = -1;
    for (int k = 0; k < d.npts; ++k) {
        P.dz[k] = d.off[3 * k];
        P.dy[k] = d.off[3 * k + 1];
        P.dx[k] = d.off[3 * k + 2];
        P.lin[k] = (int64_t)P.dz[k] * g.plane + (int64_t)P.dy[k] * g.pitch + P.dx[k];
        P.alpha[k] = d.alpha[k];
        P.beta[k] = d.has_beta ? d.beta[k] : 0.0;
    }
    gen_params_floats(P);
    return P;
}

Family select_family(const FamilyDesc& d)
{
    Family f;
    std::memset(&f, 0, sizeof(f));
    f.kind = FAM_GENERIC;
    f.name = "generic_point";
    f.gp = make_gen_params(d);
    f.g = d.g;
    f.periodic = d.periodic;
    f.has_beta = d.has_beta;
    f.levels = d.levels;
    if (d.force_generic) return f;
    int variant = 0;
    const char* name = nullptr;
    const bool wave = d.g.ndim == 3 && d.star && wave_supports(d);
    if (wave || (d.g.ndim == 3 && d.star && star3d_supports(d, &variant, &name))) {
        f.kind = wave ? FAM_WAVE : FAM_STAR3D;
        f.variant = variant;
        f.name = wave ? "wave3d_r4_bulk_zqueue" : name;
        // per-axis coefficients
        StarCoef& c = f.sc;
        int R = 0;
        for (int k = 0; k < d.npts; ++k) {
            const int32_t* o = d.off + 3 * k;
            int ax = o[0] ? 0 : (o[1] ? 1 : (o[2] ? 2 : -1));
            if (ax < 0) {
                c.c_a += d.alpha[k];
                c.c_b += d.has_beta ? d.beta[k] : 0.0;
                continue;
            }
            const int v = o[ax];
            const int j = v < 0 ? -v : v;
            const int side = v > 0 ? 1 : 0;
            c.a[ax][side][j - 1] += d.alpha[k];
            c.b[ax][side][j - 1] += d.has_beta ? d.beta[k] : 0.0;
            if (j > R) R = j;
        }
        c.R = R;
    } else if (d.g.ndim == 2 && tile2d_supports(d, &variant, &name)) {
        f.kind = FAM_2D_TILE;
        f.variant = variant;
        f.name = name;
    }
    return f;
}

cudaError_t launch_family(const Family& f, const SweepArgs& a, cudaStream_t s)
{
    switch (f.kind) {
    case FAM_STAR3D:
        return launch_star3d(f, a, s);
    case FAM_2D_TILE:
        return launch_tile2d(f, a, s);
    case FAM_WAVE:
        return launch_wave(f, a, s);
    case FAM_CONS:
        return launch_cons_sweep(f, a, s);
    default: {
        GenParams P = f.gp;
        P.src = a.src;
        P.src_amp = a.src_amp;
        P.src_count = a.src_count;
        P.step = a.step;
        return launch_generic_sweep(f.g.esize, a.in, a.out, a.prev, a.kappa, P, s);
    }
    }
}

cudaError_t launch_family_adjoint(const Family& f, const AdjointArgs& a, cudaStream_t s)
{
    if (f.kind == FAM_CONS) return launch_cons_adjoint(f, a, s);
    if (f.kind == FAM_STAR3D && star3d_adjoint_fuse(f) >= a.steps) return launch_star3d_adjoint(f, a, s);
    if (a.steps != 1) return cudaErrorInvalidValue;  // callers fuse only what the family supports
    return launch_generic_adjoint(f.g.esize, a.u, a.lam_in, a.lam_out, a.kappa, a.gk, f.gp, s);
}

}  // namespace st
