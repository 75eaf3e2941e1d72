// sc_mfie_host.cpp -- host side of the first correction beyond physical
// optics (Sec. II's Liouville-Neumann series of the MFIE; kernels in
// sc_mfie.cu): node geometry, the beam's Zernike path as polynomials for the
// device, the polar rule, and the launches per chunk of omegas.
#include <math.h>

#include <algorithm>

#include "sc_host.h"

namespace sch {

const char* mfie_unsupported(const sc_mirror_t* m, const sc_incident_t* in)
{
    if (m->r_min != 0.0) return "the MFIE correction needs a disk (r_min = 0): its rays run from each node to the rim";
    if (in->profile > SC_PROFILE_TOPHAT)
        return "the MFIE correction needs a collimated beam (Gaussian, super-Gaussian or top-hat)";
    if (in->order != 0) return "the MFIE correction needs a beam of order 0";
    return nullptr;
}

namespace {

// c_j Z_j in the device form P(u^2 + v^2) {1, Re, Im}((u + iv)^|m|):
// R_n^|m|(rho) = sum_s c_s rho^(n - 2s) = rho^|m| sum_s c_s (rho^2)^((n - |m|)/2 - s).
sc::MfieZern zern_term(int j, double coef)
{
    int n, m;
    noll_nm(j, n, m);
    const int am = m < 0 ? -m : m;
    sc::MfieZern z{};
    z.m = am;
    z.kind = m == 0 ? 0 : (m > 0 ? 1 : 2);
    z.deg = (n - am) / 2;
    const double nrm = (m == 0 ? sqrt(n + 1.0) : sqrt(2.0 * (n + 1.0))) * coef;
    for (int s = 0; s <= z.deg; ++s) {
        const double c = ((s & 1) ? -1.0 : 1.0) * tgamma(n - s + 1.0) /
                         (tgamma(s + 1.0) * tgamma((n + am) / 2 - s + 1.0) * tgamma((n - am) / 2 - s + 1.0));
        z.p[z.deg - s] = c * nrm;
    }
    return z;
}

}  // namespace

sc_status mfie_correction(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in, int n_omega,
                          const double* d_pts, int n_points, const double* d_amp, const double* d_k, void* dE,
                          void* dB, bool f64)
{
    if (const char* why = mfie_unsupported(m, in)) return fail(ctx, SC_ERR_INVALID, "%s", why);
    // surface nodes in the node table's order (ring i, angle l): x, y, z, dS
    std::vector<double> gr, gw;
    radial_rule(m, gr, gw);
    const int nr = m->q.n_r, nt = m->q.n_theta;
    const double dth = 2.0 * kPi / nt;
    std::vector<double4> geo((size_t)nr * nt);
    for (int i = 0; i < nr; ++i) {
        const SurfPt sp = surf_at(m, gr[i]);
        const double dS = sqrt(1.0 + sp.dzdr * sp.dzdr) * gr[i] * gw[i] * dth;
        for (int l = 0; l < nt; ++l)
            geo[(size_t)i * nt + l] = make_double4(gr[i] * cos(l * dth), gr[i] * sin(l * dth), sp.z, dS);
    }
    std::vector<sc::MfieZern> zern;
    for (size_t i = 0; i < in->zern.size(); ++i)
        if (in->zern[i] != 0.0) zern.push_back(zern_term((int)i + 2, in->zern[i]));
    std::vector<double> gl(2 * (size_t)ctx->mfie_rho), gx, gwr;
    gauss_legendre(ctx->mfie_rho, 0.0, 1.0, gx, gwr);
    std::copy(gx.begin(), gx.end(), gl.begin());
    std::copy(gwr.begin(), gwr.end(), gl.begin() + ctx->mfie_rho);

    sc_status st;
    const size_t ns = geo.size();
    if ((st = ensure(ctx, ctx->mfie_geo, ns * sizeof(double4))) != SC_OK) return st;
    if ((st = ensure(ctx, ctx->mfie_gl, gl.size() * sizeof(double))) != SC_OK) return st;
    if (!zern.empty() && (st = ensure(ctx, ctx->mfie_zern, zern.size() * sizeof(sc::MfieZern))) != SC_OK)
        return st;
    // dJ for a chunk of omegas: at most 512 MiB
    const size_t per_omega = ns * 3 * sizeof(double2);
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>(n_omega, (size_t(512) << 20) / per_omega));
    if ((st = ensure(ctx, ctx->mfie_dJ, (size_t)chunk * per_omega)) != SC_OK) return st;
    SC_CUDA(cudaMemcpyAsync(ctx->mfie_geo.p, geo.data(), ns * sizeof(double4), cudaMemcpyHostToDevice, ctx->stream),
            "upload MFIE nodes");
    SC_CUDA(cudaMemcpyAsync(ctx->mfie_gl.p, gl.data(), gl.size() * sizeof(double), cudaMemcpyHostToDevice,
                            ctx->stream), "upload MFIE rule");
    if (!zern.empty())
        SC_CUDA(cudaMemcpyAsync(ctx->mfie_zern.p, zern.data(), zern.size() * sizeof(sc::MfieZern),
                                cudaMemcpyHostToDevice, ctx->stream), "upload MFIE Zernike terms");
    // (copies from pageable memory return once the bytes are staged, so the
    // host vectors may go out of scope after them)
    sc::MfieLaunch a{};
    a.surface = m->surface;
    a.f = m->f;
    a.c_ell = m->c;
    a.e_ell = m->e;
    a.zref = m->surface == 2 ? 2.0 * (m->c - m->e) : 2.0 * m->f;
    a.r_max = m->r_max;
    a.profile = in->profile;
    a.sg_order = in->sg_order;
    a.pol = in->pol;
    a.w0 = in->w0;
    a.cos_a = cos(in->angle);
    a.sin_a = sin(in->angle);
    a.zern = (const sc::MfieZern*)ctx->mfie_zern.p;
    a.n_zern = (int)zern.size();
    a.r_norm = m->r_max;
    a.gx = (const double*)ctx->mfie_gl.p;
    a.gw = a.gx + ctx->mfie_rho;
    a.n_rho = ctx->mfie_rho;
    a.n_phi = ctx->mfie_phi;
    a.geo = (const double4*)ctx->mfie_geo.p;
    a.n_surf = (int)ns;
    a.dJ = (double2*)ctx->mfie_dJ.p;
    sc::MfieFieldLaunch b{};
    b.geo = a.geo;
    b.n_surf = a.n_surf;
    b.dJ = a.dJ;
    b.pts = d_pts;
    b.n_pts = n_points;
    b.f64 = f64 ? 1 : 0;
    b.out_stride_omega = (long long)n_points * 3;
    const size_t elem = f64 ? sizeof(double2) : sizeof(float2);
    for (int o0 = 0; o0 < n_omega; o0 += chunk) {
        const int c = std::min(chunk, n_omega - o0);
        a.kval = d_k + o0;
        a.n_omega = c;
        int r = sc::launch_mfie_current(a, ctx->stream);
        if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "MFIE current kernel launch");
        ctx->ctr.launches += r;
        b.kval = d_k + o0;
        b.n_omega = c;
        b.amp = d_amp + 2 * (size_t)o0;
        b.E = (char*)dE + (size_t)o0 * n_points * 3 * elem;
        b.B = dB ? (char*)dB + (size_t)o0 * n_points * 3 * elem : nullptr;
        r = sc::launch_mfie_field(b, ctx->stream);
        if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "MFIE field kernel launch");
        ctx->ctr.launches += r;
    }
    return SC_OK;
}

}  // namespace sch
