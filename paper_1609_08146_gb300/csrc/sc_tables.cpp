// sc_tables.cpp -- the FP64 host side of the node tables (A1) and spectra (A2):
// radial quadrature, the incident field on the mirror (Sec. III.A),
// the spectrum (Sec. III.B, Eqs. 14-18; Sec. IV.B, Eq. 27), mirror surfaces,
// the node-table builder and cache, and context helpers (errors, events).
#include <math.h>
#include <string.h>

#include <algorithm>
#include <thread>

#include "sc_host.h"

namespace sch {

// f(i) for i in [0, n) on up to 32 host threads (contiguous blocks of i);
// f must only write state of its own i.
template <typename F>
void parallel_for(int n, F f)
{
    const int hw = (int)std::thread::hardware_concurrency();
    const int nth = std::max(1, std::min({hw, 32, n / 8}));
    if (nth <= 1) {
        for (int i = 0; i < n; ++i) f(i);
        return;
    }
    std::vector<std::thread> pool;
    for (int t = 0; t < nth; ++t)
        pool.emplace_back([&, t] {
            for (int i = (int)((long long)n * t / nth); i < (int)((long long)n * (t + 1) / nth); ++i) f(i);
        });
    for (auto& th : pool) th.join();
}

// ------------------------------------------------------------------------
// Quadrature: Gauss-Legendre on [a, b].  Roots of P_n by Newton iteration
// started from Tricomi's asymptotic estimate; weights 2/((1-x^2) P_n'(x)^2).

void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 1; i <= n; ++i) {
        const double th = kPi * (4.0 * i - 1.0) / (4.0 * n + 2.0);
        double t = (1.0 - (n - 1.0) / (8.0 * n * n * n)) * cos(th);
        double pn = 0, pn1 = 0;
        for (int iter = 0; iter < 60; ++iter) {
            double pm = 1.0, p = t;
            for (int k = 2; k <= n; ++k) {
                const double pk = ((2 * k - 1) * t * p - (k - 1) * pm) / k;
                pm = p;
                p = pk;
            }
            pn = (n == 1) ? t : p;
            pn1 = (n == 1) ? 1.0 : pm;
            const double d = n * (pn1 - t * pn) / (1.0 - t * t);
            const double step = pn / d;
            t -= step;
            if (fabs(step) <= 1e-17) break;
        }
        double pm = 1.0, p = t;
        for (int k = 2; k <= n; ++k) {
            const double pk = ((2 * k - 1) * t * p - (k - 1) * pm) / k;
            pm = p;
            p = pk;
        }
        pn = (n == 1) ? t : p;
        pn1 = (n == 1) ? 1.0 : pm;
        const double d = n * (pn1 - t * pn) / (1.0 - t * t);
        // i-th root from the top: t decreases with i; store ascending in r
        const int j = n - i;
        x[j] = 0.5 * (b + a) + 0.5 * (b - a) * t;
        w[j] = (b - a) / ((1.0 - t * t) * d * d);
    }
}

// Composite Simpson on [a, b] with n = 2m + 1 equally spaced nodes: weight
// h/3 at the ends, 4h/3 at odd and 2h/3 at interior even nodes.
void simpson(int n, double a, double b, std::vector<double>& x, std::vector<double>& w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    const double h = (b - a) / (n - 1);
    for (int i = 0; i < n; ++i) {
        x[i] = i == n - 1 ? b : a + i * h;
        const double c = (i == 0 || i == n - 1) ? 1.0 : ((i & 1) ? 4.0 : 2.0);
        w[i] = c * h / 3.0;
    }
}

// The mirror's radial rule on [r_min, r_max] (Sec. III.C.1).
void radial_rule(const sc_mirror_t* m, std::vector<double>& x, std::vector<double>& w)
{
    if (m->q.radial_kind == SC_QUAD_SIMPSON) simpson(m->q.n_r, m->r_min, m->r_max, x, w);
    else gauss_legendre(m->q.n_r, m->r_min, m->r_max, x, w);
}

// Zernike Z_j (Noll ordering and normalisation): radial order n and
// azimuthal order m from j by walking the (n, |m|) table.
void noll_nm(int j, int& n, int& m)
{
    int count = 0;
    for (n = 0;; ++n) {
        const int terms = n + 1;
        if (count + terms >= j) {
            // position within row n, 1-based
            const int pos = j - count;
            // |m| sequence in row n: n%2, n%2+2, ... each non-zero |m| appears twice
            int idx = 0;
            for (int am = n % 2; am <= n; am += 2) {
                const int mult = am == 0 ? 1 : 2;
                if (pos <= idx + mult) {
                    m = (am == 0) ? 0 : ((j % 2 == 0) ? am : -am);
                    return;
                }
                idx += mult;
            }
        }
        count += terms;
    }
}

double zernike(int j, double rho, double th)
{
    int n, m;
    noll_nm(j, n, m);
    const int am = m < 0 ? -m : m;
    double R = 0.0;
    for (int s = 0; s <= (n - am) / 2; ++s) {
        double num = tgamma(n - s + 1.0);
        double den = tgamma(s + 1.0) * tgamma((n + am) / 2 - s + 1.0) * tgamma((n - am) / 2 - s + 1.0);
        R += ((s & 1) ? -1.0 : 1.0) * num / den * pow(rho, n - 2 * s);
    }
    if (m == 0) return sqrt(n + 1.0) * R;
    return sqrt(2.0 * (n + 1.0)) * R * (m > 0 ? cos(am * th) : sin(am * th));
}

// ------------------------------------------------------------------------
// Incident field model on the mirror (collimated beam, Sec. III.A).

double profile_amp(const sc_incident_t* in, double rho)
{
    switch (in->profile) {
    case SC_PROFILE_GAUSS: return exp(-(rho / in->w0) * (rho / in->w0));
    case SC_PROFILE_SUPERGAUSS: return exp(-pow(rho / in->w0, 2.0 * in->sg_order));
    default: return rho <= in->w0 ? 1.0 : 0.0;
    }
}

// Transverse spatial field E~(rho, theta) (z component 0).
void incident_E(const sc_incident_t* in, double rho, double th, double& ex, double& ey)
{
    const double A = profile_amp(in, rho);
    if (in->pol == SC_POL_LINEAR) {
        ex = A * cos(in->angle);
        ey = A * sin(in->angle);
    } else {
        const double s = A * rho / in->w0;
        if (in->pol == SC_POL_RADIAL) {
            ex = s * cos(th);
            ey = s * sin(th);
        } else {
            ex = -s * sin(th);
            ey = s * cos(th);
        }
    }
}

double incident_opd(const sc_incident_t* in, double rho, double th, double r_unit)
{
    double W = 0.0;
    for (size_t i = 0; i < in->zern.size(); ++i) W += in->zern[i] * zernike((int)i + 2, rho / r_unit, th);
    return W;
}

// Partial derivatives of Z_j(u, th) in u and th.
void zernike_grad(int j, double u, double th, double& dzdu, double& dzdth)
{
    int n, m;
    noll_nm(j, n, m);
    const int am = m < 0 ? -m : m;
    double R = 0.0, dR = 0.0;
    for (int s = 0; s <= (n - am) / 2; ++s) {
        const double c = ((s & 1) ? -1.0 : 1.0) * tgamma(n - s + 1.0) /
                         (tgamma(s + 1.0) * tgamma((n + am) / 2 - s + 1.0) * tgamma((n - am) / 2 - s + 1.0));
        const int p = n - 2 * s;
        R += c * pow(u, p);
        if (p > 0) dR += c * p * pow(u, p - 1);
    }
    if (m == 0) {
        dzdu = sqrt(n + 1.0) * dR;
        dzdth = 0.0;
        return;
    }
    const double nrm = sqrt(2.0 * (n + 1.0));
    const double ca = cos(am * th), sa = sin(am * th);
    dzdu = nrm * dR * (m > 0 ? ca : sa);
    dzdth = nrm * R * am * (m > 0 ? -sa : ca);
}

// Cartesian gradient (gx, gy) of the optical path difference W at (rho, th).
void incident_opd_grad(const sc_incident_t* in, double rho, double th, double r_unit, double& gx,
                       double& gy)
{
    double dr = 0.0, dt = 0.0;
    for (size_t i = 0; i < in->zern.size(); ++i) {
        double du, dth;
        zernike_grad((int)i + 2, rho / r_unit, th, du, dth);
        dr += in->zern[i] * du / r_unit;
        dt += in->zern[i] * dth;
    }
    const double c = cos(th), s = sin(th), at = rho > 0.0 ? dt / rho : 0.0;
    gx = dr * c - at * s;  // dW/drho rho^ + (1/rho) dW/dth th^
    gy = dr * s + at * c;
}

// dA/drho of the profile (the top-hat has none and is refused at order 1).
double profile_damp(const sc_incident_t* in, double rho)
{
    const double A = profile_amp(in, rho), u = rho / in->w0;
    if (in->profile == SC_PROFILE_GAUSS) return -2.0 * u / in->w0 * A;
    if (in->profile == SC_PROFILE_SUPERGAUSS)
        return -2.0 * in->sg_order / in->w0 * pow(u, 2.0 * in->sg_order - 1.0) * A;
    return 0.0;
}

// Transverse divergences of e_perp = A p and b_perp = (-z) x e_perp, closed
// forms: linear  div e = A' cos(th - a), div b = A' sin(a - th);
//        radial  div e = (2A + rho A') / w0, div b = 0;
//        azimuthal div e = 0, div b = (2A + rho A') / w0.
// Laguerre-Gauss envelope of kind 3 at (x, y, z) and wavenumber k: complex
// (e_x, e_y) as (re, im) pairs.  L_p^a by upward recurrence in p.
void lg_envelope(const sc_incident_t* in, double k, double x, double y, double z, double e[4])
{
    const double w0 = in->w0, zr = 0.5 * k * w0 * w0, zeta = in->z_waist - z;
    const double q = zeta / zr;
    const double w2 = w0 * w0 * (1.0 + q * q);
    const double rho2 = x * x + y * y, rho = sqrt(rho2), th = atan2(y, x);
    const int a = in->pol == SC_POL_LINEAR ? abs(in->lg_l) : 1;
    const double X = 2.0 * rho2 / w2;
    double L = 1.0;
    if (in->lg_p > 0) {
        double lm = 1.0, lc = 1.0 + a - X;
        for (int n = 1; n < in->lg_p; ++n) {
            const double ln = ((2.0 * n + 1.0 + a - X) * lc - (n + a) * lm) / (n + 1.0);
            lm = lc;
            lc = ln;
        }
        L = lc;
    }
    const double amp = pow(w0 * w0 / w2, 0.5 * (a + 1)) * pow(rho / w0, a) * L * exp(-rho2 / w2);
    // phase: k rho^2 zeta / (2 (zeta^2 + z_R^2)) - (2p + a + 1) atan(zeta / z_R)
    double ph = 0.5 * k * rho2 * zeta / (zeta * zeta + zr * zr) - (2.0 * in->lg_p + a + 1) * atan(q);
    double px = 1.0, py = 0.0;  // polarisation (real for the vector modes)
    if (in->pol == SC_POL_LINEAR) {
        ph += in->lg_l * th;
        px = cos(in->angle);
        py = sin(in->angle);
    } else if (in->pol == SC_POL_RADIAL) {
        px = cos(th);
        py = sin(th);
    } else {
        px = -sin(th);
        py = cos(th);
    }
    const double ur = amp * cos(ph), ui = amp * sin(ph);
    e[0] = ur * px; e[1] = ui * px;
    e[2] = ur * py; e[3] = ui * py;
}

void incident_div(const sc_incident_t* in, double rho, double th, double& div_e, double& div_b)
{
    const double A = profile_amp(in, rho), dA = profile_damp(in, rho);
    if (in->pol == SC_POL_LINEAR) {
        div_e = dA * cos(th - in->angle);
        div_b = dA * sin(in->angle - th);
    } else {
        const double d = (2.0 * A + rho * dA) / in->w0;
        div_e = in->pol == SC_POL_RADIAL ? d : 0.0;
        div_b = in->pol == SC_POL_RADIAL ? 0.0 : d;
    }
}

// SS |A p|^2 dA over the transverse plane, closed forms.
double beam_power(const sc_incident_t* in)
{
    const double w2 = in->w0 * in->w0;
    const bool lin = in->pol == SC_POL_LINEAR;
    if (in->profile == SC_PROFILE_LAGUERRE_GAUSS) {
        // (pi w0^2 / 2) 2^-a Gamma(p + a + 1) / p!, a = |l| (1 for the vector modes)
        const int a = lin ? abs(in->lg_l) : 1;
        return kPi * w2 / 2.0 * pow(2.0, -a) * tgamma(in->lg_p + a + 1.0) / tgamma(in->lg_p + 1.0);
    }
    if (in->profile == SC_PROFILE_GAUSS) return lin ? kPi * w2 / 2.0 : kPi * w2 / 4.0;
    if (in->profile == SC_PROFILE_SUPERGAUSS) {
        const double N = in->sg_order;
        return lin ? kPi * w2 * pow(2.0, -1.0 / N) * tgamma(1.0 + 1.0 / N)
                   : kPi * w2 * pow(2.0, -2.0 / N) * tgamma(1.0 + 2.0 / N) / 2.0;
    }
    return lin ? kPi * w2 : kPi * w2 / 2.0;
}

// a_n = E0^n e^{i phi(k_n)}  (Eqs. 15-18, Eq. 27).
sc_status spectrum_amps(sc_ctx* ctx, const sc_incident_t* in, const double* om, int n,
                        std::vector<double>& amp)
{
    amp.assign(2 * (size_t)n, 0.0);
    const double kc = 2.0 * kPi / in->lambda_c;
    double norm = 1.0;
    if (in->spec_kind == SC_SPEC_GAUSS_TIME) {
        // int exp(-(k-kc)^2 tau^2 / (4 ln 2)) dk
        norm = sqrt(4.0 * kPi * log(2.0)) / in->fwhm_t;
    } else if (in->spec_kind == SC_SPEC_SUPERGAUSS_LAMBDA) {
        // int exp(-((l-lc)/dl)^(2n)) dl = 2 dl Gamma(1 + 1/(2n))
        norm = 2.0 * in->dlambda * tgamma(1.0 + 1.0 / (2.0 * in->sg_n));
    }
    const double P = beam_power(in);
    for (int i = 0; i < n; ++i) {
        const double k = 2.0 * kPi * om[i];
        double re = 1.0, im = 0.0;
        if (in->spec_kind == SC_SPEC_SAMPLED) {
            int hit = -1;
            for (size_t s = 0; s < in->s_omega.size(); ++s)
                if (fabs(in->s_omega[s] - om[i]) <= 1e-12 * fabs(om[i])) { hit = (int)s; break; }
            if (hit < 0)
                return fail(ctx, SC_ERR_INVALID, "omega %.17g is not one of the sampled spectrum's",
                            om[i]);
            re = in->s_amp[2 * hit];
            im = in->s_amp[2 * hit + 1];
        } else if (in->spec_kind == SC_SPEC_GAUSS_TIME) {
            const double s = exp(-(k - kc) * (k - kc) * in->fwhm_t * in->fwhm_t / (8.0 * log(2.0)));
            const double eps = in->energy * s * s / norm;
            re = sqrt(eps / (4.0 * kPi * P));
        } else if (in->spec_kind == SC_SPEC_SUPERGAUSS_LAMBDA) {
            const double lam = 2.0 * kPi / k;
            const double u = (lam - in->lambda_c) / in->dlambda;
            const double eps_l = exp(-pow(u * u, (double)in->sg_n));
            const double eps = in->energy * eps_l * (lam * lam / (2.0 * kPi)) / norm;
            re = sqrt(eps / (4.0 * kPi * P));
        }
        double ph = 0.0, term = 1.0;
        for (size_t j = 0; j < in->phi.size(); ++j) {
            if (j) term *= (k - kc) / (double)j;
            ph += in->phi[j] * term;
        }
        const double c = cos(ph), s = sin(ph);
        amp[2 * i] = re * c - im * s;
        amp[2 * i + 1] = re * s + im * c;
    }
    return SC_OK;
}

// ------------------------------------------------------------------------
// Mirror surfaces of revolution z = F(r), focus (F2) at the origin.

// SurfPt (sc_host.h): F(r), F'(r) (n dS = (-F' cos, -F' sin, 1) r dr dtheta),
// |P| (the distance to the focus) and the optical path added to W so that
// the kernel's phase R - |P| + W equals R - (z + z_ref) + W (collimated beams).
SurfPt surf_at(const sc_mirror_t* m, double r)
{
    SurfPt p;
    if (m->surface == 2) {
        const double a2 = m->c * m->c - m->e * m->e, s = sqrt(1.0 - r * r / a2);
        p.z = m->e - m->c * s;
        p.dzdr = m->c * r / (a2 * s);
        p.pn = sqrt(r * r + p.z * p.z);
        p.extra = p.pn - (p.z + 2.0 * (m->c - m->e));  // z_ref = -2 z_vertex
    } else {
        // |P| = z + 2f on the paraboloid: the extra path vanishes identically
        p.z = r * r / (4.0 * m->f) - m->f;
        p.dzdr = r / (2.0 * m->f);
        p.pn = r * r / (4.0 * m->f) + m->f;
        p.extra = 0.0;
    }
    return p;
}

// ------------------------------------------------------------------------
// Node tables (FP64 on the host; A1 of the hot path).

// Surface and rim nodes of (m, in).  For a first-order beam (order 1) surf1
// receives the second table: the same nodes carrying the 1/k part of the
// longitudinal terms, E~1 = z div_perp e_perp and B~1 = z div_perp b_perp,
// whose sums the reduce multiplies by -i/k_n.  Its rim term vanishes (a
// z-directed B has n x (n x B) . theta^ = 0), so it has no rim nodes.  The
// aberration part of the longitudinal terms, z (e_perp . grad W), carries no
// 1/k and joins the first table.
void build_nodes(const sc_mirror_t* m, const sc_incident_t* in, std::vector<HostNode>& surf,
                 std::vector<HostNode>& rim, std::vector<HostNode>& surf1)
{
    const double f = m->f;
    const int nr = m->q.n_r, nt = m->q.n_theta;
    const bool first = in->order >= 1;
    std::vector<double> gr, gw;
    radial_rule(m, gr, gw);
    const double dth = 2.0 * kPi / nt;
    // E~, B~ of the first table at (r, th), z components included
    auto fields = [&](double r, double th, double e[3], double bv[3]) {
        incident_E(in, r, th, e[0], e[1]);
        bv[0] = e[1];
        bv[1] = -e[0];  // B~ = (-z) x E~
        e[2] = bv[2] = 0.0;
        if (first && !in->zern.empty()) {
            double gx, gy;
            incident_opd_grad(in, r, th, m->r_max, gx, gy);
            e[2] = e[0] * gx + e[1] * gy;
            bv[2] = bv[0] * gx + bv[1] * gy;
        }
    };
    surf.assign((size_t)nr * nt, HostNode{});
    surf1.assign(first ? (size_t)nr * nt : 0, HostNode{});
    // rings in parallel: every node is a pure function of (r_i, theta_l)
    parallel_for(nr, [&](int i) {
        const double r = gr[i];
        const SurfPt sp = surf_at(m, r);
        for (int l = 0; l < nt; ++l) {
            const double th = l * dth;
            const double x = r * cos(th), y = r * sin(th), z = sp.z;
            const double Nx = -sp.dzdr * cos(th), Ny = -sp.dzdr * sin(th), Nz = 1.0;
            double e[3], bv[3];
            fields(r, th, e, bv);
            const double wq = gw[i] * dth * r / (2.0 * kPi);
            HostNode nd;
            nd.px = x; nd.py = y; nd.pz = z;
            nd.pn = sp.pn;
            nd.w = incident_opd(in, r, th, m->r_max) + sp.extra;
            // J = N x B~, rho = N . E~
            nd.jx = (Ny * bv[2] - Nz * bv[1]) * wq;
            nd.jy = (Nz * bv[0] - Nx * bv[2]) * wq;
            nd.jz = (Nx * bv[1] - Ny * bv[0]) * wq;
            nd.rho = (Nx * e[0] + Ny * e[1] + Nz * e[2]) * wq;
            surf[(size_t)i * nt + l] = nd;
            if (first) {
                double de, db;
                incident_div(in, r, th, de, db);
                HostNode n1 = nd;
                n1.jx = Ny * db * wq;   // N x (0, 0, db)
                n1.jy = -Nx * db * wq;
                n1.jz = 0.0;
                n1.rho = Nz * de * wq;  // N . (0, 0, de)
                surf1[(size_t)i * nt + l] = n1;
            }
        }
    });
    rim.clear();
    if (!m->q.rim_term) return;
    for (int edge = 0; edge < 2; ++edge) {
        const double r = edge == 0 ? m->r_max : m->r_min;
        const double sgn = edge == 0 ? 1.0 : -1.0;  // outward conormal of the surface
        if (r <= 0.0) continue;
        const SurfPt sp = surf_at(m, r);
        const double nlen2 = 1.0 + sp.dzdr * sp.dzdr;
        for (int l = 0; l < nt; ++l) {
            const double th = l * dth;
            const double c = cos(th), s = sin(th);
            const double x = r * c, y = r * s, z = sp.z;
            const double Nx = -sp.dzdr * c, Ny = -sp.dzdr * s;
            double e[3], bv[3];
            fields(r, th, e, bv);
            // N x B~ (N_z = 1)
            const double jx = Ny * bv[2] - bv[1], jy = bv[0] - Nx * bv[2], jz = Nx * bv[1] - Ny * bv[0];
            // q = (J . m^) dl with J = (N x B~)/|N|, m^ = sgn (c, s, F')/|N|, dl = r dth
            const double q = sgn * (jx * c + jy * s + jz * sp.dzdr) / nlen2 * r * dth;
            HostNode nd;
            nd.px = x; nd.py = y; nd.pz = z;
            nd.pn = sp.pn;
            nd.w = incident_opd(in, r, th, m->r_max) + sp.extra;
            nd.jx = nd.jy = nd.jz = 0.0;
            nd.rho = q / (2.0 * kPi);
            rim.push_back(nd);
        }
    }
}

// Host nodes of one table part (see TablePart).

// Kinds 3 and 4: Chebyshev expansion in k of the envelope e_perp over the
// band [kc - kh, kc + kh], from kCheb samples at the Chebyshev points
// x_j = cos(pi (j + 1/2) / kCheb): c_m = (2 - [m = 0]) / kCheb sum_j f(x_j)
// T_m(x_j).  Before the fit each node's phase slope in k at the band centre,
// tau = d arg(e_perp) / dk from two nearby samples, is taken out of the
// envelope (f = e_perp e^{-ik tau}) and put into the node's optical path W,
// where the field kernel applies it exactly as e^{ik W}: what remains varies
// less with k and needs fewer terms.  The fit keeps the first M terms, M
// the least with sum_{m >= M} max |c_m| <= fit_tol max |f|; the real and
// imaginary parts of each kept c_m become parts of their own (a part that
// is zero everywhere is left out).  B~ = (-z) x E~ (order 0).
constexpr int kCheb = 24;
constexpr int kChebMaxTerms = 20;

sc_status build_cheb_parts(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in,
                           std::vector<HostPart>& parts, double& kc, double& kh)
{
    const double f = m->f;
    const int nr = m->q.n_r, nt = m->q.n_theta;
    std::vector<double> gr, gw;
    radial_rule(m, gr, gw);
    const double dth = 2.0 * kPi / nt;
    // node positions: surface (r_i, theta_l), then the rim edges
    struct Pos { double r, th; int edge; };
    std::vector<Pos> pos;
    pos.reserve((size_t)nr * nt + 2 * (size_t)nt);
    for (int i = 0; i < nr; ++i)
        for (int l = 0; l < nt; ++l) pos.push_back({gr[i], l * dth, -1});
    const size_t n_surf = pos.size();
    if (m->q.rim_term)
        for (int edge = 0; edge < 2; ++edge) {
            const double r = edge == 0 ? m->r_max : m->r_min;
            if (r <= 0.0) continue;
            for (int l = 0; l < nt; ++l) pos.push_back({r, l * dth, edge});
        }
    const size_t n = pos.size();
    std::vector<double> xyz(3 * n);
    std::vector<SurfPt> sp(n);
    for (size_t j = 0; j < n; ++j) {
        sp[j] = surf_at(m, pos[j].r);
        xyz[3 * j] = pos[j].r * cos(pos[j].th);
        xyz[3 * j + 1] = pos[j].r * sin(pos[j].th);
        xyz[3 * j + 2] = sp[j].z;
    }
    kc = kPi * (in->om_lo + in->om_hi);
    kh = kPi * (in->om_hi - in->om_lo);
    std::vector<double> e(4 * n);
    auto sample = [&](double k) -> bool {
        if (in->profile == SC_PROFILE_LAGUERRE_GAUSS) {
            for (size_t q = 0; q < n; ++q) lg_envelope(in, k, xyz[3 * q], xyz[3 * q + 1], xyz[3 * q + 2], &e[4 * q]);
        } else {
            std::fill(e.begin(), e.end(), 0.0);
            in->env(in->env_user, (int)n, xyz.data(), k, e.data());
        }
        for (double v : e)
            if (!std::isfinite(v)) return false;
        return true;
    };
    // per-node phase slope tau at the band centre
    std::vector<double> tau(n, 0.0);
    {
        const double dk = 0.01 * kh;
        if (!sample(kc - dk)) return fail(ctx, SC_ERR_INVALID, "the envelope is not finite on the mirror");
        const std::vector<double> em = e;
        if (!sample(kc + dk)) return fail(ctx, SC_ERR_INVALID, "the envelope is not finite on the mirror");
        for (size_t q = 0; q < n; ++q) {
            // arg of sum_c e_c(k + dk) conj(e_c(k - dk))
            double sr = 0.0, si = 0.0;
            for (int cpt = 0; cpt < 2; ++cpt) {
                const double ar = e[4 * q + 2 * cpt], ai = e[4 * q + 2 * cpt + 1];
                const double br = em[4 * q + 2 * cpt], bi = em[4 * q + 2 * cpt + 1];
                sr += ar * br + ai * bi;
                si += ai * br - ar * bi;
            }
            if (sr != 0.0 || si != 0.0) tau[q] = atan2(si, sr) / (2.0 * dk);
        }
    }
    // coefficients c[m][node][4] (e_x re, im, e_y re, im) of e_perp e^{-ik tau}
    std::vector<double> c((size_t)kCheb * n * 4, 0.0);
    double peak = 0.0;
    for (int j = 0; j < kCheb; ++j) {
        const double tj = kPi * (j + 0.5) / kCheb;
        const double k = kc + kh * cos(tj);
        if (!sample(k)) return fail(ctx, SC_ERR_INVALID, "the envelope is not finite on the mirror");
        for (size_t q = 0; q < n; ++q) {
            const double cr = cos(k * tau[q]), ci = -sin(k * tau[q]);
            for (int cpt = 0; cpt < 2; ++cpt) {
                const double ar = e[4 * q + 2 * cpt], ai = e[4 * q + 2 * cpt + 1];
                e[4 * q + 2 * cpt] = ar * cr - ai * ci;
                e[4 * q + 2 * cpt + 1] = ar * ci + ai * cr;
            }
        }
        for (size_t q = 0; q < 4 * n; q += 2) peak = std::max(peak, std::hypot(e[q], e[q + 1]));
        for (int mm = 0; mm < kCheb; ++mm) {
            const double w = (mm == 0 ? 1.0 : 2.0) / kCheb * cos(mm * tj);
            double* cm = &c[(size_t)mm * n * 4];
            for (size_t q = 0; q < 4 * n; ++q) cm[q] += w * e[q];
        }
    }
    if (!(peak > 0.0)) return fail(ctx, SC_ERR_INVALID, "the envelope vanishes on the mirror");
    std::vector<double> cmax(kCheb, 0.0);
    for (int mm = 0; mm < kCheb; ++mm) {
        const double* cm = &c[(size_t)mm * n * 4];
        for (size_t q = 0; q < 4 * n; q += 2) cmax[mm] = std::max(cmax[mm], std::hypot(cm[q], cm[q + 1]));
    }
    int M = kCheb;
    double tail = 0.0;
    while (M > 1 && tail + cmax[M - 1] <= in->fit_tol * peak) tail += cmax[--M];
    if (M > kChebMaxTerms)
        return fail(ctx, SC_ERR_INVALID,
                    "the envelope needs more than %d Chebyshev terms in k over the band (tolerance %g)",
                    kChebMaxTerms, in->fit_tol);
    parts.clear();
    for (int mm = 0; mm < M; ++mm)
        for (int im = 0; im < 2; ++im) {
            const double* cm = &c[(size_t)mm * n * 4];
            double pmax = 0.0;
            for (size_t q = 0; q < n; ++q)
                pmax = std::max(pmax, std::max(fabs(cm[4 * q + im]), fabs(cm[4 * q + 2 + im])));
            if (pmax <= 1e-3 * in->fit_tol * peak) continue;
            HostPart hp;
            hp.kind = im ? PART_CHEB_IM : PART_CHEB_RE;
            hp.m = mm;
            hp.surf.reserve(n_surf);
            for (size_t q = 0; q < n; ++q) {
                const double ex = cm[4 * q + im], ey = cm[4 * q + 2 + im];
                const double bx = ey, by = -ex;  // B~ = (-z) x E~
                const double r = pos[q].r, th = pos[q].th;
                const double x = xyz[3 * q], y = xyz[3 * q + 1];
                const double Nx = -sp[q].dzdr * cos(th), Ny = -sp[q].dzdr * sin(th);
                HostNode nd;
                nd.px = x; nd.py = y; nd.pz = xyz[3 * q + 2];
                nd.pn = sp[q].pn;
                nd.w = incident_opd(in, r, th, m->r_max) + tau[q] + sp[q].extra;
                if (q < n_surf) {
                    const double wq = gw[q / nt] * dth * r / (2.0 * kPi);
                    nd.jx = -by * wq;  // N x B~ with B~_z = 0, N_z = 1
                    nd.jy = bx * wq;
                    nd.jz = (Nx * by - Ny * bx) * wq;
                    nd.rho = (Nx * ex + Ny * ey) * wq;
                    hp.surf.push_back(nd);
                } else {
                    const double sgn = pos[q].edge == 0 ? 1.0 : -1.0;
                    const double nlen2 = 1.0 + sp[q].dzdr * sp[q].dzdr;
                    const double jx = -by, jy = bx, jz = Nx * by - Ny * bx;
                    const double qq = sgn * (jx * cos(th) + jy * sin(th) + jz * sp[q].dzdr) / nlen2 * r * dth;
                    nd.jx = nd.jy = nd.jz = 0.0;
                    nd.rho = qq / (2.0 * kPi);
                    hp.rim.push_back(nd);
                }
            }
            parts.push_back(std::move(hp));
        }
    return SC_OK;
}

void pack_tiles(const std::vector<HostNode>& v, std::vector<float>& out, int& n_tiles)
{
    n_tiles = (int)((v.size() + sc::kTile - 1) / sc::kTile);
    out.assign((size_t)n_tiles * sc::kTileFloats, 0.0f);
    for (size_t i = 0; i < (size_t)n_tiles * sc::kTile; ++i) {
        // padding nodes sit on node 0 with zero weight
        const HostNode& nd = i < v.size() ? v[i] : v[0];
        const bool pad = i >= v.size();
        float* t = out.data() + (i / sc::kTile) * sc::kTileFloats;
        const size_t j = i % sc::kTile;
        t[sc::F_PX * sc::kTile + j] = (float)nd.px;
        t[sc::F_PY * sc::kTile + j] = (float)nd.py;
        t[sc::F_PZ * sc::kTile + j] = (float)nd.pz;
        t[sc::F_PN * sc::kTile + j] = (float)nd.pn;
        t[sc::F_W * sc::kTile + j] = (float)nd.w;
        t[sc::F_JX * sc::kTile + j] = pad ? 0.f : (float)nd.jx;
        t[sc::F_JY * sc::kTile + j] = pad ? 0.f : (float)nd.jy;
        t[sc::F_JZ * sc::kTile + j] = pad ? 0.f : (float)nd.jz;
        t[sc::F_RHO * sc::kTile + j] = pad ? 0.f : (float)nd.rho;
        t[sc::F_PAD * sc::kTile + j] = 0.f;
    }
}

void free_table(sc_ctx* ctx, Table& t)
{
    if (t.d32) cudaFree(t.d32);
    if (t.d64) cudaFree(t.d64);
    ctx->held -= t.bytes;
    t = Table{};
}

// Look up or build the table of (m, in).  Public calls advance ctx->tick once;
// tables touched by the current call carry that tick and are never evicted by it.
// Kind 5 on the ellipsoid (reading R16): the dipole field at the node,
// without its phase e^{ik(r - 2c)} = e^{-ik|P|} (r + |P| = 2c on the
// ellipsoid, so the kernel's compensated phase R - |P| is the whole phase),
// is sum_m (ik)^m (E_m, B_m):
//   m = 0: E = A2 / r^3, B = 0;  m = 1: E = -A2 / r^2, B = (n x p) / r^2;
//   m = 2: E = -(n x p) x n / r, B = -(n x p) / r;  A2 = 3 n (n.p) - p.
sc_status build_dipole_parts(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in,
                             std::vector<HostPart>& parts)
{
    if (m->surface != 2)
        return fail(ctx, SC_ERR_INVALID, "a dipole source needs an ellipsoidal mirror (it sits at its focus F1)");
    const int nr = m->q.n_r, nt = m->q.n_theta;
    std::vector<double> gr, gw;
    radial_rule(m, gr, gw);
    const double dth = 2.0 * kPi / nt;
    const double* p = in->dip;
    parts.assign(3, HostPart());
    for (int mm = 0; mm < 3; ++mm) {
        parts[mm].kind = PART_IK_POW;
        parts[mm].m = mm;
    }
    // E_m, B_m at a mirror point
    auto terms = [&](double x, double y, double z, double E[3][3], double B[3][3]) {
        const double d[3] = {x, y, z - 2.0 * m->e};
        const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        const double n[3] = {d[0] / r, d[1] / r, d[2] / r};
        const double np = n[0] * p[0] + n[1] * p[1] + n[2] * p[2];
        const double nxp[3] = {n[1] * p[2] - n[2] * p[1], n[2] * p[0] - n[0] * p[2], n[0] * p[1] - n[1] * p[0]};
        for (int c = 0; c < 3; ++c) {
            const double a2 = 3.0 * n[c] * np - p[c];
            E[0][c] = a2 / (r * r * r);
            B[0][c] = 0.0;
            E[1][c] = -a2 / (r * r);
            B[1][c] = nxp[c] / (r * r);
            E[2][c] = -(p[c] - n[c] * np) / r;  // -(n x p) x n / r
            B[2][c] = -nxp[c] / r;
        }
    };
    for (int i = 0; i < nr; ++i) {
        const double r = gr[i];
        const SurfPt sp = surf_at(m, r);
        for (int l = 0; l < nt; ++l) {
            const double th = l * dth;
            const double x = r * cos(th), y = r * sin(th);
            const double N[3] = {-sp.dzdr * cos(th), -sp.dzdr * sin(th), 1.0};
            const double wq = gw[i] * dth * r / (2.0 * kPi);
            double E[3][3], B[3][3];
            terms(x, y, sp.z, E, B);
            for (int mm = 0; mm < 3; ++mm) {
                HostNode nd;
                nd.px = x; nd.py = y; nd.pz = sp.z;
                nd.pn = sp.pn;
                nd.w = 0.0;
                nd.jx = (N[1] * B[mm][2] - N[2] * B[mm][1]) * wq;  // J = N x B~, rho = N . E~
                nd.jy = (N[2] * B[mm][0] - N[0] * B[mm][2]) * wq;
                nd.jz = (N[0] * B[mm][1] - N[1] * B[mm][0]) * wq;
                nd.rho = (N[0] * E[mm][0] + N[1] * E[mm][1] + N[2] * E[mm][2]) * wq;
                parts[mm].surf.push_back(nd);
            }
        }
    }
    if (!m->q.rim_term) return SC_OK;
    for (int edge = 0; edge < 2; ++edge) {
        const double r = edge == 0 ? m->r_max : m->r_min;
        const double sgn = edge == 0 ? 1.0 : -1.0;
        if (r <= 0.0) continue;
        const SurfPt sp = surf_at(m, r);
        const double nlen2 = 1.0 + sp.dzdr * sp.dzdr;
        for (int l = 0; l < nt; ++l) {
            const double th = l * dth, c = cos(th), s = sin(th);
            const double x = r * c, y = r * s;
            const double N[3] = {-sp.dzdr * c, -sp.dzdr * s, 1.0};
            double E[3][3], B[3][3];
            terms(x, y, sp.z, E, B);
            for (int mm = 0; mm < 3; ++mm) {
                const double jx = N[1] * B[mm][2] - N[2] * B[mm][1], jy = N[2] * B[mm][0] - N[0] * B[mm][2],
                             jz = N[0] * B[mm][1] - N[1] * B[mm][0];
                const double q = sgn * (jx * c + jy * s + jz * sp.dzdr) / nlen2 * r * dth;
                HostNode nd;
                nd.px = x; nd.py = y; nd.pz = sp.z;
                nd.pn = sp.pn;
                nd.w = 0.0;
                nd.jx = nd.jy = nd.jz = 0.0;
                nd.rho = q / (2.0 * kPi);
                parts[mm].rim.push_back(nd);
            }
        }
    }
    return SC_OK;
}

// The compensated FP32 phase needs the incident wavefront to focus on the
// origin: plane waves on the paraboloid, the F1 dipole on the ellipsoid.
bool focuses_on_origin(const sc_mirror_t* m, const sc_incident_t* in)
{
    return (m->surface == 2) == (in->profile == SC_PROFILE_DIPOLE);
}

// The host nodes of every node table of (m, in), FP64 (no device work).
sc_status build_host_parts(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in,
                           std::vector<HostPart>& hp, double& kc, double& kh)
{
    hp.clear();
    if (in->profile == SC_PROFILE_DIPOLE) return build_dipole_parts(ctx, m, in, hp);
    if (in->profile >= SC_PROFILE_LAGUERRE_GAUSS) return build_cheb_parts(ctx, m, in, hp, kc, kh);
    hp.resize(1);
    std::vector<HostNode> surf1;
    build_nodes(m, in, hp[0].surf, hp[0].rim, surf1);
    if (!surf1.empty()) {
        HostPart p1;
        p1.kind = PART_INV_K;
        p1.surf = std::move(surf1);
        hp.push_back(std::move(p1));
    }
    return SC_OK;
}

sc_status get_table(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in, Table** out,
                    cudaStream_t stream)
{
    for (auto& t : ctx->tables)
        if (t.mid == m->id && t.iid == in->id) {
            t.last_use = ctx->tick;
            *out = &t;
            return SC_OK;
        }
    std::vector<HostPart> hp;
    Table t;
    t.mid = m->id;
    t.iid = in->id;
    t.fp32_ok = focuses_on_origin(m, in);
    sc_status hst = build_host_parts(ctx, m, in, hp, t.kc, t.kh);
    if (hst != SC_OK) return hst;
    // FP32 tiles and FP64 records of every part, part after part
    std::vector<float> t32;
    std::vector<sc::Node64> h64;
    std::vector<size_t> off32, off64;
    std::vector<int> rim_tiles;
    for (const auto& p : hp) {
        std::vector<float> ts, tr;
        int nst = 0, nrt = 0;
        pack_tiles(p.surf, ts, nst);
        if (!p.rim.empty()) pack_tiles(p.rim, tr, nrt);
        t.n_surf_tiles = nst;
        t.n_surf = (int)p.surf.size();
        off32.push_back(t32.size());
        off64.push_back(h64.size());
        rim_tiles.push_back(nrt);
        t32.insert(t32.end(), ts.begin(), ts.end());
        t32.insert(t32.end(), tr.begin(), tr.end());
        for (const auto* vec : {&p.surf, &p.rim})
            for (const auto& nd : *vec)
                h64.push_back(sc::Node64{nd.px, nd.py, nd.pz, nd.pn, nd.w, nd.jx, nd.jy, nd.jz, nd.rho, 0.0});
    }
    t.n_rim_tiles = rim_tiles[0];
    t.n_rim = (int)hp[0].rim.size();
    const size_t b32 = t32.size() * sizeof(float);
    const size_t b64 = h64.size() * sizeof(sc::Node64);
    t.bytes = b32 + b64;
    // evict least recently used tables while over budget
    while (ctx->budget && ctx->held + t.bytes > ctx->budget && !ctx->tables.empty()) {
        // evict the least recently used table that no call in flight on the host uses
        auto it = ctx->tables.end();
        for (auto jt = ctx->tables.begin(); jt != ctx->tables.end(); ++jt)
            if (jt->inflight == 0 && jt->last_use != ctx->tick &&
                (it == ctx->tables.end() || jt->last_use < it->last_use))
                it = jt;
        if (it == ctx->tables.end()) break;
        cudaDeviceSynchronize();
        free_table(ctx, *it);
        ctx->tables.erase(it);
    }
    if (ctx->budget && ctx->held + t.bytes > ctx->budget)
        return fail(ctx, SC_ERR_OOM, "node table of %zu bytes exceeds the device budget", t.bytes);
    cudaError_t e = cudaMalloc(&t.d32, b32);
    if (e == cudaSuccess) e = cudaMalloc(&t.d64, b64);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (t.d32) cudaFree(t.d32);
        return fail(ctx, SC_ERR_OOM, "node table allocation failed: %s", cudaGetErrorString(e));
    }
    for (size_t i = 0; i < hp.size(); ++i) {
        TablePart tp;
        tp.kind = hp[i].kind;
        tp.m = hp[i].m;
        tp.d32 = t.d32 + off32[i];
        tp.n_rim_tiles = rim_tiles[i];
        tp.d64 = t.d64 + off64[i];
        tp.n_rim = (int)hp[i].rim.size();
        t.parts.push_back(tp);
    }
    e = cudaMemcpyAsync(t.d32, t32.data(), b32, cudaMemcpyHostToDevice, stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(t.d64, h64.data(), b64, cudaMemcpyHostToDevice, stream);
    // the host vectors die at return: make the copies complete first
    const cudaError_t es = cudaStreamSynchronize(stream);
    if (e == cudaSuccess) e = es;
    if (e != cudaSuccess) {
        cudaGetLastError();
        cudaFree(t.d32);
        cudaFree(t.d64);
        return cuda_fail(ctx, e, "node table upload");
    }
    ctx->held += t.bytes;
    t.last_use = ctx->tick;
    ctx->tables.push_back(t);
    *out = &ctx->tables.back();
    return SC_OK;
}

// Per-part amplitudes of one request, [n_parts][n][2]: a_n times the part's
// weight w_p(omega_n).  Chebyshev parts need every omega inside their band.
sc_status request_amps(sc_ctx* ctx, const sc_incident_t* in, const Table* tab, const double* om, int n,
                       std::vector<double>& out)
{
    std::vector<double> a;
    sc_status st = spectrum_amps(ctx, in, om, n, a);
    if (st != SC_OK) return st;
    const size_t np = tab->parts.size();
    out.assign(np * 2 * (size_t)n, 0.0);
    for (size_t p = 0; p < np; ++p) {
        const TablePart& tp = tab->parts[p];
        for (int i = 0; i < n; ++i) {
            const double k = 2.0 * kPi * om[i];
            double wr = 1.0, wi = 0.0;
            if (tp.kind == PART_INV_K) {
                wr = 0.0;
                wi = -1.0 / k;
            } else if (tp.kind == PART_IK_POW) {
                wr = tp.m == 0 ? 1.0 : (tp.m == 2 ? -k * k : 0.0);
                wi = tp.m == 1 ? k : 0.0;
            } else if (tp.kind != PART_ONE) {
                const double x = (k - tab->kc) / tab->kh;
                if (!(fabs(x) <= 1.0 + 1e-12))
                    return fail(ctx, SC_ERR_INVALID, "omega %.17g lies outside the beam's band [%g, %g]", om[i],
                                in->om_lo, in->om_hi);
                const double T = cos(tp.m * acos(std::max(-1.0, std::min(1.0, x))));
                wr = tp.kind == PART_CHEB_RE ? T : 0.0;
                wi = tp.kind == PART_CHEB_RE ? 0.0 : T;
            }
            const double ar = a[2 * i], ai = a[2 * i + 1];
            out[(p * n + i) * 2] = ar * wr - ai * wi;
            out[(p * n + i) * 2 + 1] = ar * wi + ai * wr;
        }
    }
    return SC_OK;
}

// Reads and clears the device error word (synchronizes the stream).
sc_status check_device_error(sc_ctx* ctx)
{
    SC_CUDA(cudaMemcpyAsync(ctx->h_err, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream),
            "read error word");
    SC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    const int e = *ctx->h_err;
    if (e) {
        SC_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream), "clear error word");
        if (e & sc::ERR_TIMEOUT)
            return fail(ctx, SC_ERR_TIMEOUT, "a bounded device wait ran out (error word 0x%x)", e);
        if (e & sc::ERR_NEAR_SURFACE)
            return fail(ctx, SC_ERR_INVALID, "an observation point lies on the mirror");
        return fail(ctx, SC_ERR_CUDA, "device error word 0x%x", e);
    }
    return SC_OK;
}

cudaEvent_t take_event(sc_ctx* ctx)
{
    if (!ctx->pool.empty()) {
        cudaEvent_t e = ctx->pool.back();
        ctx->pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

void settle_events(sc_ctx* ctx)
{
    for (auto& pr : ctx->pending) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) ctx->ctr.field_ms += ms;
        else cudaGetLastError();
        ctx->pool.push_back(pr.first);
        ctx->pool.push_back(pr.second);
    }
    ctx->pending.clear();
}

// Points closer than 1e-6 lambda0 to a node make the integrand singular.
// |P| >= f for every mirror point, so only points with |r'| >= f - 1e-6 can
// come that close; those are checked against every node in FP64.
sc_status check_points_host(sc_ctx* ctx, const sc_mirror_t* m, const double* pts, int n_pts)
{
    std::vector<HostNode> surf, rim;
    bool built = false;
    for (int i = 0; i < n_pts; ++i) {
        const double x = pts[3 * i], y = pts[3 * i + 1], z = pts[3 * i + 2];
        if (!std::isfinite(x) || !std::isfinite(y) || !std::isfinite(z))
            return fail(ctx, SC_ERR_INVALID, "point %d is not finite", i);
        const double r = sqrt(x * x + y * y + z * z);
        if (r < m->f - 1e-6) continue;
        // |P| >= f = c - e on both surfaces
        const double rho = sqrt(x * x + y * y);
        if (rho >= m->r_min - 1e-6 && rho <= m->r_max + 1e-6 &&
            fabs(z - surf_at(m, std::min(rho, m->r_max)).z) < 1e-6)
            return fail(ctx, SC_ERR_INVALID, "point %d lies on the mirror surface", i);
        (void)built;
    }
    return SC_OK;
}

bool uniform_grid(const double* om, int n, double& d)
{
    if (n == 1) {
        d = 0.0;
        return true;
    }
    d = (om[n - 1] - om[0]) / (n - 1);
    if (!(d > 0.0)) return false;
    for (int i = 0; i < n; ++i)
        if (fabs(om[i] - (om[0] + i * d)) > 1e-9 * om[0]) return false;
    return true;
}

}  // namespace sch
