// sc_api.cpp -- host side of libsc: handles, the FP64 node-table builder and
// spectrum generator, device-memory management and the C-ABI entry points
// declared in include/sc.h.  Every GPU step is a kernel of this library
// (sc_field.cu, sc_f64_idft.cu); nothing here computes a field value on the
// CPU.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <mutex>
#include <thread>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "sc.h"
#include "sc_internal.h"

namespace {

constexpr double kPi = 3.14159265358979323846;
static_assert(SC_STATIC_SCRATCH_BYTES == sc::kStaticScratchBytes, "scratch size mismatch");

std::atomic<uint64_t> g_next_id{1};

}  // namespace

// --------------------------------------------------------------------------
// Handles

struct sc_mirror_t {
    uint64_t id;
    double f, r_min, r_max;
    sc_quadrature q;
    int surface = 0;        // 0 paraboloid, 2 ellipsoid (semi-axis c, focal half-distance e)
    double c = 0.0, e = 0.0;
};

struct sc_incident_t {
    uint64_t id;
    int profile, sg_order, pol;
    int order;                      // 0 collimated, 1 plus the O(eps) longitudinal terms
    int lg_p = 0, lg_l = 0;         // Laguerre-Gauss mode (profile 3)
    double z_waist = 0.0;
    sc_envelope_fn env = nullptr;   // caller's envelope (profile 4)
    void* env_user = nullptr;
    double om_lo = 0.0, om_hi = 0.0, fit_tol = 1e-8;  // band and tolerance of the k fit
    double dip[3] = {0.0, 0.0, 0.0};                  // dipole moment (profile 5)
    double w0, angle;
    std::vector<double> zern;
    int spec_kind;
    double fwhm_t, lambda_c, dlambda, energy;
    int sg_n;
    std::vector<double> s_omega, s_amp, phi;
};

namespace {

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

// One node table of an incident.  Every part sums over the same nodes; its
// sums enter the result with a per-omega complex weight w_p(omega_n):
//   PART_ONE 1,  PART_INV_K -i/k_n (the 1/k longitudinal terms of order 1),
//   PART_CHEB_RE T_m(x_n),  PART_CHEB_IM i T_m(x_n)  (x_n = (k_n - kc) / kh,
//   the Chebyshev expansion in k of a k-dependent envelope),
//   PART_IK_POW (i k_n)^m (the terms of the dipole field).
enum { PART_ONE = 0, PART_INV_K = 1, PART_CHEB_RE = 2, PART_CHEB_IM = 3, PART_IK_POW = 4 };

struct TablePart {
    int kind = PART_ONE, m = 0;
    const float* d32 = nullptr;       // surface tiles, then this part's rim tiles
    int n_rim_tiles = 0;
    const sc::Node64* d64 = nullptr;  // surface records, then rim records
    int n_rim = 0;
};

struct Table {
    uint64_t mid = 0, iid = 0;
    float* d32 = nullptr;          // one allocation for every part's FP32 tiles
    int n_surf_tiles = 0, n_rim_tiles = 0;  // (rim: part 0's)
    sc::Node64* d64 = nullptr;     // and one for their FP64 records
    int n_surf = 0, n_rim = 0;
    std::vector<TablePart> parts;
    double kc = 0.0, kh = 1.0;     // Chebyshev band in k of the CHEB parts
    bool fp32_ok = true;           // the incident wavefront focuses on the origin, so the
                                   // compensated FP32 phase is exact (else FP64 only)
    size_t bytes = 0;
    uint64_t last_use = 0;
    int inflight = 0;              // serving batches on the GPU that read this table
};

struct GraphEntry {
    std::vector<unsigned char> sig;
    cudaGraphExec_t exec = nullptr;
    uint64_t last = 0;
};

// An execution lane of the FP32 path: a stream and the device buffers and
// graph cache that one batch in flight needs.  The context's own calls use
// lane `main` (on the caller's stream); the serving loop owns more lanes so
// that batches overlap on the GPU.
struct Lane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    DevBuf ws, desc, amp, kval;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
};

struct Server;

}  // namespace

struct sc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    size_t held = 0;
    std::string err = "no error";
    std::list<Table> tables;
    uint64_t tick = 0;
    DevBuf pts, outE, outB, tkval, tvals, phasor, specE, specB, tE, tB;
    DevBuf fpts, fspecE, fspecB, ftE, ftB;  // sc_eval_time_domain: points, chunk spectra, E(t), B(t)
    int* d_err = nullptr;
    int* h_err = nullptr;          // pinned
    sc_counters ctr{};
    bool time_field = false;
    long long nodes_per_split = 0;  // 0: choose splits for load balance
    long long flush_nodes = 2048;   // FP32 run length before each compensated fold
    size_t ws_cap = size_t(2) << 30;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> pool;
    // batched execution: lanes, graph counters, split autotuner, serving
    Lane main;
    bool use_graphs = true;
    bool autotune = true;
    uint64_t graph_tick = 0;
    uint64_t graph_captures = 0, graph_replays = 0;
    std::map<std::tuple<int, int, int, int, int, int>, int> tuned;  // shape -> split count
    std::mutex mu;                                              // guards all of the above
    Server* server = nullptr;
};

namespace {

sc_status fail(sc_ctx* c, sc_status st, const char* fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (c) c->err = buf;
    return st;
}

sc_status cuda_fail(sc_ctx* c, cudaError_t e, const char* what)
{
    return fail(c, e == cudaErrorMemoryAllocation ? SC_ERR_OOM : SC_ERR_CUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

#define SC_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e__ = (call);                        \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, what); \
    } while (0)

sc_status ensure(sc_ctx* ctx, DevBuf& b, size_t bytes, cudaStream_t sync_stream);

sc_status ensure(sc_ctx* ctx, DevBuf& b, size_t bytes)
{
    return ensure(ctx, b, bytes, ctx->stream);
}

sc_status ensure(sc_ctx* ctx, DevBuf& b, size_t bytes, cudaStream_t sync_stream)
{
    if (b.n >= bytes) return SC_OK;
    size_t want = std::max(bytes, b.n + b.n / 2);
    if (ctx->budget && ctx->held - b.n + want > ctx->budget) {
        want = bytes;
        if (ctx->held - b.n + want > ctx->budget)
            return fail(ctx, SC_ERR_OOM, "device budget of %zu bytes exceeded (need %zu more)",
                        ctx->budget, want);
    }
    if (b.p) {
        cudaStreamSynchronize(sync_stream);
        cudaFree(b.p);
        ctx->held -= b.n;
        b.p = nullptr;
        b.n = 0;
    }
    cudaError_t e = cudaMalloc(&b.p, want);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(ctx, SC_ERR_OOM, "cudaMalloc(%zu) failed: %s", want, cudaGetErrorString(e));
    }
    b.n = want;
    ctx->held += want;
    return SC_OK;
}

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    cudaError_t e = cudaPointerGetAttributes(&a, p);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
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

struct SurfPt {
    double z, dzdr;  // F(r), F'(r): n dS = (-F' cos, -F' sin, 1) r dr dtheta
    double pn;       // |P|, the distance to the focus
    double extra;    // optical path added to W so that the kernel's phase
                     // R - |P| + W equals R - (z + z_ref) + W (collimated beams)
};

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

struct HostNode {
    double px, py, pz, pn, w, jx, jy, jz, rho;
};

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
    gauss_legendre(nr, m->r_min, m->r_max, gr, gw);
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
    surf.clear();
    surf1.clear();
    surf.reserve((size_t)nr * nt);
    if (first) surf1.reserve((size_t)nr * nt);
    for (int i = 0; i < nr; ++i) {
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
            surf.push_back(nd);
            if (first) {
                double de, db;
                incident_div(in, r, th, de, db);
                HostNode n1 = nd;
                n1.jx = Ny * db * wq;   // N x (0, 0, db)
                n1.jy = -Nx * db * wq;
                n1.jz = 0.0;
                n1.rho = Nz * de * wq;  // N . (0, 0, de)
                surf1.push_back(n1);
            }
        }
    }
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
struct HostPart {
    int kind = PART_ONE, m = 0;
    std::vector<HostNode> surf, rim;
};

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
    gauss_legendre(nr, m->r_min, m->r_max, gr, gw);
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
    gauss_legendre(nr, m->r_min, m->r_max, gr, gw);
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
    SC_CUDA(cudaMemcpyAsync(t.d32, t32.data(), b32, cudaMemcpyHostToDevice, stream), "upload node tables");
    SC_CUDA(cudaMemcpyAsync(t.d64, h64.data(), b64, cudaMemcpyHostToDevice, stream), "upload FP64 tables");
    // the host vectors die at return: make the copies complete first
    SC_CUDA(cudaStreamSynchronize(stream), "node table upload");
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


// ------------------------------------------------------------------------
// Batched FP32 execution (A8): requests are cut into chunks (<= 2048 omegas,
// points bounded by the workspace cap); chunks of one kernel class run in one
// persistent launch whose CTAs take (chunk, point block, split) items from a
// device queue; one batched FP64 reduce finishes every chunk.  The field
// launches of a batch are captured into a CUDA graph and replayed while the
// launch signature repeats.  Each chunk's split count comes from the
// autotuner cache (or the heuristic), never from the rest of the batch, so a
// request gives bitwise the same result alone or in a mix.

struct Chunk {
    sc::FieldLaunch f;      // part 0; ws assigned at execution
    sc::ReduceLaunch rl;    // ws, off assigned at execution
    const Table* tab = nullptr;  // its parts share f's points, omegas and splits
    int n_parts = 1;
    int cls = 0, ppc = 1, pb = 1;
    size_t ws_elems = 0;    // float2 elements, every part (one section each)
};

// Split a chunk's surface tiles S ways.  Every table part (same nodes) uses
// the same splits and a workspace section of its own.
void set_splits(Chunk& c, int S, int tiles)
{
    const int tps = (tiles + S - 1) / S;
    c.f.tiles_per_split = tps;
    c.f.n_splits = (tiles + tps - 1) / tps;
    c.rl.n_splits = c.f.n_splits;
    c.ws_elems = (size_t)(c.f.n_splits + 1) * c.f.n_pts * c.f.n_omega * sc::kAcc * c.n_parts;
}

int heuristic_splits(int tiles, long long pb, int slots)
{
    // enough items for dynamic balance (about 16 per resident CTA), items of
    // at least 32 node tiles, at most 64 splits
    long long s = (16LL * slots + pb - 1) / pb;
    s = std::min<long long>(s, std::max(1, tiles / 32));
    return (int)std::max<long long>(1, std::min<long long>(64, s));
}

sc_status launch_chunks_direct(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, float2* ws, size_t ws_n);

// Time one chunk with split count S (the chunk's outputs are overwritten later).
float time_chunk(sc_ctx* ctx, Lane& ln, Chunk c, int S, const Table* tab, float2* ws)
{
    set_splits(c, S, tab->n_surf_tiles);
    std::vector<Chunk> one{c};
    cudaEvent_t a = take_event(ctx), b = take_event(ctx);
    cudaEventRecord(a, ln.stream);
    sc_status st = launch_chunks_direct(ctx, ln, one, ws, c.ws_elems);
    cudaEventRecord(b, ln.stream);
    float ms = 1e30f;
    if (st == SC_OK && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaGetLastError();
    ctx->pool.push_back(a);
    ctx->pool.push_back(b);
    return ms;
}

// Split count for a chunk shape: explicit option, tuned value, or heuristic
// (tuned on first sight when the autotuner is on).
sc_status choose_splits(sc_ctx* ctx, Lane& ln, Chunk& c, const Table* tab, int slots, int* S_out)
{
    const int tiles = tab->n_surf_tiles;
    if (ctx->nodes_per_split > 0) {
        const int tps = (int)std::max<long long>(1, ctx->nodes_per_split / sc::kTile);
        *S_out = (tiles + tps - 1) / tps;
        return SC_OK;
    }
    const auto key = std::make_tuple(c.cls, tiles, tab->n_rim_tiles, c.f.n_pts, c.f.n_omega, c.n_parts);
    auto hit = ctx->tuned.find(key);
    if (hit != ctx->tuned.end()) {
        *S_out = hit->second;
        return SC_OK;
    }
    const int s0 = heuristic_splits(tiles, c.pb, slots);
    int best = s0;
    if (ctx->autotune) {
        // candidates around the heuristic, each timed once on the real chunk
        std::vector<int> cand;
        for (int s : {s0 / 2, s0, 2 * s0, 4 * s0})
            if (s >= 1 && s <= std::min(64, tiles) &&
                std::find(cand.begin(), cand.end(), s) == cand.end())
                cand.push_back(s);
        // only candidates whose whole-request workspace fits under the cap
        size_t need = 0;
        std::vector<int> fit;
        for (int s : cand) {
            const int tps = (tiles + s - 1) / s;
            const int ns = (tiles + tps - 1) / tps;
            const size_t n = (size_t)(ns + 1) * c.f.n_pts * c.f.n_omega * sc::kAcc * c.n_parts;
            if (n * sizeof(float2) <= ctx->ws_cap) {
                fit.push_back(s);
                need = std::max(need, n);
            }
        }
        if (fit.size() > 1) {
            sc_status st = ensure(ctx, ln.ws, need * sizeof(float2), ln.stream);
            if (st != SC_OK) return st;
            float best_ms = 1e30f;
            for (int s : fit) {
                const float ms = time_chunk(ctx, ln, c, s, tab, (float2*)ln.ws.p);
                if (ms < best_ms) { best_ms = ms; best = s; }
            }
        }
    }
    ctx->tuned[key] = best;
    *S_out = best;
    return SC_OK;
}

// Cut one request into chunks.  d_amp / d_k point at this request's a_n, k_n.
sc_status plan_request(sc_ctx* ctx, Lane& ln, const Table* tab, const double* omegas, int n_omega,
                       double dom, const double* d_pts, int n_points, const double* d_amp,
                       const double* d_k, float2* dE, float2* dB, std::vector<Chunk>& out)
{
    if (!tab->fp32_ok)
        return fail(ctx, SC_ERR_INVALID,
                    "this mirror and beam do not focus on the origin (e.g. a collimated beam on an "
                    "ellipsoid): the compensated FP32 phase does not apply, use SC_FP64");
    const int max_om_chunk = 2048;
    const int flush_tiles = (int)std::max<long long>(1, ctx->flush_nodes / sc::kTile);
    for (int o0 = 0; o0 < n_omega; o0 += max_om_chunk) {
        const int no = std::min(max_om_chunk, n_omega - o0);
        Chunk c;
        c.cls = sc::field_class(no);
        int slots = 1;
        sc::field_shape(c.cls, ctx->device, &c.ppc, &slots);
        const double w0 = omegas[o0];
        c.f.nodes = tab->d32;
        c.f.n_surf_tiles = tab->n_surf_tiles;
        c.f.n_rim_tiles = tab->n_rim_tiles;
        c.f.flush_tiles = flush_tiles;
        c.f.n_omega = no;
        c.f.om_hi0 = (float)w0;
        c.f.om_lo0 = (float)(w0 - (double)c.f.om_hi0);
        c.f.dom_hi = (float)dom;
        c.f.dom_lo = (float)(dom - (double)c.f.dom_hi);
        c.f.err = ctx->d_err;
        c.f.ws = nullptr;
        // the split count is chosen on the whole request's point count
        c.f.pts = d_pts;
        c.f.n_pts = n_points;
        c.pb = (n_points + c.ppc - 1) / c.ppc;
        c.rl.amp = d_amp + 2 * (size_t)o0;
        c.rl.kval = d_k + o0;
        c.rl.out_pt_stride_omega = (long long)n_points * 3;
        c.rl.E = dE + (size_t)o0 * n_points * 3;
        c.rl.B = dB ? dB + (size_t)o0 * n_points * 3 : nullptr;
        c.rl.n_pts = n_points;
        c.rl.n_omega = no;
        c.tab = tab;
        c.n_parts = (int)tab->parts.size();
        c.rl.n_parts = c.n_parts;
        c.rl.amp_stride = 2LL * n_omega;
        int S = 1;
        sc_status st = choose_splits(ctx, ln, c, tab, slots, &S);
        if (st != SC_OK) return st;
        set_splits(c, S, tab->n_surf_tiles);
        const int n_splits = c.f.n_splits;
        // point chunks bounded by the workspace cap
        const size_t per_pt = (size_t)(n_splits + 1) * no * sc::kAcc * c.n_parts;
        long long pchunk = std::max<long long>(1, (long long)(ctx->ws_cap / sizeof(float2) / per_pt));
        if (pchunk < n_points) pchunk = std::max<long long>(c.ppc, pchunk / c.ppc * c.ppc);
        for (int p0 = 0; p0 < n_points; p0 += (int)pchunk) {
            const int np = (int)std::min<long long>(pchunk, n_points - p0);
            Chunk d = c;
            d.f.pts = d_pts + 3 * (size_t)p0;
            d.f.n_pts = np;
            d.pb = (np + c.ppc - 1) / c.ppc;
            d.rl.n_pts = np;
            d.rl.E = c.rl.E + (size_t)p0 * 3;
            d.rl.B = c.rl.B ? c.rl.B + (size_t)p0 * 3 : nullptr;
            d.ws_elems = per_pt * np;
            out.push_back(d);
        }
    }
    return SC_OK;
}

// Launch a group of chunks whose workspaces fit in ws, with or without a
// CUDA graph.  Field kernels (one persistent launch per class present) go
// in the graph; the batched reduce follows on the stream.
sc_status launch_chunks(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, float2* ws, size_t ws_n, bool graph)
{
    // workspace offsets and reduce offsets
    size_t off = 0;
    long long roff = 0;
    for (auto& c : ch) {
        c.f.ws = ws + off;
        c.rl.ws = ws + off;
        c.rl.off = roff;
        off += c.ws_elems;
        roff += (long long)c.rl.n_pts * c.rl.n_omega;
    }
    if (off > ws_n) return fail(ctx, SC_ERR_OOM, "workspace plan exceeds its buffer");
    // per-class descriptor arrays
    constexpr int kClasses = sc::kNumClasses;
    std::vector<sc::WorkReq> reqs[kClasses];
    long long items[kClasses] = {};
    for (auto& c : ch)
        for (int t = 0; t < c.n_parts; ++t) {
            sc::WorkReq w;
            w.f = c.f;
            w.f.nodes = c.tab->parts[t].d32;
            w.f.n_rim_tiles = c.tab->parts[t].n_rim_tiles;
            w.f.ws = c.f.ws + (size_t)t * (c.ws_elems / c.n_parts);
            w.pb = c.pb;
            w.cls = c.cls;
            w.item0 = items[c.cls];
            items[c.cls] += (long long)c.pb * (w.f.n_splits + 1);
            reqs[c.cls].push_back(w);
        }
    std::vector<sc::ReduceLaunch> rls;
    for (auto& c : ch) rls.push_back(c.rl);
    // arena: queues (64 B each) | WorkReq arrays | ReduceLaunch array
    size_t bytes = kClasses * 64;
    size_t req_off[kClasses];
    for (int k = 0; k < kClasses; ++k) {
        req_off[k] = bytes;
        bytes += (reqs[k].size() * sizeof(sc::WorkReq) + 255) / 256 * 256;
    }
    const size_t rl_off = bytes;
    bytes += rls.size() * sizeof(sc::ReduceLaunch);
    sc_status st = ensure(ctx, ln.desc, bytes, ln.stream);
    if (st != SC_OK) return st;
    unsigned char* arena = (unsigned char*)ln.desc.p;
    for (int k = 0; k < kClasses; ++k)
        if (!reqs[k].empty())
            SC_CUDA(cudaMemcpyAsync(arena + req_off[k], reqs[k].data(), reqs[k].size() * sizeof(sc::WorkReq),
                                    cudaMemcpyHostToDevice, ln.stream), "upload work descriptors");
    SC_CUDA(cudaMemcpyAsync(arena + rl_off, rls.data(), rls.size() * sizeof(sc::ReduceLaunch),
                            cudaMemcpyHostToDevice, ln.stream), "upload reduce descriptors");

    struct L { int cls; sc::BatchLaunch b; int grid; };
    std::vector<L> launches;
    for (int k = 0; k < kClasses; ++k) {
        if (reqs[k].empty()) continue;
        int ppc = 1, slots = 1;
        sc::field_shape(k, ctx->device, &ppc, &slots);
        sc::BatchLaunch b{};
        b.reqs = (const sc::WorkReq*)(arena + req_off[k]);
        b.n_req = (int)reqs[k].size();
        b.n_items = items[k];
        b.queue = (int*)(arena + 64 * k);
        b.err = ctx->d_err;
        launches.push_back({k, b, (int)std::min<long long>(slots, items[k])});
    }
    auto issue = [&](cudaStream_t s) -> sc_status {
        SC_CUDA(cudaMemsetAsync(arena, 0, kClasses * 64, s), "reset work queues");
        for (auto& l : launches) {
            const int r = sc::launch_field_batch(l.cls, l.b, l.grid, s);
            if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "field kernel launch");
        }
        return SC_OK;
    };
    cudaEvent_t f0 = nullptr, f1 = nullptr;
    if (ctx->time_field) {
        f0 = take_event(ctx);
        f1 = take_event(ctx);
        cudaEventRecord(f0, ln.stream);
    }
    if (graph) {
        // signature: everything the captured launches depend on
        std::vector<unsigned char> sig;
        auto put = [&](const void* p, size_t n) {
            const unsigned char* q = (const unsigned char*)p;
            sig.insert(sig.end(), q, q + n);
        };
        put(&arena, sizeof arena);
        for (auto& l : launches) {
            put(&l.cls, sizeof l.cls);
            put(&l.grid, sizeof l.grid);
            put(&l.b, sizeof l.b);
        }
        cudaGraphExec_t exec = nullptr;
        for (auto& g : ln.graphs)
            if (g.sig == sig) {
                exec = g.exec;
                g.last = ++ctx->graph_tick;
                ctx->graph_replays++;
            }
        if (!exec) {
            if (!ln.cap_stream)
                SC_CUDA(cudaStreamCreateWithFlags(&ln.cap_stream, cudaStreamNonBlocking), "capture stream");
            SC_CUDA(cudaStreamBeginCapture(ln.cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
            st = issue(ln.cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(ln.cap_stream, &g);
            if (st != SC_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
            e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
            if (ln.graphs.size() >= 8) {
                auto it = std::min_element(ln.graphs.begin(), ln.graphs.end(),
                                           [](const GraphEntry& a, const GraphEntry& b) {
                                               return a.last < b.last;
                                           });
                cudaGraphExecDestroy(it->exec);
                ln.graphs.erase(it);
            }
            ln.graphs.push_back({sig, exec, ++ctx->graph_tick});
            ctx->graph_captures++;
        }
        SC_CUDA(cudaGraphLaunch(exec, ln.stream), "graph launch");
    } else {
        st = issue(ln.stream);
        if (st != SC_OK) return st;
    }
    if (ctx->time_field) {
        cudaEventRecord(f1, ln.stream);
        ctx->pending.push_back({f0, f1});
    }
    ctx->ctr.launches += launches.size();
    ctx->ctr.field_launches += launches.size();
    const int r = sc::launch_reduce_batch((const sc::ReduceLaunch*)(arena + rl_off), (int)rls.size(),
                                          roff, ln.stream);
    if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "reduce launch");
    ctx->ctr.launches += r;
    return SC_OK;
}

sc_status launch_chunks_direct(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, float2* ws, size_t ws_n)
{
    const bool t = ctx->time_field;
    ctx->time_field = false;
    sc_status st = launch_chunks(ctx, ln, ch, ws, ws_n, false);
    ctx->time_field = t;
    return st;
}

// Run chunks in groups whose workspace fits under the cap.
sc_status run_chunks(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch)
{
    const size_t cap = std::max<size_t>(ctx->ws_cap / sizeof(float2), 1);
    size_t i = 0;
    while (i < ch.size()) {
        size_t j = i, tot = 0;
        while (j < ch.size() && (j == i || tot + ch[j].ws_elems <= cap)) tot += ch[j++].ws_elems;
        sc_status st = ensure(ctx, ln.ws, tot * sizeof(float2), ln.stream);
        if (st != SC_OK) return st;
        std::vector<Chunk> part(ch.begin() + i, ch.begin() + j);
        st = launch_chunks(ctx, ln, part, (float2*)ln.ws.p, tot, ctx->use_graphs);
        if (st != SC_OK) return st;
        i = j;
    }
    return SC_OK;
}

void free_lane(Lane& ln)
{
    if (ln.stream) cudaStreamSynchronize(ln.stream);
    for (DevBuf* b : {&ln.ws, &ln.desc, &ln.amp, &ln.kval})
        if (b->p) {
            cudaFree(b->p);
            b->p = nullptr;
            b->n = 0;
        }
    for (auto& g : ln.graphs) cudaGraphExecDestroy(g.exec);
    ln.graphs.clear();
    if (ln.cap_stream) cudaStreamDestroy(ln.cap_stream);
    ln.cap_stream = nullptr;
    if (ln.own_stream && ln.stream) cudaStreamDestroy(ln.stream);
    ln.stream = nullptr;
}

// ------------------------------------------------------------------------
// Serving (A9): continuous batching of submitted requests.  A server thread
// admits queued requests in arrival order while their device memory (staged
// points and server-owned outputs) fits the context's HBM budget, batches up
// to max_batch of them and runs the batch on a free lane; with two lanes a
// new batch starts while the previous one is still on the GPU, so requests
// that arrive meanwhile overlap with it.  Completion is observed through an
// event per lane; memory returns to the budget when the caller releases the
// ticket.

struct Ticket {
    const sc_mirror_t* mirror = nullptr;
    const sc_incident_t* incident = nullptr;
    std::vector<double> omegas, host_pts;
    const double* user_pts = nullptr;   // caller's device points (or null)
    int n_points = 0, n_omega = 0;
    double dom = 0.0;
    void* E_user = nullptr;             // caller-owned device outputs (or null)
    void* B_user = nullptr;
    void* E = nullptr;                  // outputs in use
    void* B = nullptr;
    double* pts = nullptr;              // device points in use
    bool own_out = false, own_pts = false;
    size_t bytes = 0;                   // device bytes this ticket holds
    int state = 0;                      // 0 queued, 1 running, 2 done, 3 failed, 4 cancelled
    bool cancel = false;
    sc_status status = SC_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    int lane = -1;
    Table* tab = nullptr;
};

struct Server {
    static constexpr int kLanes = 2;
    std::thread th;
    bool stop = false;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Ticket> tickets;
    Lane lanes[kLanes];
    cudaEvent_t done_ev[kLanes] = {};
    std::vector<uint64_t> batch[kLanes];
    bool busy[kLanes] = {};
    size_t held = 0;                    // bytes of admitted tickets not yet released
    uint64_t next_id = 1;
    int max_batch = 64;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

size_t ticket_bytes(const Ticket& t)
{
    size_t b = 0;
    if (t.own_pts) b += (size_t)t.n_points * 3 * sizeof(double);
    if (t.own_out) b += (size_t)2 * t.n_omega * t.n_points * 3 * sizeof(float2);
    return b;
}

// Run one batch of admitted tickets on lane L (ctx->mu held).  A ticket
// whose node tables cannot be built (an envelope too rough to fit, a device
// allocation that failed) fails alone and leaves ids; the others run.
sc_status launch_batch(sc_ctx* ctx, Server* srv, int L, std::vector<uint64_t>& ids)
{
    Lane& ln = srv->lanes[L];
    ctx->tick++;
    std::vector<double> amp_all, k_all;
    std::vector<size_t> om_off, amp_off;
    std::vector<uint64_t> run;
    for (uint64_t id : ids) {
        Ticket& t = srv->tickets[id];
        t.lane = L;
        t.t_start = srv->now();
        std::vector<double> a;
        sc_status tst = get_table(ctx, t.mirror, t.incident, &t.tab, ln.stream);
        if (tst == SC_OK) tst = request_amps(ctx, t.incident, t.tab, t.omegas.data(), t.n_omega, a);
        if (tst != SC_OK) {
            t.tab = nullptr;
            t.state = 3;
            t.status = tst;
            t.t_done = srv->now();
            continue;
        }
        t.state = 1;
        t.tab->inflight++;
        run.push_back(id);
        if (t.own_pts) {
            SC_CUDA(cudaMallocAsync((void**)&t.pts, (size_t)t.n_points * 3 * sizeof(double), ln.stream),
                    "serving points");
            SC_CUDA(cudaMemcpyAsync(t.pts, t.host_pts.data(), (size_t)t.n_points * 3 * sizeof(double),
                                    cudaMemcpyHostToDevice, ln.stream), "stage points");
        } else {
            t.pts = (double*)t.user_pts;
        }
        if (t.own_out) {
            const size_t ob = (size_t)t.n_omega * t.n_points * 3 * sizeof(float2);
            SC_CUDA(cudaMallocAsync(&t.E, ob, ln.stream), "serving outputs");
            SC_CUDA(cudaMallocAsync(&t.B, ob, ln.stream), "serving outputs");
        } else {
            t.E = t.E_user;
            t.B = t.B_user;
        }
        amp_off.push_back(amp_all.size());
        om_off.push_back(k_all.size());
        amp_all.insert(amp_all.end(), a.begin(), a.end());
        for (double w : t.omegas) k_all.push_back(2.0 * kPi * w);
    }
    ids.swap(run);
    if (ids.empty()) return SC_OK;
    sc_status st;
    if ((st = ensure(ctx, ln.amp, amp_all.size() * sizeof(double), ln.stream)) != SC_OK) return st;
    if ((st = ensure(ctx, ln.kval, k_all.size() * sizeof(double), ln.stream)) != SC_OK) return st;
    SC_CUDA(cudaMemcpyAsync(ln.amp.p, amp_all.data(), amp_all.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ln.stream), "upload amplitudes");
    SC_CUDA(cudaMemcpyAsync(ln.kval.p, k_all.data(), k_all.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ln.stream), "upload wavenumbers");
    std::vector<Chunk> ch;
    for (size_t i = 0; i < ids.size(); ++i) {
        Ticket& t = srv->tickets[ids[i]];
        st = plan_request(ctx, ln, t.tab, t.omegas.data(), t.n_omega, t.dom, t.pts, t.n_points,
                          (const double*)ln.amp.p + amp_off[i], (const double*)ln.kval.p + om_off[i],
                          (float2*)t.E, (float2*)t.B, ch);
        if (st != SC_OK) return st;
        ctx->ctr.evals += (double)t.n_points * t.tab->n_surf * t.n_omega;
    }
    st = run_chunks(ctx, ln, ch);
    if (st != SC_OK) return st;
    SC_CUDA(cudaEventRecord(srv->done_ev[L], ln.stream), "completion event");
    return SC_OK;
}

void serve(sc_ctx* ctx)
{
    Server* srv = ctx->server;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (!srv->stop) {
        bool changed = false;
        // completions
        for (int L = 0; L < Server::kLanes; ++L) {
            if (!srv->busy[L]) continue;
            const cudaError_t q = cudaEventQuery(srv->done_ev[L]);
            if (q == cudaErrorNotReady) continue;
            const double t = srv->now();
            for (uint64_t id : srv->batch[L]) {
                auto it = srv->tickets.find(id);
                if (it == srv->tickets.end()) continue;
                Ticket& tk = it->second;
                if (tk.tab) tk.tab->inflight--;
                tk.tab = nullptr;
                tk.t_done = t;
                if (q != cudaSuccess) {
                    tk.state = 3;
                    tk.status = SC_ERR_CUDA;
                } else {
                    tk.state = tk.cancel ? 4 : 2;
                }
            }
            if (q != cudaSuccess) cudaGetLastError();
            srv->batch[L].clear();
            srv->busy[L] = false;
            changed = true;
        }
        // admission and launch on free lanes
        for (int L = 0; L < Server::kLanes && !srv->queue.empty(); ++L) {
            if (srv->busy[L]) continue;
            // workspace the lanes may still grow into (bounded by the cap)
            size_t reserve = size_t(16) << 20;
            for (int M = 0; M < Server::kLanes; ++M)
                if (srv->lanes[M].ws.n < ctx->ws_cap) reserve += ctx->ws_cap - srv->lanes[M].ws.n;
            std::vector<uint64_t> ids;
            while (!srv->queue.empty() && (int)ids.size() < srv->max_batch) {
                Ticket& t = srv->tickets[srv->queue.front()];
                const size_t b = ticket_bytes(t);
                // admit only what fits next to every lane's full workspace; the
                // first request of an idle server is always admitted
                const bool idle = srv->held == 0 && ids.empty();
                if (ctx->budget && !idle && ctx->held + srv->held + b + reserve > ctx->budget) break;
                t.bytes = b;
                srv->held += b;
                ids.push_back(srv->queue.front());
                srv->queue.pop_front();
            }
            if (ids.empty()) break;
            const sc_status st = launch_batch(ctx, srv, L, ids);
            if (st == SC_OK && ids.empty()) {
                changed = true;
                continue;
            }
            if (st != SC_OK) {
                cudaStreamSynchronize(srv->lanes[L].stream);
                for (uint64_t id : ids) {
                    Ticket& t = srv->tickets[id];
                    if (t.tab) t.tab->inflight--;
                    t.tab = nullptr;
                    t.state = 3;
                    t.status = st;
                    t.t_done = srv->now();
                }
            } else {
                srv->batch[L] = ids;
                srv->busy[L] = true;
            }
            changed = true;
        }
        if (changed) srv->cv.notify_all();
        srv->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

sc_status start_server(sc_ctx* ctx)
{
    if (ctx->server) return SC_OK;
    Server* srv = new Server();
    for (int L = 0; L < Server::kLanes; ++L) {
        if (cudaStreamCreateWithFlags(&srv->lanes[L].stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&srv->done_ev[L], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            delete srv;
            return fail(ctx, SC_ERR_CUDA, "serving lane set-up failed");
        }
        srv->lanes[L].own_stream = true;
    }
    ctx->server = srv;
    srv->th = std::thread(serve, ctx);
    return SC_OK;
}

void free_ticket_memory(Server* srv, Ticket& t)
{
    cudaStream_t s = t.lane >= 0 ? srv->lanes[t.lane].stream : nullptr;
    if (t.own_pts && t.pts) cudaFreeAsync(t.pts, s);
    if (t.own_out && t.E) cudaFreeAsync(t.E, s);
    if (t.own_out && t.B) cudaFreeAsync(t.B, s);
    t.pts = nullptr;
    t.E = t.B = nullptr;
    srv->held -= t.bytes;
    t.bytes = 0;
}

void stop_server(sc_ctx* ctx)
{
    Server* srv = ctx->server;
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    srv->th.join();
    cudaSetDevice(ctx->device);
    for (int L = 0; L < Server::kLanes; ++L) cudaStreamSynchronize(srv->lanes[L].stream);
    for (auto& kv : srv->tickets) {
        if (kv.second.tab) kv.second.tab->inflight--;
        free_ticket_memory(srv, kv.second);
    }
    for (int L = 0; L < Server::kLanes; ++L) {
        cudaStreamSynchronize(srv->lanes[L].stream);
        free_lane(srv->lanes[L]);
        if (srv->done_ev[L]) cudaEventDestroy(srv->done_ev[L]);
    }
    delete srv;
    ctx->server = nullptr;
}

}  // namespace

// --------------------------------------------------------------------------
// C-ABI

extern "C" {

sc_status sc_create(int device, void* cuda_stream, size_t hbm_budget_bytes, sc_ctx** out)
{
    if (!out) return SC_ERR_INVALID;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
        cudaGetLastError();
        return SC_ERR_CUDA;
    }
    if (device < 0 || device >= ndev) return SC_ERR_INVALID;
    if (cudaSetDevice(device) != cudaSuccess) return SC_ERR_CUDA;
    sc_ctx* ctx = new sc_ctx();
    ctx->device = device;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->main.stream = ctx->stream;
    ctx->budget = hbm_budget_bytes;
    if (cudaMalloc(&ctx->d_err, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->h_err, sizeof(int)) != cudaSuccess ||
        cudaMemset(ctx->d_err, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        if (ctx->d_err) cudaFree(ctx->d_err);
        delete ctx;
        return SC_ERR_CUDA;
    }
    *out = ctx;
    return SC_OK;
}

sc_status sc_destroy(sc_ctx* ctx)
{
    if (!ctx) return SC_OK;
    stop_server(ctx);
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    settle_events(ctx);
    for (auto& t : ctx->tables) free_table(ctx, t);
    for (DevBuf* b : {&ctx->pts, &ctx->outE, &ctx->outB, &ctx->tkval, &ctx->tvals, &ctx->phasor,
                      &ctx->specE, &ctx->specB, &ctx->tE, &ctx->tB, &ctx->fpts, &ctx->fspecE,
                      &ctx->fspecB, &ctx->ftE, &ctx->ftB})
        if (b->p) cudaFree(b->p);
    free_lane(ctx->main);
    for (cudaEvent_t e : ctx->pool) cudaEventDestroy(e);
    if (ctx->d_err) cudaFree(ctx->d_err);
    if (ctx->h_err) cudaFreeHost(ctx->h_err);
    delete ctx;
    return SC_OK;
}

const char* sc_last_error(const sc_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

sc_status sc_mirror(sc_ctx* ctx, double f, double r_min, double r_max, const sc_quadrature* q,
                    sc_mirror_t** out)
{
    if (!out || !q) return fail(ctx, SC_ERR_INVALID, "null argument");
    *out = nullptr;
    if (!(f > 0.0) || !(r_min >= 0.0) || !(r_max > r_min) || q->n_r < 1 || q->n_theta < 1 ||
        q->radial_kind != SC_QUAD_GAUSS_LEGENDRE)
        return fail(ctx, SC_ERR_INVALID,
                    "invalid mirror (f=%g r_min=%g r_max=%g n_r=%d n_theta=%d kind=%d)", f, r_min,
                    r_max, q->n_r, q->n_theta, q->radial_kind);
    sc_mirror_t* m = new sc_mirror_t();
    m->id = g_next_id++;
    m->f = f;
    m->r_min = r_min;
    m->r_max = r_max;
    m->q = *q;
    *out = m;
    return SC_OK;
}

sc_status sc_mirror_ellipsoid(sc_ctx* ctx, double c, double e, double r_min, double r_max,
                              const sc_quadrature* q, sc_mirror_t** out)
{
    if (!out || !q) return fail(ctx, SC_ERR_INVALID, "null argument");
    *out = nullptr;
    if (!(e > 0.0) || !(c > e) || !(r_min >= 0.0) || !(r_max > r_min) || !(r_max * r_max < c * c - e * e) ||
        q->n_r < 1 || q->n_theta < 1 || q->radial_kind != SC_QUAD_GAUSS_LEGENDRE)
        return fail(ctx, SC_ERR_INVALID, "invalid ellipsoidal mirror (c=%g e=%g r_min=%g r_max=%g)", c, e, r_min,
                    r_max);
    sc_mirror_t* m = new sc_mirror_t();
    m->id = g_next_id++;
    m->surface = 2;
    m->c = c;
    m->e = e;
    m->f = c - e;
    m->r_min = r_min;
    m->r_max = r_max;
    m->q = *q;
    *out = m;
    return SC_OK;
}

void sc_mirror_free(sc_mirror_t* m) { delete m; }

sc_status sc_incident(sc_ctx* ctx, const sc_profile* prof, const sc_polarization* pol,
                      const sc_spectrum* spec, sc_incident_t** out)
{
    if (!out || !prof || !pol || !spec) return fail(ctx, SC_ERR_INVALID, "null argument");
    *out = nullptr;
    if (prof->kind < 0 || prof->kind > 5 || !(prof->w0 > 0.0) ||
        (prof->kind == SC_PROFILE_SUPERGAUSS && prof->sg_order < 1) || prof->n_zernike < 0 ||
        prof->n_zernike > 64 || (prof->n_zernike > 0 && !prof->zernike_noll_waves))
        return fail(ctx, SC_ERR_INVALID, "invalid beam profile");
    if (prof->order < 0 || prof->order > 1 || (prof->order == 1 && prof->kind >= SC_PROFILE_TOPHAT))
        return fail(ctx, SC_ERR_INVALID, "beam order must be 0 or 1 (1 needs a smooth collimated profile)");
    if (prof->kind == SC_PROFILE_DIPOLE &&
        (!(prof->dipole[0] != 0.0 || prof->dipole[1] != 0.0 || prof->dipole[2] != 0.0) ||
         spec->kind == SC_SPEC_GAUSS_TIME || spec->kind == SC_SPEC_SUPERGAUSS_LAMBDA))
        return fail(ctx, SC_ERR_INVALID, "a dipole needs a nonzero moment and a SAMPLED or MONO spectrum");
    if (prof->kind == SC_PROFILE_LAGUERRE_GAUSS || prof->kind == SC_PROFILE_ENVELOPE) {
        if (!(prof->omega_lo > 0.0) || !(prof->omega_hi > prof->omega_lo))
            return fail(ctx, SC_ERR_INVALID, "kinds 3-4 need a band 0 < omega_lo < omega_hi");
        if (prof->kind == SC_PROFILE_LAGUERRE_GAUSS &&
            (prof->lg_p < 0 || prof->lg_p > 32 || (pol && pol->kind != SC_POL_LINEAR && abs(prof->lg_l) != 1)))
            return fail(ctx, SC_ERR_INVALID, "Laguerre-Gauss needs 0 <= p <= 32 and |l| = 1 when radial or azimuthal");
        if (prof->kind == SC_PROFILE_ENVELOPE &&
            (!prof->envelope || spec->kind == SC_SPEC_GAUSS_TIME || spec->kind == SC_SPEC_SUPERGAUSS_LAMBDA))
            return fail(ctx, SC_ERR_INVALID, "an envelope beam needs a function and a SAMPLED or MONO spectrum");
    }
    if (pol->kind < 0 || pol->kind > 2) return fail(ctx, SC_ERR_INVALID, "invalid polarization");
    if (spec->kind < 0 || spec->kind > 3) return fail(ctx, SC_ERR_INVALID, "invalid spectrum kind");
    if (!(spec->lambda_c > 0.0) && spec->kind != SC_SPEC_MONO && spec->kind != SC_SPEC_SAMPLED)
        return fail(ctx, SC_ERR_INVALID, "lambda_c must be positive");
    if (spec->kind == SC_SPEC_GAUSS_TIME && !(spec->fwhm_t > 0.0))
        return fail(ctx, SC_ERR_INVALID, "fwhm_t must be positive");
    if (spec->kind == SC_SPEC_SUPERGAUSS_LAMBDA && (!(spec->dlambda > 0.0) || spec->sg_n < 1))
        return fail(ctx, SC_ERR_INVALID, "dlambda must be positive and sg_n >= 1");
    if (spec->kind == SC_SPEC_SAMPLED && (spec->n < 1 || !spec->omega || !spec->amp_re_im))
        return fail(ctx, SC_ERR_INVALID, "sampled spectrum needs n >= 1 omegas and amplitudes");
    if (spec->n_phi < 0 || (spec->n_phi > 0 && !spec->phi_taylor))
        return fail(ctx, SC_ERR_INVALID, "invalid spectral phase");
    sc_incident_t* in = new sc_incident_t();
    in->id = g_next_id++;
    in->profile = prof->kind;
    in->sg_order = prof->sg_order;
    in->order = prof->order;
    in->w0 = prof->w0;
    in->lg_p = prof->lg_p;
    in->lg_l = prof->lg_l;
    in->z_waist = prof->z_waist;
    in->env = prof->envelope;
    in->env_user = prof->envelope_user;
    in->om_lo = prof->omega_lo;
    in->om_hi = prof->omega_hi;
    in->fit_tol = prof->fit_tol > 0.0 ? prof->fit_tol : 1e-8;
    for (int c = 0; c < 3; ++c) in->dip[c] = prof->dipole[c];
    in->zern.assign(prof->zernike_noll_waves, prof->zernike_noll_waves + prof->n_zernike);
    in->pol = pol->kind;
    in->angle = pol->angle_rad;
    in->spec_kind = spec->kind;
    in->fwhm_t = spec->fwhm_t;
    in->lambda_c = spec->lambda_c > 0.0 ? spec->lambda_c : 1.0;
    in->dlambda = spec->dlambda;
    in->sg_n = spec->sg_n;
    in->energy = spec->energy;
    if (spec->kind == SC_SPEC_SAMPLED) {
        in->s_omega.assign(spec->omega, spec->omega + spec->n);
        in->s_amp.assign(spec->amp_re_im, spec->amp_re_im + 2 * spec->n);
    }
    if (spec->n_phi > 0) in->phi.assign(spec->phi_taylor, spec->phi_taylor + spec->n_phi);
    *out = in;
    return SC_OK;
}

void sc_incident_free(sc_incident_t* in) { delete in; }

sc_status sc_table_count(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in, int* n_tables,
                         int* fp32_ok)
{
    if (!m || !in || !n_tables) return fail(ctx, SC_ERR_INVALID, "null argument");
    std::vector<HostPart> hp;
    double kc = 0.0, kh = 1.0;
    sc_status st = build_host_parts(ctx, m, in, hp, kc, kh);
    if (st != SC_OK) return st;
    *n_tables = (int)hp.size();
    if (fp32_ok) *fp32_ok = focuses_on_origin(m, in) ? 1 : 0;
    return SC_OK;
}

sc_status sc_spectrum_eval(sc_ctx* ctx, const sc_incident_t* inc, const double* omegas, int n,
                           double* amp_re_im)
{
    if (!inc || !omegas || !amp_re_im || n < 1) return fail(ctx, SC_ERR_INVALID, "invalid argument");
    std::vector<double> a;
    sc_status st = spectrum_amps(ctx, inc, omegas, n, a);
    if (st != SC_OK) return st;
    memcpy(amp_re_im, a.data(), a.size() * sizeof(double));
    return SC_OK;
}

// sc_eval after validation, with ctx->mu held and the device set (dom: the
// omega step of the uniform grid the FP32 path needs).
static sc_status eval_unlocked(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in,
                               const double* omegas, int n_omega, const double* points_xyz,
                               int n_points, sc_precision prec, double dom, void* E_out,
                               void* B_out, sc_eval_stats* stats)
{
    const bool pts_dev = is_device_ptr(points_xyz);
    const bool e_dev = is_device_ptr(E_out);
    const bool b_dev = B_out ? is_device_ptr(B_out) : e_dev;
    if (B_out && e_dev != b_dev) return fail(ctx, SC_ERR_INVALID, "E_out and B_out must both be host or both device");

    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        ev0 = take_event(ctx);
        ev1 = take_event(ctx);
        cudaEventRecord(ev0, ctx->stream);
    }
    const double field_ms_before = ctx->ctr.field_ms;
    const uint64_t launches_before = ctx->ctr.launches;
    const bool timing_before = ctx->time_field;
    if (stats) ctx->time_field = true;

    Table* tab = nullptr;
    sc_status st = get_table(ctx, m, in, &tab, ctx->stream);
    if (st != SC_OK) return st;
    std::vector<double> amp;  // [part][omega][2]
    st = request_amps(ctx, in, tab, omegas, n_omega, amp);
    if (st != SC_OK) return st;
    std::vector<double> kv(n_omega);
    for (int i = 0; i < n_omega; ++i) kv[i] = 2.0 * kPi * omegas[i];

    // points on the device
    const double* d_pts = points_xyz;
    if (!pts_dev) {
        st = check_points_host(ctx, m, points_xyz, n_points);
        if (st != SC_OK) return st;
        if ((st = ensure(ctx, ctx->pts, (size_t)n_points * 3 * sizeof(double))) != SC_OK) return st;
        SC_CUDA(cudaMemcpyAsync(ctx->pts.p, points_xyz, (size_t)n_points * 3 * sizeof(double),
                                cudaMemcpyHostToDevice, ctx->stream), "upload points");
        d_pts = (const double*)ctx->pts.p;
    }
    if ((st = ensure(ctx, ctx->main.amp, amp.size() * sizeof(double))) != SC_OK) return st;
    if ((st = ensure(ctx, ctx->main.kval, kv.size() * sizeof(double))) != SC_OK) return st;
    SC_CUDA(cudaMemcpyAsync(ctx->main.amp.p, amp.data(), amp.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ctx->stream), "upload amplitudes");
    SC_CUDA(cudaMemcpyAsync(ctx->main.kval.p, kv.data(), kv.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ctx->stream), "upload wavenumbers");

    const size_t elem = prec == SC_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t out_bytes = (size_t)n_omega * n_points * 3 * elem;
    void* dE = E_out;
    void* dB = B_out;
    if (!e_dev) {
        if ((st = ensure(ctx, ctx->outE, out_bytes)) != SC_OK) return st;
        dE = ctx->outE.p;
        if (B_out) {
            if ((st = ensure(ctx, ctx->outB, out_bytes)) != SC_OK) return st;
            dB = ctx->outB.p;
        }
    }
    // the staging buffers may have moved: refresh pointers taken before
    if (!pts_dev) d_pts = (const double*)ctx->pts.p;
    const double* d_amp = (const double*)ctx->main.amp.p;
    const double* d_k = (const double*)ctx->main.kval.p;

    const double evals = (double)n_points * (double)tab->n_surf * (double)n_omega;

    if (prec == SC_FP64) {
        cudaEvent_t f0 = nullptr, f1 = nullptr;
        if (ctx->time_field) {
            f0 = take_event(ctx);
            f1 = take_event(ctx);
            cudaEventRecord(f0, ctx->stream);
        }
        for (size_t p = 0; p < tab->parts.size(); ++p) {
            const TablePart& tp = tab->parts[p];
            sc::Field64Launch a;
            a.surf = tp.d64;
            a.n_surf = tab->n_surf;
            a.rim = tp.d64 + tab->n_surf;
            a.n_rim = tp.n_rim;
            a.pts = d_pts;
            a.n_pts = n_points;
            a.kval = d_k;
            a.n_omega = n_omega;
            a.amp = d_amp + p * 2 * (size_t)n_omega;
            a.E = (double2*)dE;
            a.B = (double2*)dB;
            a.accumulate = p > 0;
            const int r = sc::launch_field_f64(a, ctx->stream);
            if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "FP64 field kernel launch");
            ctx->ctr.launches += r;
            ctx->ctr.field_launches += 1;
        }
        if (ctx->time_field) {
            cudaEventRecord(f1, ctx->stream);
            ctx->pending.push_back({f0, f1});
        }
    } else {
        std::vector<Chunk> ch;
        st = plan_request(ctx, ctx->main, tab, omegas, n_omega, dom, d_pts, n_points, d_amp, d_k,
                          (float2*)dE, (float2*)dB, ch);
        if (st != SC_OK) return st;
        st = run_chunks(ctx, ctx->main, ch);
        if (st != SC_OK) return st;
    }
    ctx->ctr.evals += evals;

    if (!e_dev) {
        SC_CUDA(cudaMemcpyAsync(E_out, dE, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "download E");
        if (B_out)
            SC_CUDA(cudaMemcpyAsync(B_out, dB, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "download B");
    }
    if (stats) cudaEventRecord(ev1, ctx->stream);
    if (stats || !e_dev) {
        st = check_device_error(ctx);
        if (st != SC_OK) return st;
    }
    if (stats) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        ctx->pool.push_back(ev0);
        ctx->pool.push_back(ev1);
        settle_events(ctx);
        stats->evals = evals;
        stats->total_ms = ms;
        stats->field_ms = ctx->ctr.field_ms - field_ms_before;
        stats->launches = (int)(ctx->ctr.launches - launches_before);
        stats->tables = (int)tab->parts.size();
        ctx->time_field = timing_before;
    }
    return SC_OK;
}

sc_status sc_eval(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in, const double* omegas,
                  int n_omega, const double* points_xyz, int n_points, sc_precision prec,
                  void* E_out, void* B_out, sc_eval_stats* stats)
{
    if (!ctx) return SC_ERR_INVALID;
    if (!m || !in || !omegas || !points_xyz || !E_out || n_omega < 1 || n_points < 1)
        return fail(ctx, SC_ERR_INVALID, "invalid argument");
    if (prec != SC_FP32_COMP && prec != SC_FP64) return fail(ctx, SC_ERR_INVALID, "bad precision");
    for (int i = 0; i < n_omega; ++i)
        if (!(omegas[i] > 0.0) || !std::isfinite(omegas[i]))
            return fail(ctx, SC_ERR_INVALID, "omega[%d] must be positive", i);
    double dom = 0.0;
    if (prec == SC_FP32_COMP && !uniform_grid(omegas, n_omega, dom))
        return fail(ctx, SC_ERR_INVALID, "SC_FP32_COMP needs a uniform, increasing omega grid");
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->tick++;

    return eval_unlocked(ctx, m, in, omegas, n_omega, points_xyz, n_points, prec, dom, E_out, B_out, stats);
}

static sc_status time_domain_unlocked(sc_ctx* ctx, sc_precision prec, const void* E_spec,
                                      const void* B_spec, const double* omegas, int n_omega,
                                      int n_points, const double* times, int n_t, float* E_t,
                                      float* B_t, double dk, int accumulate);

sc_status sc_eval_time_domain(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in,
                              const double* omegas, int n_omega, const double* points_xyz, int n_points,
                              sc_precision prec, const double* times, int n_t, int omega_chunk, float* E_t,
                              float* B_t, sc_eval_stats* stats)
{
    if (!ctx) return SC_ERR_INVALID;
    if (!m || !in || !omegas || !points_xyz || !times || !E_t || n_omega < 1 || n_points < 1 || n_t < 1)
        return fail(ctx, SC_ERR_INVALID, "invalid argument");
    if (prec != SC_FP32_COMP && prec != SC_FP64) return fail(ctx, SC_ERR_INVALID, "bad precision");
    for (int i = 0; i < n_omega; ++i)
        if (!(omegas[i] > 0.0) || !std::isfinite(omegas[i]))
            return fail(ctx, SC_ERR_INVALID, "omega[%d] must be positive", i);
    double dom = 0.0;
    if (!uniform_grid(omegas, n_omega, dom))
        return fail(ctx, SC_ERR_INVALID, "the inverse transform needs a uniform omega grid");
    const bool out_dev = is_device_ptr(E_t);
    if (B_t && is_device_ptr(B_t) != out_dev)
        return fail(ctx, SC_ERR_INVALID, "E_t and B_t must both be host or both device");
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->tick++;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    if (stats) {
        ev0 = take_event(ctx);
        ev1 = take_event(ctx);
        cudaEventRecord(ev0, ctx->stream);
    }
    const double field_ms_before = ctx->ctr.field_ms;
    const uint64_t launches_before = ctx->ctr.launches;
    const bool timing_before = ctx->time_field;
    if (stats) ctx->time_field = true;
    sc_status st;
    // points on the device, once
    const double* d_pts = points_xyz;
    if (!is_device_ptr(points_xyz)) {
        st = check_points_host(ctx, m, points_xyz, n_points);
        if (st != SC_OK) return st;
        if ((st = ensure(ctx, ctx->fpts, (size_t)n_points * 3 * sizeof(double))) != SC_OK) return st;
        SC_CUDA(cudaMemcpyAsync(ctx->fpts.p, points_xyz, (size_t)n_points * 3 * sizeof(double),
                                cudaMemcpyHostToDevice, ctx->stream), "upload points");
        d_pts = (const double*)ctx->fpts.p;
    }
    // time-domain sums on the device
    const size_t out_bytes = (size_t)n_t * n_points * 3 * sizeof(float);
    float* dEt = E_t;
    float* dBt = B_t;
    if (!out_dev) {
        if ((st = ensure(ctx, ctx->ftE, out_bytes)) != SC_OK) return st;
        if (B_t && (st = ensure(ctx, ctx->ftB, out_bytes)) != SC_OK) return st;
        dEt = (float*)ctx->ftE.p;
        dBt = B_t ? (float*)ctx->ftB.p : nullptr;
    }
    // omega chunks: by default as many omegas as keep a chunk's E and B spectra
    // within 32 GiB, rounded down to a power of two (the field kernels' omega
    // classes) when the grid does not fit whole
    const size_t elem = prec == SC_FP64 ? sizeof(double2) : sizeof(float2);
    const size_t per_omega = (size_t)n_points * 3 * elem;
    int chunk = omega_chunk;
    if (chunk <= 0) {
        const size_t fit = std::max<size_t>(1, (size_t(32) << 30) / (2 * per_omega));
        if (fit >= (size_t)n_omega) {
            chunk = n_omega;
        } else {
            chunk = 1;
            while ((size_t)chunk * 2 <= fit) chunk *= 2;
        }
    }
    chunk = std::min(chunk, n_omega);
    if ((st = ensure(ctx, ctx->fspecE, (size_t)chunk * per_omega)) != SC_OK) return st;
    if (B_t && (st = ensure(ctx, ctx->fspecB, (size_t)chunk * per_omega)) != SC_OK) return st;
    const double dk = n_omega > 1 ? 2.0 * kPi * dom : 1.0;
    double evals = 0.0;
    for (int o0 = 0; o0 < n_omega; o0 += chunk) {
        const int c = std::min(chunk, n_omega - o0);
        st = eval_unlocked(ctx, m, in, omegas + o0, c, d_pts, n_points, prec, dom, ctx->fspecE.p,
                           B_t ? ctx->fspecB.p : nullptr, nullptr);
        if (st != SC_OK) return st;
        st = time_domain_unlocked(ctx, prec, ctx->fspecE.p, B_t ? ctx->fspecB.p : nullptr, omegas + o0, c,
                                  n_points, times, n_t, dEt, dBt, dk, o0 > 0);
        if (st != SC_OK) return st;
        for (const auto& t : ctx->tables)
            if (t.mid == m->id && t.iid == in->id) evals += (double)n_points * t.n_surf * c;
    }
    if (!out_dev) {
        SC_CUDA(cudaMemcpyAsync(E_t, dEt, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "download E(t)");
        if (B_t) SC_CUDA(cudaMemcpyAsync(B_t, dBt, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "download B(t)");
    }
    if (stats) cudaEventRecord(ev1, ctx->stream);
    st = check_device_error(ctx);
    if (stats) {
        ctx->time_field = timing_before;
        if (st != SC_OK) return st;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        ctx->pool.push_back(ev0);
        ctx->pool.push_back(ev1);
        settle_events(ctx);
        stats->evals = evals;
        stats->total_ms = ms;
        stats->field_ms = ctx->ctr.field_ms - field_ms_before;
        stats->launches = (int)(ctx->ctr.launches - launches_before);
        stats->tables = 0;
        for (const auto& t : ctx->tables)
            if (t.mid == m->id && t.iid == in->id) stats->tables = (int)t.parts.size();
    }
    return st;
}

sc_status sc_eval_batch(sc_ctx* ctx, const sc_request* reqs, int n_req, sc_eval_stats* stats)
{
    if (!ctx) return SC_ERR_INVALID;
    if (!reqs || n_req < 1) return fail(ctx, SC_ERR_INVALID, "invalid argument");
    std::vector<double> dom(n_req);
    size_t n_om_total = 0;
    for (int r = 0; r < n_req; ++r) {
        const sc_request& q = reqs[r];
        if (!q.mirror || !q.incident || !q.omegas || !q.points_xyz || !q.E_out || q.n_omega < 1 ||
            q.n_points < 1)
            return fail(ctx, SC_ERR_INVALID, "request %d: invalid argument", r);
        for (int i = 0; i < q.n_omega; ++i)
            if (!(q.omegas[i] > 0.0) || !std::isfinite(q.omegas[i]))
                return fail(ctx, SC_ERR_INVALID, "request %d: omega[%d] must be positive", r, i);
        if (!uniform_grid(q.omegas, q.n_omega, dom[r]))
            return fail(ctx, SC_ERR_INVALID, "request %d: needs a uniform, increasing omega grid", r);
        if (!is_device_ptr(q.points_xyz) || !is_device_ptr(q.E_out) ||
            (q.B_out && !is_device_ptr(q.B_out)))
            return fail(ctx, SC_ERR_INVALID, "request %d: points and outputs must be device buffers", r);
        if (!focuses_on_origin(q.mirror, q.incident))
            return fail(ctx, SC_ERR_INVALID, "request %d: the FP32 path needs an incident wavefront focused "
                                             "on the origin", r);
        n_om_total += q.n_omega;
    }
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    ctx->tick++;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    const double field_ms_before = ctx->ctr.field_ms;
    const uint64_t launches_before = ctx->ctr.launches;
    const bool timing_before = ctx->time_field;
    if (stats) {
        ev0 = take_event(ctx);
        ev1 = take_event(ctx);
        cudaEventRecord(ev0, ctx->stream);
        ctx->time_field = true;
    }
    std::vector<Table*> tabs(n_req);
    double evals = 0.0;
    for (int r = 0; r < n_req; ++r) {
        sc_status st = get_table(ctx, reqs[r].mirror, reqs[r].incident, &tabs[r], ctx->main.stream);
        if (st != SC_OK) return st;
        evals += (double)reqs[r].n_points * tabs[r]->n_surf * reqs[r].n_omega;
    }
    // per-part spectra and wavenumbers of all requests, one upload
    std::vector<double> amp_all, k_all(n_om_total);
    std::vector<size_t> amp_off(n_req), om_off(n_req);
    size_t o = 0;
    for (int r = 0; r < n_req; ++r) {
        std::vector<double> a;
        sc_status st = request_amps(ctx, reqs[r].incident, tabs[r], reqs[r].omegas, reqs[r].n_omega, a);
        if (st != SC_OK) return st;
        amp_off[r] = amp_all.size();
        om_off[r] = o;
        amp_all.insert(amp_all.end(), a.begin(), a.end());
        for (int i = 0; i < reqs[r].n_omega; ++i) k_all[o + i] = 2.0 * kPi * reqs[r].omegas[i];
        o += reqs[r].n_omega;
    }
    sc_status st;
    Lane& ln = ctx->main;
    if ((st = ensure(ctx, ln.amp, amp_all.size() * sizeof(double))) != SC_OK) return st;
    if ((st = ensure(ctx, ln.kval, k_all.size() * sizeof(double))) != SC_OK) return st;
    SC_CUDA(cudaMemcpyAsync(ln.amp.p, amp_all.data(), amp_all.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ln.stream), "upload amplitudes");
    SC_CUDA(cudaMemcpyAsync(ln.kval.p, k_all.data(), k_all.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ln.stream), "upload wavenumbers");
    std::vector<Chunk> ch;
    for (int r = 0; r < n_req; ++r) {
        const sc_request& q = reqs[r];
        st = plan_request(ctx, ln, tabs[r], q.omegas, q.n_omega, dom[r], q.points_xyz, q.n_points,
                          (const double*)ln.amp.p + amp_off[r], (const double*)ln.kval.p + om_off[r],
                          (float2*)q.E_out, (float2*)q.B_out, ch);
        if (st != SC_OK) return st;
    }
    st = run_chunks(ctx, ln, ch);
    if (st != SC_OK) return st;
    ctx->ctr.evals += evals;
    if (stats) {
        cudaEventRecord(ev1, ctx->stream);
        st = check_device_error(ctx);
        ctx->time_field = timing_before;
        if (st != SC_OK) return st;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, ev0, ev1);
        ctx->pool.push_back(ev0);
        ctx->pool.push_back(ev1);
        settle_events(ctx);
        stats->evals = evals;
        stats->total_ms = ms;
        stats->field_ms = ctx->ctr.field_ms - field_ms_before;
        stats->launches = (int)(ctx->ctr.launches - launches_before);
        stats->tables = 0;
        for (const Table* t : tabs) stats->tables = std::max(stats->tables, (int)t->parts.size());
    }
    return SC_OK;
}

sc_status sc_eval_fp32_static(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in,
                              double omega0, double domega, int n_omega, const double* amp_re_im,
                              const double* points_xyz, int n_points, void* E_out, void* B_out)
{
    // No device allocation on this path: the table must already be resident,
    // a_n and k_n travel through the static scratch, and so do the partials.
    constexpr int kMaxOmega = 2048;
    if (!ctx) return SC_ERR_INVALID;
    if (!m || !in || !amp_re_im || !points_xyz || !E_out || n_points < 1 || n_omega < 1)
        return fail(ctx, SC_ERR_INVALID, "invalid argument");
    if (n_omega > kMaxOmega)
        return fail(ctx, SC_ERR_INVALID, "n_omega %d exceeds %d for the static-scratch path", n_omega,
                    kMaxOmega);
    if (!(omega0 > 0.0) || !(domega >= 0.0) || (n_omega > 1 && !(domega > 0.0)))
        return fail(ctx, SC_ERR_INVALID, "omega grid must be positive and increasing");
    const size_t header = (size_t)n_omega * 3 * sizeof(double);   // a_n (2) and k_n (1)
    const size_t header_al = (header + 255) / 256 * 256;
    const size_t ws_bytes = (size_t)2 * n_points * n_omega * sc::kAcc * sizeof(float2);
    if (header_al + ws_bytes > sc::kStaticScratchBytes)
        return fail(ctx, SC_ERR_INVALID,
                    "request needs %zu bytes of static scratch; the limit is %zu (points x omegas "
                    "<= %zu)", header_al + ws_bytes, sc::kStaticScratchBytes,
                    (sc::kStaticScratchBytes - header_al) / (2 * sc::kAcc * sizeof(float2)));
    std::lock_guard<std::mutex> lock(ctx->mu);
    Table* tab = nullptr;
    for (auto& t : ctx->tables)
        if (t.mid == m->id && t.iid == in->id) tab = &t;
    if (!tab)
        return fail(ctx, SC_ERR_INVALID,
                    "node table not resident: run sc_eval once for this mirror and incident first");
    if (tab->parts.size() > 1)
        return fail(ctx, SC_ERR_INVALID, "a beam with %zu node tables needs sc_eval", tab->parts.size());
    if (!tab->fp32_ok)
        return fail(ctx, SC_ERR_INVALID, "this mirror and beam need the FP64 path of sc_eval");
    ctx->tick++;
    void* scratch = nullptr;
    cudaError_t e = sc::static_scratch(ctx->device, &scratch);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "static scratch address");
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    double hdr[3 * kMaxOmega];
    for (int i = 0; i < n_omega; ++i) {
        hdr[2 * i] = amp_re_im[2 * i];
        hdr[2 * i + 1] = amp_re_im[2 * i + 1];
        hdr[2 * n_omega + i] = 2.0 * kPi * (omega0 + i * domega);
    }
    double* d_amp = (double*)scratch;
    double* d_k = d_amp + 2 * (size_t)n_omega;
    // pageable source: the call returns once the bytes are staged
    SC_CUDA(cudaMemcpyAsync(d_amp, hdr, header, cudaMemcpyHostToDevice, ctx->stream),
            "upload a_n, k_n");
    float2* ws = (float2*)((unsigned char*)scratch + header_al);
    sc::FieldLaunch f;
    f.nodes = tab->d32;
    f.n_surf_tiles = tab->n_surf_tiles;
    f.n_rim_tiles = tab->n_rim_tiles;
    f.tiles_per_split = tab->n_surf_tiles;  // one surface split and the rim slot
    f.n_splits = 1;
    f.flush_tiles = (int)std::max<long long>(1, ctx->flush_nodes / sc::kTile);
    f.pts = points_xyz;
    f.n_pts = n_points;
    f.n_omega = n_omega;
    f.om_hi0 = (float)omega0;
    f.om_lo0 = (float)(omega0 - (double)f.om_hi0);
    f.dom_hi = (float)domega;
    f.dom_lo = (float)(domega - (double)f.dom_hi);
    f.ws = ws;
    f.err = ctx->d_err;
    int r = sc::launch_field_f32(f, ctx->stream);
    if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "field kernel launch");
    ctx->ctr.launches += r;
    ctx->ctr.field_launches += 1;
    sc::ReduceLaunch rl;
    rl.ws = ws;
    rl.n_splits = 1;
    rl.n_pts = n_points;
    rl.n_omega = n_omega;
    rl.amp = d_amp;
    rl.kval = d_k;
    rl.out_pt_stride_omega = (long long)n_points * 3;
    rl.E = (float2*)E_out;
    rl.B = (float2*)B_out;
    r = sc::launch_reduce_f32(rl, ctx->stream);
    if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "reduce kernel launch");
    ctx->ctr.launches += r;
    ctx->ctr.evals += (double)n_points * tab->n_surf * n_omega;
    return SC_OK;
}

// sc_time_domain after validation, with ctx->mu held and the device set: dk
// is the step of the full uniform grid (the omegas may be one chunk of it);
// accumulate adds to E_t, B_t (device outputs only) instead of storing.
static sc_status time_domain_unlocked(sc_ctx* ctx, sc_precision prec, const void* E_spec,
                                      const void* B_spec, const double* omegas, int n_omega,
                                      int n_points, const double* times, int n_t, float* E_t,
                                      float* B_t, double dk, int accumulate)
{
    const size_t elem = prec == SC_FP64 ? sizeof(double2) : sizeof(float2);
    const long long n_vals = (long long)n_points * 3;
    const size_t spec_bytes = (size_t)n_omega * n_vals * elem;
    const size_t out_bytes = (size_t)n_t * n_vals * sizeof(float);
    const bool in_dev = is_device_ptr(E_spec);
    const bool out_dev = is_device_ptr(E_t);
    if (accumulate && !out_dev) return fail(ctx, SC_ERR_INVALID, "accumulation needs device outputs");
    sc_status st;
    std::vector<double> kv(n_omega);
    for (int i = 0; i < n_omega; ++i) kv[i] = 2.0 * kPi * omegas[i];
    if ((st = ensure(ctx, ctx->tkval, kv.size() * sizeof(double))) != SC_OK) return st;
    if ((st = ensure(ctx, ctx->tvals, (size_t)n_t * sizeof(double))) != SC_OK) return st;
    if ((st = ensure(ctx, ctx->phasor, (size_t)n_omega * n_t * sizeof(float2))) != SC_OK) return st;
    const void* dEs = E_spec;
    const void* dBs = B_spec;
    if (!in_dev) {
        if ((st = ensure(ctx, ctx->specE, spec_bytes)) != SC_OK) return st;
        if (B_spec && (st = ensure(ctx, ctx->specB, spec_bytes)) != SC_OK) return st;
        SC_CUDA(cudaMemcpyAsync(ctx->specE.p, E_spec, spec_bytes, cudaMemcpyHostToDevice, ctx->stream), "upload E spectrum");
        if (B_spec)
            SC_CUDA(cudaMemcpyAsync(ctx->specB.p, B_spec, spec_bytes, cudaMemcpyHostToDevice, ctx->stream), "upload B spectrum");
        dEs = ctx->specE.p;
        dBs = B_spec ? ctx->specB.p : nullptr;
    }
    float* dEt = E_t;
    float* dBt = B_t;
    if (!out_dev) {
        if ((st = ensure(ctx, ctx->tE, out_bytes)) != SC_OK) return st;
        if (B_t && (st = ensure(ctx, ctx->tB, out_bytes)) != SC_OK) return st;
        dEt = (float*)ctx->tE.p;
        dBt = B_t ? (float*)ctx->tB.p : nullptr;
    }
    SC_CUDA(cudaMemcpyAsync(ctx->tkval.p, kv.data(), kv.size() * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload wavenumbers");
    SC_CUDA(cudaMemcpyAsync(ctx->tvals.p, times, (size_t)n_t * sizeof(double), cudaMemcpyHostToDevice, ctx->stream), "upload times");
    for (int pass = 0; pass < (B_spec ? 2 : 1); ++pass) {
        sc::IdftLaunch l;
        l.F = pass == 0 ? dEs : dBs;
        l.f64 = prec == SC_FP64;
        l.n_omega = n_omega;
        l.n_vals = n_vals;
        l.kval = (const double*)ctx->tkval.p;
        l.t = (const double*)ctx->tvals.p;
        l.n_t = n_t;
        l.dk = dk;
        l.out = pass == 0 ? dEt : dBt;
        l.phasor = (float2*)ctx->phasor.p;
        l.accumulate = accumulate;
        const int r = sc::launch_idft(l, ctx->stream);
        if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "inverse transform launch");
        ctx->ctr.launches += r;
    }
    if (!out_dev) {
        SC_CUDA(cudaMemcpyAsync(E_t, dEt, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "download E(t)");
        if (B_t) SC_CUDA(cudaMemcpyAsync(B_t, dBt, out_bytes, cudaMemcpyDeviceToHost, ctx->stream), "download B(t)");
        SC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    }
    return SC_OK;
}

sc_status sc_time_domain(sc_ctx* ctx, sc_precision prec, const void* E_spec, const void* B_spec,
                         const double* omegas, int n_omega, int n_points, const double* times,
                         int n_t, float* E_t, float* B_t)
{
    if (!ctx) return SC_ERR_INVALID;
    if (!E_spec || !E_t || !omegas || !times || n_omega < 1 || n_points < 1 || n_t < 1 ||
        (B_spec == nullptr) != (B_t == nullptr))
        return fail(ctx, SC_ERR_INVALID, "invalid argument");
    double dom = 0.0;
    if (!uniform_grid(omegas, n_omega, dom))
        return fail(ctx, SC_ERR_INVALID, "the inverse transform needs a uniform omega grid");
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const double dk = n_omega > 1 ? 2.0 * kPi * dom : 1.0;
    return time_domain_unlocked(ctx, prec, E_spec, B_spec, omegas, n_omega, n_points, times, n_t, E_t, B_t,
                                dk, 0);
}

sc_status sc_submit(sc_ctx* ctx, const sc_request* req, uint64_t* ticket)
{
    if (!ctx) return SC_ERR_INVALID;
    if (!req || !ticket || !req->mirror || !req->incident || !req->omegas || !req->points_xyz ||
        req->n_omega < 1 || req->n_points < 1 || req->n_omega > 2048 * 64)
        return fail(ctx, SC_ERR_INVALID, "invalid request");
    double dom = 0.0;
    for (int i = 0; i < req->n_omega; ++i)
        if (!(req->omegas[i] > 0.0) || !std::isfinite(req->omegas[i]))
            return fail(ctx, SC_ERR_INVALID, "omega[%d] must be positive", i);
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!uniform_grid(req->omegas, req->n_omega, dom))
        return fail(ctx, SC_ERR_INVALID, "serving needs a uniform, increasing omega grid");
    if (!focuses_on_origin(req->mirror, req->incident))
        return fail(ctx, SC_ERR_INVALID, "serving runs the FP32 path, whose compensated phase needs an "
                                         "incident wavefront focused on the origin");
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    Ticket t;
    t.mirror = req->mirror;
    t.incident = req->incident;
    t.omegas.assign(req->omegas, req->omegas + req->n_omega);
    t.n_points = req->n_points;
    t.n_omega = req->n_omega;
    t.dom = dom;
    if (is_device_ptr(req->points_xyz)) {
        t.user_pts = req->points_xyz;
    } else {
        sc_status st = check_points_host(ctx, req->mirror, req->points_xyz, req->n_points);
        if (st != SC_OK) return st;
        t.host_pts.assign(req->points_xyz, req->points_xyz + 3 * (size_t)req->n_points);
        t.own_pts = true;
    }
    if (req->E_out) {
        if (!is_device_ptr(req->E_out) || (req->B_out && !is_device_ptr(req->B_out)))
            return fail(ctx, SC_ERR_INVALID, "caller-owned serving outputs must be device buffers");
        t.E_user = req->E_out;
        t.B_user = req->B_out;
    } else {
        t.own_out = true;
    }
    const size_t b = ticket_bytes(t);
    if (ctx->budget && b > ctx->budget)
        return fail(ctx, SC_ERR_BUSY, "request needs %zu device bytes, more than the whole budget %zu", b,
                    ctx->budget);
    sc_status st = start_server(ctx);
    if (st != SC_OK) return st;
    Server* srv = ctx->server;
    t.t_submit = srv->now();
    const uint64_t id = srv->next_id++;
    srv->tickets.emplace(id, std::move(t));
    srv->queue.push_back(id);
    *ticket = id;
    srv->cv.notify_all();
    return SC_OK;
}

sc_status sc_poll(sc_ctx* ctx, uint64_t ticket, int* done)
{
    if (!ctx || !done) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->server) return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    auto it = ctx->server->tickets.find(ticket);
    if (it == ctx->server->tickets.end())
        return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    const Ticket& t = it->second;
    *done = t.state >= 2;
    if (t.state == 3) return fail(ctx, t.status, "request failed");
    if (t.state == 4) return fail(ctx, SC_ERR_CANCELLED, "request cancelled");
    return SC_OK;
}

sc_status sc_wait(sc_ctx* ctx, uint64_t ticket, double timeout_s)
{
    if (!ctx) return SC_ERR_INVALID;
    std::unique_lock<std::mutex> lk(ctx->mu);
    if (!ctx->server) return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Server* srv = ctx->server;
    const auto deadline = std::chrono::steady_clock::now() +
                          std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                              std::chrono::duration<double>(timeout_s));
    for (;;) {
        auto it = srv->tickets.find(ticket);
        if (it == srv->tickets.end())
            return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
        const Ticket& t = it->second;
        if (t.state == 2) return SC_OK;
        if (t.state == 3) return fail(ctx, t.status, "request failed");
        if (t.state == 4) return fail(ctx, SC_ERR_CANCELLED, "request cancelled");
        if (srv->cv.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto jt = srv->tickets.find(ticket);
            if (jt != srv->tickets.end() && jt->second.state == 2) return SC_OK;
            return fail(ctx, SC_ERR_TIMEOUT, "request %llu not done after %.3f s",
                        (unsigned long long)ticket, timeout_s);
        }
    }
}

sc_status sc_cancel(sc_ctx* ctx, uint64_t ticket)
{
    if (!ctx) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->server) return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Server* srv = ctx->server;
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end())
        return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Ticket& t = it->second;
    if (t.state == 0) {
        srv->queue.erase(std::find(srv->queue.begin(), srv->queue.end(), ticket));
        t.state = 4;
        t.t_done = srv->now();
    } else if (t.state == 1) {
        t.cancel = true;  // its batch finishes; the result is discarded
    }
    srv->cv.notify_all();
    return SC_OK;
}

sc_status sc_fetch(sc_ctx* ctx, uint64_t ticket, void* E_dst, void* B_dst)
{
    if (!ctx) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->server) return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Server* srv = ctx->server;
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end())
        return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Ticket& t = it->second;
    if (t.state != 2) return fail(ctx, SC_ERR_BUSY, "request %llu is not done", (unsigned long long)ticket);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const size_t ob = (size_t)t.n_omega * t.n_points * 3 * sizeof(float2);
    cudaStream_t s = srv->lanes[t.lane].stream;
    if (E_dst) SC_CUDA(cudaMemcpyAsync(E_dst, t.E, ob, cudaMemcpyDefault, s), "fetch E");
    if (B_dst && t.B) SC_CUDA(cudaMemcpyAsync(B_dst, t.B, ob, cudaMemcpyDefault, s), "fetch B");
    SC_CUDA(cudaStreamSynchronize(s), "fetch");
    return SC_OK;
}

sc_status sc_release(sc_ctx* ctx, uint64_t ticket)
{
    if (!ctx) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->server) return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    Server* srv = ctx->server;
    auto it = srv->tickets.find(ticket);
    if (it == srv->tickets.end())
        return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (it->second.state == 1) return fail(ctx, SC_ERR_BUSY, "request %llu is still running", (unsigned long long)ticket);
    if (it->second.state == 0) srv->queue.erase(std::find(srv->queue.begin(), srv->queue.end(), ticket));
    cudaSetDevice(ctx->device);
    free_ticket_memory(srv, it->second);
    srv->tickets.erase(it);
    srv->cv.notify_all();
    return SC_OK;
}

sc_status sc_ticket_times(sc_ctx* ctx, uint64_t ticket, double* t_submit, double* t_start, double* t_done)
{
    if (!ctx) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    if (!ctx->server) return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    auto it = ctx->server->tickets.find(ticket);
    if (it == ctx->server->tickets.end())
        return fail(ctx, SC_ERR_NOT_FOUND, "unknown ticket %llu", (unsigned long long)ticket);
    if (t_submit) *t_submit = it->second.t_submit;
    if (t_start) *t_start = it->second.t_start;
    if (t_done) *t_done = it->second.t_done;
    return SC_OK;
}

sc_status sc_selftest_wait(sc_ctx* ctx)
{
    if (!ctx) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int r = sc::launch_wait_selftest(ctx->d_err, ctx->stream);
    if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "self-test launch");
    return check_device_error(ctx);
}

sc_status sc_measure_alu_peaks(sc_ctx* ctx, double* fp32_lane_ops_per_s, double* fp32x2_lane_ops_per_s,
                               double* mufu_ops_per_s)
{
    if (!ctx || !fp32_lane_ops_per_s || !fp32x2_lane_ops_per_s || !mufu_ops_per_s)
        return fail(ctx, SC_ERR_INVALID, "null argument");
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    const int iters[3] = {16384, 8192, 2048};
    double* outs[3] = {fp32_lane_ops_per_s, fp32x2_lane_ops_per_s, mufu_ops_per_s};
    int grids[3];
    int max_grid = 1;
    for (int k = 0; k < 3; ++k) max_grid = std::max(max_grid, grids[k] = sc::alu_probe_grid(k, ctx->device));
    float* sink = nullptr;
    SC_CUDA(cudaMallocAsync((void**)&sink, (size_t)max_grid * 512 * sizeof(float), ctx->stream), "probe sink");
    cudaEvent_t e0 = take_event(ctx), e1 = take_event(ctx);
    sc_status st = SC_OK;
    for (int k = 0; k < 3 && st == SC_OK; ++k) {
        float best = 0.f;
        for (int rep = 0; rep < 4 && st == SC_OK; ++rep) {  // the first launch warms up
            cudaEventRecord(e0, ctx->stream);
            const int r = sc::launch_alu_probe(k, iters[k], sink, grids[k], 512, ctx->stream);
            cudaEventRecord(e1, ctx->stream);
            if (r < 0) {
                st = cuda_fail(ctx, (cudaError_t)(-r), "ALU probe launch");
                break;
            }
            ctx->ctr.launches++;
            const cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) {
                st = cuda_fail(ctx, e, "ALU probe");
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && (best == 0.f || ms < best)) best = ms;
        }
        const double ops = (double)grids[k] * 512.0 * (double)sc::alu_probe_ops_per_thread(iters[k]);
        *outs[k] = best > 0.f ? ops / (1e-3 * best) : 0.0;
    }
    cudaFreeAsync(sink, ctx->stream);
    ctx->pool.push_back(e0);
    ctx->pool.push_back(e1);
    if (st != SC_OK) return st;
    SC_CUDA(cudaStreamSynchronize(ctx->stream), "ALU probes");
    return SC_OK;
}

sc_status sc_get_counters(sc_ctx* ctx, sc_counters* out)
{
    if (!ctx || !out) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    sc_status st = check_device_error(ctx);
    settle_events(ctx);
    *out = ctx->ctr;
    out->graph_captures = ctx->graph_captures;
    out->graph_replays = ctx->graph_replays;
    return st;
}

sc_status sc_reset_counters(sc_ctx* ctx)
{
    if (!ctx) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    SC_CUDA(cudaSetDevice(ctx->device), "cudaSetDevice");
    SC_CUDA(cudaStreamSynchronize(ctx->stream), "stream synchronize");
    settle_events(ctx);
    ctx->ctr = sc_counters{};
    return SC_OK;
}

sc_status sc_set_option(sc_ctx* ctx, int option, long long value)
{
    if (!ctx) return SC_ERR_INVALID;
    std::lock_guard<std::mutex> lock(ctx->mu);
    switch (option) {
    case SC_OPT_TIME_FIELD: ctx->time_field = value != 0; return SC_OK;
    case SC_OPT_NODES_PER_SPLIT:
        if (value != 0 && (value < sc::kTile || value % sc::kTile))
            return fail(ctx, SC_ERR_INVALID, "nodes per split must be a positive multiple of %d", sc::kTile);
        ctx->nodes_per_split = value;
        return SC_OK;
    case SC_OPT_FLUSH_NODES:
        if (value < sc::kTile || value % sc::kTile)
            return fail(ctx, SC_ERR_INVALID, "flush length must be a positive multiple of %d", sc::kTile);
        ctx->flush_nodes = value;
        return SC_OK;
    case SC_OPT_GRAPHS: ctx->use_graphs = value != 0; return SC_OK;
    case SC_OPT_AUTOTUNE: ctx->autotune = value != 0; return SC_OK;
    case SC_OPT_WORKSPACE_CAP:
        if (value < (1 << 20)) return fail(ctx, SC_ERR_INVALID, "workspace cap below 1 MiB");
        ctx->ws_cap = (size_t)value;
        return SC_OK;
    default: return fail(ctx, SC_ERR_INVALID, "unknown option %d", option);
    }
}

}  // extern "C"
