// sc_api.cpp -- the C-ABI entry points declared in include/sc.h, and the
// error and device-memory helpers of the host side.  The node tables, the
// batched execution and the serving loop live in sc_tables.cpp, sc_batch.cpp
// and sc_serve.cpp (shared declarations in sc_host.h).  Every GPU step is a
// kernel of this library (sc_field.cu, sc_reduce.cu, sc_f64_idft.cu);
// nothing here computes a field value on the CPU.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>

#include "sc_host.h"

using namespace sch;

namespace {

static_assert(SC_STATIC_SCRATCH_BYTES == sc::kStaticScratchBytes, "scratch size mismatch");

std::atomic<uint64_t> g_next_id{1};

}  // namespace

namespace sch {

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

}  // namespace sch

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
        if (ctx->h_err) cudaFreeHost(ctx->h_err);
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
                      &ctx->fspecB, &ctx->ftE, &ctx->ftB, &ctx->mfie_geo, &ctx->mfie_zern, &ctx->mfie_gl,
                      &ctx->mfie_dJ})
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

namespace {

// n_r >= 1 Gauss-Legendre nodes, or an odd n_r >= 3 for composite Simpson
bool quadrature_ok(const sc_quadrature* q)
{
    if (q->n_r < 1 || q->n_theta < 1) return false;
    if (q->radial_kind == SC_QUAD_GAUSS_LEGENDRE) return true;
    return q->radial_kind == SC_QUAD_SIMPSON && q->n_r >= 3 && (q->n_r & 1) == 1;
}

}  // namespace

sc_status sc_mirror(sc_ctx* ctx, double f, double r_min, double r_max, const sc_quadrature* q,
                    sc_mirror_t** out)
{
    if (!out || !q) return fail(ctx, SC_ERR_INVALID, "null argument");
    *out = nullptr;
    if (!(f > 0.0) || !(r_min >= 0.0) || !(r_max > r_min) || !quadrature_ok(q))
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
        !quadrature_ok(q))
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
// The tile shape a call chose (kernel class, its layout, node splits), or -1s.
static void fill_shape(sc_eval_stats* st, int cls, int splits)
{
    st->kernel_class = cls;
    st->splits = splits;
    if (cls >= 0) {
        sc::class_layout(cls, &st->threads_per_point, &st->omegas_per_thread);
    } else {
        st->threads_per_point = -1;
        st->omegas_per_thread = -1;
    }
}

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

    if (ctx->mfie_order > 0)
        if (const char* why = mfie_unsupported(m, in)) return fail(ctx, SC_ERR_INVALID, "%s", why);
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
    int shape_cls = -1, shape_splits = -1;  // reported in stats (FP32 path)

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
        if (!ch.empty()) {
            ctx->shape_cls = shape_cls = ch[0].cls;
            ctx->shape_splits = shape_splits = ch[0].f.n_splits;
        }
        st = run_chunks(ctx, ctx->main, ch);
        if (st != SC_OK) return st;
    }
    ctx->ctr.evals += evals;
    // the first MFIE correction beyond physical optics (Sec. II), added to the outputs
    if (ctx->mfie_order > 0) {
        st = mfie_correction(ctx, m, in, n_omega, d_pts, n_points, d_amp, d_k, dE, dB, prec == SC_FP64);
        if (st != SC_OK) return st;
    }

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
        fill_shape(stats, shape_cls, shape_splits);
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
    int first_cls = -1, first_splits = -1;
    for (int o0 = 0; o0 < n_omega; o0 += chunk) {
        const int c = std::min(chunk, n_omega - o0);
        ctx->shape_cls = ctx->shape_splits = -1;
        st = eval_unlocked(ctx, m, in, omegas + o0, c, d_pts, n_points, prec, dom, ctx->fspecE.p,
                           B_t ? ctx->fspecB.p : nullptr, nullptr);
        if (st != SC_OK) return st;
        if (o0 == 0) {
            first_cls = ctx->shape_cls;
            first_splits = ctx->shape_splits;
        }
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
        fill_shape(stats, first_cls, first_splits);
    }
    return st;
}

sc_status sc_eval_batch(sc_ctx* ctx, const sc_request* reqs, int n_req, sc_eval_stats* stats)
{
    if (!ctx) return SC_ERR_INVALID;
    if (!reqs || n_req < 1) return fail(ctx, SC_ERR_INVALID, "invalid argument");
    if (ctx->mfie_order > 0)
        return fail(ctx, SC_ERR_INVALID, "the MFIE correction runs through sc_eval and sc_eval_time_domain only");
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
    int first_cls = -1, first_splits = -1;
    for (int r = 0; r < n_req; ++r) {
        const sc_request& q = reqs[r];
        st = plan_request(ctx, ln, tabs[r], q.omegas, q.n_omega, dom[r], q.points_xyz, q.n_points,
                          (const double*)ln.amp.p + amp_off[r], (const double*)ln.kval.p + om_off[r],
                          (float2*)q.E_out, (float2*)q.B_out, ch);
        if (st != SC_OK) return st;
        if (r == 0 && !ch.empty()) {
            first_cls = ch[0].cls;
            first_splits = ch[0].f.n_splits;
        }
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
        fill_shape(stats, first_cls, first_splits);
    }
    return SC_OK;
}

sc_status sc_eval_fp32_static(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in,
                              double omega0, double domega, int n_omega, const double* amp_re_im,
                              const double* points_xyz, int n_points, void* E_out, void* B_out)
{
    // No device allocation and no host-to-device copy on this path: the table
    // must already be resident, a_n is the caller's device array, and k_n and
    // the split partials live in the static scratch.
    constexpr int kMaxOmega = 2048;
    if (!ctx) return SC_ERR_INVALID;
    if (!m || !in || !amp_re_im || !points_xyz || !E_out || n_points < 1 || n_omega < 1)
        return fail(ctx, SC_ERR_INVALID, "invalid argument");
    if (!is_device_ptr(amp_re_im) || !is_device_ptr(points_xyz) || !is_device_ptr(E_out) ||
        (B_out && !is_device_ptr(B_out)))
        return fail(ctx, SC_ERR_INVALID,
                    "amp_re_im, points_xyz, E_out and B_out must be device memory on this path");
    if (ctx->mfie_order > 0)
        return fail(ctx, SC_ERR_INVALID, "the MFIE correction runs through sc_eval and sc_eval_time_domain only");
    if (n_omega > kMaxOmega)
        return fail(ctx, SC_ERR_INVALID, "n_omega %d exceeds %d for the static-scratch path", n_omega,
                    kMaxOmega);
    if (!(omega0 > 0.0) || !(domega >= 0.0) || (n_omega > 1 && !(domega > 0.0)))
        return fail(ctx, SC_ERR_INVALID, "omega grid must be positive and increasing");
    const size_t header = (size_t)n_omega * sizeof(double);   // k_n
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
    double* d_k = (double*)scratch;
    int r = sc::launch_kgrid(d_k, omega0, domega, n_omega, ctx->stream);
    if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "k grid kernel launch");
    ctx->ctr.launches += r;
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
    r = sc::launch_field_f32(f, ctx->stream);
    if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "field kernel launch");
    ctx->ctr.launches += r;
    ctx->ctr.field_launches += 1;
    sc::ReduceLaunch rl;
    rl.ws = ws;
    rl.n_splits = 1;
    rl.n_pts = n_points;
    rl.n_omega = n_omega;
    rl.amp = amp_re_im;
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
    if (ctx->mfie_order > 0)
        return fail(ctx, SC_ERR_INVALID, "the MFIE correction runs through sc_eval and sc_eval_time_domain only");
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
    t.evals = (double)req->n_points * req->mirror->q.n_r * req->mirror->q.n_theta * req->n_omega;
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
    if (option == SC_OPT_SERVE_PRIORITY) {
        // the lanes are set up when the server starts: stop an idle server
        // (the next sc_submit starts it again with the new policy)
        {
            std::lock_guard<std::mutex> lock(ctx->mu);
            if (ctx->server && !ctx->server->tickets.empty())
                return fail(ctx, SC_ERR_BUSY, "serving policy: release every ticket first");
        }
        sch::stop_server(ctx);
        std::lock_guard<std::mutex> lock(ctx->mu);
        ctx->serve_priority = value != 0;
        return SC_OK;
    }
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
    case SC_OPT_OMEGA_CHUNKS: ctx->omega_chunks = value != 0; return SC_OK;
    case SC_OPT_CLASS_STREAMS: ctx->class_streams = value != 0; return SC_OK;
    case SC_OPT_TILE_LAYOUT:
        if (value < -1 || value > 1) return fail(ctx, SC_ERR_INVALID, "tile layout must be -1, 0 or 1");
        ctx->tile_layout = (int)value;
        return SC_OK;
    case SC_OPT_WORKSPACE_CAP:
        if (value < (1 << 20)) return fail(ctx, SC_ERR_INVALID, "workspace cap below 1 MiB");
        ctx->ws_cap = (size_t)value;
        return SC_OK;
    case SC_OPT_MFIE_ORDER:
        if (value < 0 || value > 1) return fail(ctx, SC_ERR_INVALID, "MFIE order must be 0 or 1");
        ctx->mfie_order = (int)value;
        return SC_OK;
    case SC_OPT_MFIE_RHO:
    case SC_OPT_MFIE_PHI:
        if (value < 1 || value > 65536) return fail(ctx, SC_ERR_INVALID, "polar rule size out of range");
        (option == SC_OPT_MFIE_RHO ? ctx->mfie_rho : ctx->mfie_phi) = (int)value;
        return SC_OK;
    case SC_OPT_FAIL_COPY:
        if (value < -1 || value > (1 << 30)) return fail(ctx, SC_ERR_INVALID, "tile index out of range");
        ctx->fail_tile = (int)value;
        return SC_OK;
    default: return fail(ctx, SC_ERR_INVALID, "unknown option %d", option);
    }
}

}  // extern "C"
