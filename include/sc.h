/*
 * sc.h -- C-ABI of libsc, the GB300 (sm_103a) evaluator of the
 * physical-optics Stratton-Chu focal field of a parabolic mirror
 * (Dumont et al., arXiv:1609.08146).
 *
 * What it computes.  For every frequency omega_n of an incident pulse and
 * every observation point r' near the focus, the reflected field of
 * Sec. II, Eq. 11 (physical-optics surface currents after Stokes' theorem):
 *
 *   E'(r', k) = 2 SS { ik (n x B_inc) g + (n . E_inc) grad g } dS
 *               - (2/ik) O grad g [n x (n x B_inc)] . dl
 *   B'(r', k) = 2 SS (n x B_inc) x grad g dS,   g = e^{ikR} / (4 pi R)
 *
 * discretised by tensor-product quadrature on the mirror (Sec. III.C.1),
 * followed on request by the semi-discrete inverse transform of Sec. III.B,
 * Eq. 13.  The mirror is the paraboloid z = r^2/(4f) - f of Eq. 21 with its
 * focus at the origin; the incident beam travels along -z (Sec. III.A).
 *
 * Units: lengths in lambda0 (the reference wavelength), c = 1, angular
 * frequencies omega in units of omega0 = 2 pi c / lambda0, so the
 * wavenumber is k = 2 pi omega; times in lambda0 / c.
 *
 * Conventions shared by every call:
 *  - Status codes only: no call aborts, prints or throws.  On failure the
 *    context keeps a message readable with sc_last_error().
 *  - Every GPU step runs in this library's own CUDA kernels on the stream
 *    given to sc_create(); there is no CPU fallback.  A call that takes
 *    device buffers is asynchronous on that stream unless it says otherwise.
 *  - Pointers marked "host or device" are classified with
 *    cudaPointerGetAttributes; host buffers are staged through device memory
 *    owned by the context and the call then returns after its results are
 *    back in host memory.
 *  - The library owns every handle and every device table it creates; the
 *    caller owns every input and output buffer it passes.
 *  - Complex arrays are interleaved (re, im).
 */
#ifndef SC_H
#define SC_H

#include <stddef.h>
#include <stdint.h>

/* The library is built with hidden symbols; everything declared here is its
 * exported interface. */
#if defined(__GNUC__) && !defined(__CUDA_ARCH__)
#pragma GCC visibility push(default)
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SC_OK = 0,
    SC_ERR_INVALID = 1,   /* bad argument or geometry                        */
    SC_ERR_OOM = 2,       /* device allocation failed or budget exceeded     */
    SC_ERR_CUDA = 3,      /* a CUDA runtime call failed                      */
    SC_ERR_TIMEOUT = 4,   /* a bounded device wait ran out                   */
    SC_ERR_BUSY = 5,      /* request can never be admitted                   */
    SC_ERR_CANCELLED = 6, /* request cancelled before completion             */
    SC_ERR_NOT_FOUND = 7  /* unknown ticket                                  */
} sc_status;

typedef struct sc_ctx sc_ctx;
typedef struct sc_mirror_t sc_mirror_t;
typedef struct sc_incident_t sc_incident_t;

/* ---------------------------------------------------------------------- */
/* Context                                                                 */

/*
 * Create a context bound to CUDA device `device` and stream `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `hbm_budget_bytes`
 * caps the device memory the context itself holds (node tables, workspace,
 * staging); 0 means "no cap beyond what cudaMalloc grants".
 * Errors: SC_ERR_INVALID (null out, bad device), SC_ERR_CUDA.
 */
sc_status sc_create(int device, void* cuda_stream, size_t hbm_budget_bytes, sc_ctx** out);

/* Release every device buffer and handle cache of the context.  Waits for
 * the context's stream.  NULL is accepted. */
sc_status sc_destroy(sc_ctx* ctx);

/* Message of the most recent failing call on this context (owned by the
 * context, valid until its next call).  Never NULL. */
const char* sc_last_error(const sc_ctx* ctx);

/* ---------------------------------------------------------------------- */
/* Mirror (Sec. III.A; Sec. III.C.1, Eq. 21 and the quadrature it names)    */

/*
 * Radial rule on [r_min, r_max] (Sec. III.C.1 names "Simpson or
 * Gauss-Legendre"; the angular rule is always the periodic trapezoid):
 *   SC_QUAD_GAUSS_LEGENDRE  n_r >= 1 Gauss-Legendre nodes (exact for
 *                           polynomials of degree 2 n_r - 1);
 *   SC_QUAD_SIMPSON         composite Simpson, n_r odd >= 3 equally spaced
 *                           nodes r_i = r_min + i h, h = (r_max - r_min) /
 *                           (n_r - 1), both ends included, weights h/3 (1, 4,
 *                           2, 4, ..., 2, 4, 1) (exact for cubics, error
 *                           O(h^4)).  A node at r = 0 carries zero weight.
 */
enum { SC_QUAD_GAUSS_LEGENDRE = 0, SC_QUAD_SIMPSON = 1 };

typedef struct {
    int radial_kind; /* SC_QUAD_GAUSS_LEGENDRE or SC_QUAD_SIMPSON (above)             */
    int n_r;         /* >= 1 (Gauss-Legendre), odd >= 3 (Simpson)                     */
    int n_theta;     /* >= 1, periodic trapezoid theta_l = 2 pi l / n_theta           */
    int rim_term;    /* 1: include the boundary line integral of Eq. 11 (outer rim,   */
                     /*    and the inner rim when r_min > 0)                          */
} sc_quadrature;

/*
 * Describe the paraboloid z = r^2/(4f) - f (focus at the origin) cut to
 * r_min <= r <= r_max, and the quadrature used on it.
 * Errors: SC_ERR_INVALID when f <= 0, r_min < 0, r_min >= r_max, n_r < 1,
 * n_theta < 1, an unknown radial_kind, or SC_QUAD_SIMPSON with an even n_r
 * or n_r < 3.  The handle is host-side only;
 * device tables are built lazily per (mirror, incident) pair by sc_eval.
 */
/*
 * Ellipsoidal mirror (beyond paraboloids; Sec. III.C names the ellipsoid as
 * a mirror where the paraboloid's phase cancellation fails): the lower cap
 * z = e - c sqrt(1 - r^2/a^2), a^2 = c^2 - e^2, of the ellipsoid of
 * revolution with semi-axis c along z and focal half-distance e, cut to
 * r_min <= r <= r_max < a.  Its lower focus F2 is the origin, its upper
 * focus F1 = (0, 0, 2e), its vertex at -(c - e); as e -> oo with c - e = f
 * it becomes the paraboloid of focal length f.
 *   Every ray from F1 reaches F2 over the path 2c, so a point source at F1
 *   (SC_PROFILE_DIPOLE) keeps the compensated phase of the FP32 path
 *   exact.  A collimated beam (kinds 0-4, phase reference z_ref =
 *   2(c - e)) does not focus on the origin; its phase is exact only in
 *   FP64, and the SC_FP32_COMP path rejects it.
 * Errors: SC_ERR_INVALID when not 0 < e < c, r_min < 0, r_min >= r_max,
 * r_max >= a, or a quadrature as for sc_mirror is invalid.
 */
sc_status sc_mirror_ellipsoid(sc_ctx* ctx, double c, double e, double r_min, double r_max,
                              const sc_quadrature* q, sc_mirror_t** out);

sc_status sc_mirror(sc_ctx* ctx, double f, double r_min, double r_max, const sc_quadrature* q,
                    sc_mirror_t** out);
void sc_mirror_free(sc_mirror_t* m);

/* ---------------------------------------------------------------------- */
/* Incident field (Sec. III.A; Sec. III.B, Eqs. 14-18; Sec. IV.B, Eq. 27)   */

enum {
    SC_PROFILE_GAUSS = 0,
    SC_PROFILE_SUPERGAUSS = 1,
    SC_PROFILE_TOPHAT = 2,
    SC_PROFILE_LAGUERRE_GAUSS = 3, /* paraxial LG mode with finite Rayleigh range */
    SC_PROFILE_ENVELOPE = 4,       /* the caller's envelope function             */
    SC_PROFILE_DIPOLE = 5          /* electric dipole at an ellipsoid's focus F1 */
};

/*
 * Caller's transverse envelope (SC_PROFILE_ENVELOPE): for n mirror points
 * xyz[n][3] and one wavenumber k, write e_perp at each point as
 * e[n][2][2] = (E_x re, im), (E_y re, im).  It stands for measured maps of
 * every frequency component on the mirror and for spatio-temporal couplings
 * (Sec. III.A, Sec. III.B).  The library calls it from the calling thread
 * while it builds a node table (inside sc_eval / sc_eval_batch / the
 * serving thread for sc_submit), never concurrently with itself.
 */
typedef void (*sc_envelope_fn)(void* user, int n, const double* xyz, double k, double* e);
enum { SC_POL_LINEAR = 0, SC_POL_RADIAL = 1, SC_POL_AZIMUTHAL = 2 };
enum {
    SC_SPEC_MONO = 0,              /* a_n = 1                                     */
    SC_SPEC_GAUSS_TIME = 1,        /* Gaussian pulse, intensity FWHM fwhm_t       */
    SC_SPEC_SUPERGAUSS_LAMBDA = 2, /* Eq. 27 in wavelength, centre lambda_c,      */
                                   /* width dlambda, order sg_n                   */
    SC_SPEC_SAMPLED = 3            /* a_n given at n omegas                       */
};

/*
 * Beam on the mirror.  Kinds 0-2 are the collimated beam below; kinds 3 and
 * 4 have a complex envelope that depends on k (see after the struct).
 *
 * Collimated beam on the mirror (the Supplementary Material with the
 * paper's explicit fields is not available; this is the waist-plane limit
 * of its paraxial modes): E_inc = A(rho) p(theta) e^{-ik(z + 2f)} e^{ikW},
 * B_inc = (-z_hat) x E_inc.
 *   A: Gaussian exp(-rho^2/w0^2), super-Gaussian exp(-(rho/w0)^(2 sg_order)),
 *      or top-hat (1 for rho <= w0, 0 beyond).
 *   W: optical path difference sum_j c_j Z_j(rho / r_max, theta), Noll
 *      ordering and normalisation, j = 2 .. n_zernike + 1, c_j in waves at
 *      lambda0 (the caller's array is copied).
 *   order: 0 the collimated beam above, which satisfies div E = 0 only to
 *      O(eps), eps = lambda / (pi w0) (Sec. III.A); 1 adds the first-order
 *      longitudinal terms
 *        E_z = -(i/k) div_perp(e_perp e^{ikW}) e^{-ik(z + 2f)},
 *        B_z = -(i/k) div_perp(b_perp e^{ikW}) e^{-ik(z + 2f)},
 *      e_perp = A p, b_perp = (-z_hat) x e_perp, so that div E = div B = 0
 *      and Maxwell's curl equations hold to O(eps^2).  The 1/k part has its
 *      own node table and doubles the field-sum work; the top-hat (no
 *      transverse derivative) is invalid with order 1.
 */
typedef struct {
    int kind;
    double w0;
    int sg_order;
    int n_zernike;
    const double* zernike_noll_waves;
    int order;
    /* kinds 3 and 4 */
    int lg_p, lg_l;           /* Laguerre-Gauss indices (kind 3)                    */
    double z_waist;           /* waist plane of the Laguerre-Gauss beam (kind 3)    */
    sc_envelope_fn envelope;  /* kind 4; must stay valid while the handle lives    */
    void* envelope_user;
    double omega_lo, omega_hi;  /* band of every omega later evaluated (kinds 3, 4) */
    double fit_tol;           /* truncation tolerance of the fit in k, relative to  */
                              /* the envelope's peak (<= 0: 1e-8)                   */
    double dipole[3];         /* kind 5: the dipole moment p                        */
} sc_profile;

/*
 * Kind 5, the exact field of an electric dipole p at the upper focus F1 of
 * an ellipsoidal mirror (time factor e^{-i omega t}, c = 1):
 *   E = e^{ikr} [k^2 (n x p) x n / r + (3 n (n.p) - p)(1/r^3 - ik/r^2)],
 *   B = e^{ikr} (n x p)(k^2/r + ik/r^2),   r = |P - F1|, n = (P - F1)/r,
 * times e^{-ik 2c} (t = 0 is the focal arrival at F2).  Its k-dependence
 * is sum_m (ik)^m (E_m, B_m), m = 0, 1, 2: three node tables.  It needs an
 * ellipsoidal mirror and a SAMPLED or MONO spectrum (Eq. 16 has no beam
 * power for it); order 0 only.
 */

/*
 * Kinds 3 and 4: E_inc = e_perp(x, y, z; k) e^{-ik(z + 2f)} e^{ikW}, B_inc =
 * (-z_hat) x E_inc (order 0 only).
 *   Kind 3, the Laguerre-Gauss mode (p, l) of the paraxial wave equation,
 *   travelling along -z with its waist (radius w0) at z = z_waist: with
 *   zeta = z_waist - z, z_R = k w0^2 / 2, w = w0 sqrt(1 + (zeta/z_R)^2),
 *   1/R = zeta / (zeta^2 + z_R^2) and psi = atan(zeta / z_R),
 *     u = (w0/w)^(|l|+1) (rho/w0)^|l| L_p^|l|(2 rho^2/w^2) e^{-rho^2/w^2}
 *         e^{ik rho^2 / (2R)} e^{-i(2p+|l|+1) psi},
 *   e_perp = u e^{i l theta} p (linear), u rho_hat or u theta_hat (radial,
 *   azimuthal; |l| = 1).  As z_R -> oo it is the collimated beam above.
 *   Kind 4, the caller's envelope function.  Its spectrum must be SAMPLED
 *   or MONO (Eq. 16 has no beam power for it).
 * The node table holds a Chebyshev expansion in k over [2 pi omega_lo,
 * 2 pi omega_hi] of e_perp e^{-ik tau(node)}, sum_m c_m(node) T_m(x(k)),
 * tau being each node's phase slope in k at the band centre (added to the
 * node's optical path, so a pulse-front tilt costs nothing), truncated where
 * the remaining coefficients sum below fit_tol times the envelope's peak;
 * the real and imaginary parts of each c_m are tables of their own, so a
 * beam costs one field pass per table (see sc_eval_stats.tables).  An
 * envelope that needs more than 20 terms over the band is rejected.
 */

/* p: fixed direction (cos angle, sin angle, 0), or rho_hat * rho/w0
 * (radial), or theta_hat * rho/w0 (azimuthal). */
typedef struct {
    int kind;
    double angle_rad;
} sc_polarization;

/*
 * Spectrum a_n = E0^n e^{i phi(k_n)} (Eqs. 15, 16, 18).  For
 * GAUSS_TIME and SUPERGAUSS_LAMBDA the power spectrum eps(k) (energy per
 * unit k, Eq. 17 normalised to `energy`) gives E0^n = sqrt(eps(k_n) /
 * (4 pi P)), P = SS |A p|^2 dA over the transverse plane.  Eq. 27 is read
 * with a minus sign in its exponent and includes |d lambda/dk|.
 * phi(k) = sum_j phi_taylor[j] (k - k_c)^j / j!, k_c = 2 pi / lambda_c.
 * GAUSS_TIME: field spectrum exp(-(k - k_c)^2 fwhm_t^2 / (8 ln 2)).
 * SAMPLED: n, omega[n], amp_re_im[2n]; sc_eval then needs the same omegas.
 */
typedef struct {
    int kind;
    double fwhm_t;
    double lambda_c;
    double dlambda;
    int sg_n;
    double energy;
    int n;
    const double* omega;
    const double* amp_re_im;
    int n_phi;
    const double* phi_taylor;
} sc_spectrum;

/* Copy the description of an incident beam.  Errors: SC_ERR_INVALID
 * (unknown kind, w0 <= 0, sg_order < 1, n_zernike outside 0..64, order not
 * 0 or 1, order 1 with a top-hat or kinds 3-5, a zero dipole (kind 5), kind
 * 5 with a GAUSS_TIME or SUPERGAUSS_LAMBDA spectrum, lg_p < 0, |lg_l| != 1 for a
 * radial or azimuthal kind 3, kind 4 without a function, kinds 3-4 without
 * 0 < omega_lo < omega_hi, kind 4 with a GAUSS_TIME or SUPERGAUSS_LAMBDA
 * spectrum, a spectrum with non-positive width or lambda_c, SAMPLED with
 * n < 1). */
sc_status sc_incident(sc_ctx* ctx, const sc_profile* prof, const sc_polarization* pol,
                      const sc_spectrum* spec, sc_incident_t** out);
void sc_incident_free(sc_incident_t* inc);

/*
 * How a (mirror, incident) pair will be evaluated, on the host only (no device
 * work; ctx may be NULL): the number of node tables, i.e. of field passes per
 * evaluation (1 for a collimated beam, 2 at order 1, the Chebyshev terms of a
 * k-dependent envelope, 3 for a dipole), and whether the compensated FP32
 * path applies (1) or only SC_FP64 does (0).  fp32_ok may be NULL.  Builds
 * the tables' FP64 nodes to count them, so it costs what a table build costs
 * on the host.  Errors: SC_ERR_INVALID (null arguments, a dipole without an
 * ellipsoid, an envelope too rough to fit).
 */
sc_status sc_table_count(sc_ctx* ctx, const sc_mirror_t* mirror, const sc_incident_t* inc, int* n_tables,
                         int* fp32_ok);

/*
 * How the FP32 path cuts a request of n_omega uniform omegas into chunks, on
 * the host only (ctx may be NULL: planning on).  Each chunk is one pass of a
 * field kernel over the node tables.  The sizes minimise the summed field
 * time of the chunks under field throughputs per omega count measured on
 * GB300, each extra chunk charged 2% of a 32-omega chunk: e.g. 65 omegas run
 * as 64 + 1 (on 16 threads of 8 omegas, 7 would idle), 33 as 1 + 32.
 * pairs_per_omega = points x surface nodes of the request; below 2^22 only
 * full grouped capacities (64, 128, ... omegas) are cut off.  With
 * SC_OPT_OMEGA_CHUNKS = 0 on ctx: one chunk per 2048 omegas.  Writes up to
 * max_sizes chunk sizes in order and their count to *n_sizes.
 * Errors: SC_ERR_INVALID (n_omega < 1, negative pairs, NULL n_sizes, or more
 * chunks than max_sizes; *n_sizes is set in that case).
 */
sc_status sc_plan_omega_chunks(sc_ctx* ctx, int n_omega, long long pairs_per_omega, int* sizes, int max_sizes,
                               int* n_sizes);

/* Evaluate a_n (Eqs. 16 and 18) at n host omegas into host amp_re_im[2n]. */
sc_status sc_spectrum_eval(sc_ctx* ctx, const sc_incident_t* inc, const double* omegas, int n,
                           double* amp_re_im);

/* ---------------------------------------------------------------------- */
/* Field evaluation (Sec. II, Eq. 11; the hot path)                         */

typedef enum { SC_FP32_COMP = 0, SC_FP64 = 1 } sc_precision;

typedef struct {
    double evals;       /* points x surface nodes x omegas of this call          */
    double field_ms;    /* CUDA-event time of the field-sum launches              */
    double total_ms;    /* CUDA-event time of the whole call on the stream        */
    int launches;       /* kernels launched by the call                           */
    int tables;         /* node tables summed per evaluation (field passes; for a */
                        /* batch the largest over its requests)                   */
    /* the tile shape chosen for the (first request's) first omega chunk on the   */
    /* FP32 path, or -1 on the FP64 path: kernel class, threads per point, omegas */
    /* per thread (the measured default layout for its omega count, or the       */
    /* autotuner's choice between it and an alternative) and node splits         */
    int kernel_class;
    int threads_per_point;
    int omegas_per_thread;
    int splits;
} sc_eval_stats;

/*
 * E(r'_p, omega_n) and B(r'_p, omega_n), reflected field only.
 *   omegas      host, n_omega >= 1 values (> 0).  SC_FP32_COMP needs a uniform
 *               grid (|omega_n - omega_0 - n d| <= 1e-9 omega_0); SC_FP64 takes
 *               any grid.
 *   points_xyz  host or device, [n_points][3] doubles.
 *   E_out,B_out host or device, [n_omega][n_points][3] complex: float2 pairs
 *               for SC_FP32_COMP, double2 pairs for SC_FP64.  B_out may be NULL.
 *   stats       nullable; when given the call synchronizes the stream and
 *               fills it.
 * The first call for a (mirror, incident) pair builds its node table (FP64 on
 * the host, uploaded once, then resident in HBM).
 * Errors: SC_ERR_INVALID (null pointers, n_points < 1, n_omega < 1, omega <= 0,
 * non-uniform grid for SC_FP32_COMP, SAMPLED spectrum whose omegas differ,
 * a point closer than 1e-6 lambda0 to the mirror), SC_ERR_OOM, SC_ERR_CUDA,
 * SC_ERR_TIMEOUT (a bounded device wait ran out; outputs undefined).
 */
sc_status sc_eval(sc_ctx* ctx, const sc_mirror_t* mirror, const sc_incident_t* inc,
                  const double* omegas, int n_omega, const double* points_xyz, int n_points,
                  sc_precision prec, void* E_out, void* B_out, sc_eval_stats* stats);

/*
 * Semi-discrete inverse transform, Sec. III.B Eq. 13, for a real field on a
 * positive-frequency grid: F(t_m) = 2 Re sum_n F_n e^{-i k_n t_m} dk with
 * dk = 2 pi (omega_1 - omega_0) (uniform grid required) or dk = 1 when
 * n_omega = 1.
 *   E_spec,B_spec  host or device spectra laid out as sc_eval writes them
 *                  (element type chosen by prec); B_spec may be NULL.
 *   times          host, n_t values.
 *   E_t,B_t        host or device, float [n_t][n_points][3]; B_t NULL iff
 *                  B_spec is NULL.
 * Errors: SC_ERR_INVALID, SC_ERR_OOM, SC_ERR_CUDA.
 */
sc_status sc_time_domain(sc_ctx* ctx, sc_precision prec, const void* E_spec, const void* B_spec,
                         const double* omegas, int n_omega, int n_points, const double* times,
                         int n_t, float* E_t, float* B_t);

/*
 * The time-domain field without the spectral field (Sec. III.B, Eq. 13 applied
 * to the spectra of Eq. 11): the omegas are evaluated in chunks, and each
 * chunk's spectra are transformed and added into E_t, B_t, so device memory
 * holds one chunk of spectra at a time whatever n_omega is.  Equal to sc_eval
 * followed by sc_time_domain up to the FP32 rounding of the chunk sums.
 *   omegas        host, a uniform increasing grid (both precisions).
 *   points_xyz    host or device, [n_points][3] doubles.
 *   times         host, n_t values.
 *   omega_chunk   omegas per chunk, or <= 0: the whole grid when its E and B
 *                 spectra fit in 32 GiB, else the largest power of two that
 *                 does.
 *   E_t, B_t      host or device, float [n_t][n_points][3]; B_t may be NULL.
 *   stats         nullable, as for sc_eval (synchronizes).
 * Synchronizes the context stream.  Errors: as sc_eval and sc_time_domain.
 */
sc_status sc_eval_time_domain(sc_ctx* ctx, const sc_mirror_t* mirror, const sc_incident_t* inc,
                              const double* omegas, int n_omega, const double* points_xyz, int n_points,
                              sc_precision prec, const double* times, int n_t, int omega_chunk,
                              float* E_t, float* B_t, sc_eval_stats* stats);

/*
 * Allocation-free variant of sc_eval for the SC_FP32_COMP path.  The paper
 * has no counterpart: this entry point exists for callers that cannot call
 * cudaMalloc while they evaluate -- services that hand all device memory to
 * their own pools at start-up (an allocation would fail or escape their
 * accounting), and real-time or latency-bound loops that forbid cudaMalloc
 * and cudaFree because those calls can block on the whole device.  It
 * allocates nothing: no cudaMalloc, no cudaFree, no allocating library
 * routine, and it copies nothing from the host.  The wavenumbers k_n and the
 * split partials live in a fixed 64 MiB static device array of the library
 * (SC_STATIC_SCRATCH_BYTES), which every GPU that loads the library holds
 * until the process exits.
 *   Preconditions: the node table of (mirror, inc) is already resident in
 *   ctx, i.e. sc_eval ran once for this pair (that call may allocate), and
 *   the pair needs a single node table on the FP32 path (sc_table_count
 *   gives 1 table and fp32_ok 1: a collimated beam of order 0 on the
 *   paraboloid).  Other pairs are rejected with SC_ERR_INVALID: use sc_eval.
 *   omega_n = omega0 + n * domega, n < n_omega (<= 2048), omega0 > 0.
 *   amp_re_im   device, [n_omega][2] doubles, caller-owned (e.g. filled from
 *               sc_spectrum_eval); read by the call's kernels.
 *   points_xyz  device, [n_points][3] doubles.
 *   E_out,B_out device, [n_omega][n_points][3] float2 pairs; B_out may be NULL.
 * A host pointer in any of these is rejected with SC_ERR_INVALID.  The
 * scratch needed is 2 x 96 x n_points x n_omega bytes plus 8 x n_omega
 * (rounded up to 256); larger requests are rejected with SC_ERR_INVALID and
 * a message giving the limit.  The first call on a device looks up the
 * array's device address (which may load the library's module) and leaves
 * the caller's current device as it was; make that first call before any
 * stream capture begins.  Every call shares the array and
 * leaves its contents behind; each call writes every value it later reads,
 * so nothing needs clearing, but calls whose GPU work overlaps (other
 * streams, other contexts on the same device) race on it.  Asynchronous on
 * the context stream: as for sc_eval with device buffers and no stats, a
 * bounded device wait that runs out is reported as SC_ERR_TIMEOUT by the
 * context's next call that synchronizes (sc_get_counters, or an sc_eval
 * with stats).
 * Errors: SC_ERR_INVALID, SC_ERR_CUDA.
 */
#define SC_STATIC_SCRATCH_BYTES ((size_t)64 << 20)
sc_status sc_eval_fp32_static(sc_ctx* ctx, const sc_mirror_t* mirror, const sc_incident_t* inc,
                              double omega0, double domega, int n_omega, const double* amp_re_im,
                              const double* points_xyz, int n_points, void* E_out, void* B_out);

/*
 * Batched evaluation (SC_FP32_COMP): many requests of uneven size -- each its
 * own mirror, beam, uniform omega grid and point set -- in one scheduled
 * pass.  Work items (request, omega chunk, point block, node split) of all
 * requests are drained by one persistent kernel per kernel class from a
 * device queue, the field launches are captured in a CUDA graph (replayed
 * while the batch shape repeats), and one FP64 reduction finishes every
 * request.  Each request's tiling depends only on its own shape, so its
 * result is bitwise the same as sc_eval of that request alone.
 * This is the batching pattern of the hot path; the paper computes one
 * problem at a time with a domain decomposition over points (Sec. III.C.2).
 *   omegas      host; points_xyz, E_out, B_out device (B_out may be NULL);
 *               layouts as for sc_eval with SC_FP32_COMP.
 * Asynchronous on the context stream unless stats is given.
 * Errors: as sc_eval; SC_ERR_INVALID names the failing request (checked
 * before any work, including the FP32 precondition of each request).
 */
typedef struct {
    const sc_mirror_t* mirror;
    const sc_incident_t* incident;
    const double* omegas;
    int n_omega;
    const double* points_xyz;
    int n_points;
    void* E_out;
    void* B_out;
} sc_request;

sc_status sc_eval_batch(sc_ctx* ctx, const sc_request* reqs, int n_req, sc_eval_stats* stats);

/* ---------------------------------------------------------------------- */
/* Serving: continuous batching of submitted requests                       */
/*
 * A server thread (started by the first sc_submit) admits queued requests in
 * arrival order while the device memory they need fits the context's HBM
 * budget (staged points and, for requests without outputs, the outputs the
 * server allocates), batches them and runs each batch as sc_eval_batch does
 * on a free lane (a stream with its own buffers), so a batch starts while
 * others are still on the GPU.  Node tables stay resident between requests.
 * The paper has one problem per run; this is the serving pattern of the hot
 * path.
 *   Short requests first (SC_OPT_SERVE_PRIORITY = 1, the default): a request
 *   of at most 1e11 evaluations (points x surface nodes x omegas) is short.
 *   Short requests run on two lanes of the highest stream priority, in
 *   batches of up to 64 requests that close at 3e10 evaluations.  Long
 *   requests run one per lane on two lanes of the lowest priority, with their
 *   chunks cut by points into launches of about 6e10 evaluations (larger
 *   where that would leave a launch fewer than 4 work items per resident
 *   CTA), each launched when the previous one completes.  A short request
 *   then waits for at most one such launch of a long one, never for all of
 *   it.  Results are bitwise those of the request alone either way.
 *   SC_OPT_SERVE_PRIORITY = 0: two lanes of the default priority, first come
 *   first served, batches of up to 64 requests, launches not bounded.
 *
 * sc_submit   req->points_xyz host (copied) or device (kept by reference);
 *             req->E_out/B_out NULL: server-owned outputs, read them with
 *             sc_fetch; else caller-owned device outputs (float2 layout of
 *             sc_eval).  Caller-owned buffers must stay valid until done.
 *             SC_ERR_BUSY: the request alone exceeds the budget.
 *             SC_ERR_INVALID at once when the (mirror, incident) pair does
 *             not focus on the origin (the FP32 path's precondition).  A
 *             request whose node tables cannot be built (an envelope too
 *             rough to fit, a failed table allocation) fails its own ticket
 *             with that status; the rest of its batch runs.
 * sc_poll     *done = 1 once finished, failed or cancelled (the status says
 *             which: SC_OK, the failure, or SC_ERR_CANCELLED).
 * sc_wait     blocks up to timeout_s; SC_ERR_TIMEOUT if still running.
 * sc_cancel   drops a queued request, or discards a running one's result.
 * sc_fetch    copies a finished request's E, B (host or device dst, either
 *             nullable) and synchronizes.
 * sc_release  frees the ticket and its server-owned memory (SC_ERR_BUSY
 *             while its batch runs); memory returns to the admission budget.
 * sc_ticket_times  seconds since the server started: submitted, started on
 *             the GPU, observed finished (latency = t_done - t_submit).
 * Errors: SC_ERR_NOT_FOUND for unknown tickets; others as sc_eval.
 */
sc_status sc_submit(sc_ctx* ctx, const sc_request* req, uint64_t* ticket);
sc_status sc_poll(sc_ctx* ctx, uint64_t ticket, int* done);
sc_status sc_wait(sc_ctx* ctx, uint64_t ticket, double timeout_s);
sc_status sc_cancel(sc_ctx* ctx, uint64_t ticket);
sc_status sc_fetch(sc_ctx* ctx, uint64_t ticket, void* E_dst, void* B_dst);
sc_status sc_release(sc_ctx* ctx, uint64_t ticket);
sc_status sc_ticket_times(sc_ctx* ctx, uint64_t ticket, double* t_submit, double* t_start,
                          double* t_done);

/* ---------------------------------------------------------------------- */
/* Counters (measurement)                                                  */

typedef struct {
    uint64_t launches;       /* kernels launched by this context since reset       */
    uint64_t field_launches; /* field-sum kernel launches since reset              */
    double field_ms;         /* summed CUDA-event time of those launches           */
    double evals;            /* points x nodes x omegas issued since reset         */
    uint64_t graph_captures; /* CUDA graphs captured for batched launches           */
    uint64_t graph_replays;  /* launches that replayed a cached graph               */
} sc_counters;

/*
 * Measured throughput of the arithmetic pipes that bound the field sum (the
 * per-evaluation FMA work of Eq. 11 and the per-pair rsqrt, rcp and sincos
 * of the phase, Sec. III.C): streams of independent FP32 FMAs, of packed
 * FFMA2 (two lane-ops each) and of MUFU rsqrt.approx, on every SM of the
 * context's device, best of three timed launches after one warm-up, about
 * 0.1 s of GPU work in all.  Outputs are operations per second (lane-ops
 * for the FMA forms).  Synchronizes the context stream.
 * Errors: SC_ERR_INVALID on a NULL argument; SC_ERR_CUDA if a launch fails.
 */
sc_status sc_measure_alu_peaks(sc_ctx* ctx, double* fp32_lane_ops_per_s, double* fp32x2_lane_ops_per_s,
                               double* mufu_ops_per_s);

/*
 * Failure-path self-test (no counterpart in the paper).  Launches one bounded
 * wait, of the kind every field kernel uses for its bulk copies and table
 * hand-overs, on an mbarrier that nothing completes.  The wait gives up
 * after its wall-time limit (about one second), the kernel returns, and the
 * call reports SC_ERR_TIMEOUT; the context stays usable.  Synchronizes.
 */
sc_status sc_selftest_wait(sc_ctx* ctx);

/* Synchronizes the context stream and returns the counters. */
sc_status sc_get_counters(sc_ctx* ctx, sc_counters* out);
sc_status sc_reset_counters(sc_ctx* ctx);

/* Tuning / instrumentation options (value semantics per option). */
enum {
    SC_OPT_TIME_FIELD = 1,      /* 1: bracket each field-sum launch with events  */
    SC_OPT_NODES_PER_SPLIT = 2, /* surface nodes per split (multiple of 32), or 0 */
                                /* to pick the split count for load balance       */
    SC_OPT_WORKSPACE_CAP = 3,   /* max workspace bytes per launch chunk           */
    SC_OPT_FLUSH_NODES = 4,     /* nodes summed in an FP32 run before it is folded */
                                /* into the compensated partial (multiple of 32;   */
                                /* default 2048, at most 512 for beams fitted in k)*/
    SC_OPT_GRAPHS = 5,          /* 1 (default): capture/replay field launches       */
    SC_OPT_AUTOTUNE = 6,        /* 1 (default): time split-count candidates on the  */
                                /* first request of each shape and cache the best   */
                                /* (chunks above 1.2e12 evaluations are not timed:  */
                                /* they take the most splits whose workspace fits)  */
    SC_OPT_OMEGA_CHUNKS = 7,    /* 1 (default): cut a request's omegas into chunks  */
                                /* that keep the field kernels' threads busy;      */
                                /* 0: one chunk per 2048 omegas                     */
    SC_OPT_MFIE_ORDER = 9,      /* 0 (default): physical optics; 1: add the first  */
                                /* correction of the MFIE's Liouville-Neumann      */
                                /* series (see below; sc_eval, sc_eval_time_domain) */
    SC_OPT_MFIE_RHO = 10,       /* its polar rule: Gauss-Legendre points per ray    */
                                /* (default 64)                                     */
    SC_OPT_MFIE_PHI = 11,       /* ... and rays about each node (default 128)       */
    SC_OPT_CLASS_STREAMS = 12,  /* 1 (default): the field launches of a batch's     */
                                /* kernel classes run as concurrent branches        */
    SC_OPT_TILE_LAYOUT = 13,    /* tile shape of the FP32 field kernel (threads per */
                                /* point x omegas per thread) for chunks of 8,      */
                                /* 9..16, 33..64 and 65..128 omegas, which have two */
                                /* near layouts: -1 (default) the autotuner times   */
                                /* both on the first chunk of each shape when       */
                                /* SC_OPT_AUTOTUNE is on (else the default); 0 the  */
                                /* default layout; 1 the alternative.  Other omega  */
                                /* counts have one layout.  sc_eval_stats reports   */
                                /* the layout taken                                 */
    SC_OPT_SERVE_PRIORITY = 14, /* 1 (default): serving runs short requests first   */
                                /* and long ones in bounded launches (see Serving); */
                                /* 0: first come first served.  Stops an idle      */
                                /* server (the next sc_submit restarts it);         */
                                /* SC_ERR_BUSY while a ticket is not yet released   */
    SC_OPT_FAIL_COPY = 8        /* failure-path test, -1 (default) off: in every   */
                                /* batched FP32 field launch, the work item 0 skips */
                                /* the bulk copy of its node tile `value`, so the   */
                                /* wait for that tile runs out (no fault, no copy   */
                                /* in flight); the launch then stops and the call   */
                                /* reports SC_ERR_TIMEOUT                           */
};
sc_status sc_set_option(sc_ctx* ctx, int option, long long value);

/*
 * The first correction beyond physical optics (SC_OPT_MFIE_ORDER = 1).  Sec. II
 * writes the mirror current as the solution of the magnetic-field integral
 * equation (1/2) J = J_inc + n x PV SS J x grad g dS and solves it by its
 * Liouville-Neumann series, whose first term is physical optics, J0 =
 * 2 J_inc (all of the field above).  With the option set, sc_eval (and
 * sc_eval_time_domain, which calls it per chunk) adds the next term:
 *   dJ(r_t) = 2 n_t x PV SS J0(r) x grad g(r, r_t) dS(r)
 * at every surface node r_t, and the field of dJ at the points, from
 * Sancer's representation with n x E = 0 (Eq. 10's form for a general
 * current): E += SS {ik dJ g + (i/k) grad grad g . dJ} dS, B += SS dJ x
 * grad g dS, on the mirror's own nodes.  The principal value is taken in
 * polar coordinates about each node (Gauss-Legendre in rho from the node to
 * the rim, SC_OPT_MFIE_RHO points; SC_OPT_MFIE_PHI rays), whose Jacobian
 * cancels the O(1/R) integrand.  The polar rule must resolve the phase of
 * g between mirror points (tens of points per wavelength of path along a
 * ray), and the node grid must resolve dJ: the correction is meant for
 * mirrors of tens to hundreds of wavelengths, where it is of order
 * lambda / (curvature radius).  Both correction sums run in FP64 and cost
 * n_nodes x n_rho x n_phi and n_points x n_nodes evaluations per omega.
 * Needs a disk (r_min = 0), a paraboloid or ellipsoid, and a collimated beam
 * (kinds 0-2) of order 0; other pairs, sc_eval_batch, sc_submit and
 * sc_eval_fp32_static are refused with SC_ERR_INVALID while the option is set.
 */

#ifdef __cplusplus
}
#endif

#if defined(__GNUC__) && !defined(__CUDA_ARCH__)
#pragma GCC visibility pop
#endif

#endif /* SC_H */
