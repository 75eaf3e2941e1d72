/*
 * sc_oracle.c -- plain, slow, FP64 CPU oracle for the physical-optics
 * Stratton-Chu focal field of a parabolic mirror.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the test-suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; it is written directly from the paper
 * (Dumont et al., "Efficiently parallelized modeling of tightly focused,
 * large bandwidth laser pulses", arXiv:1609.08146):
 *
 *   - Sec. II, Eq. 11 (label eq:theory.stratton-chu-poa-og): reflected field
 *     E' = 2 SS { ik (n x B_inc) g + (n . E_inc) grad g } dS
 *          - (2/ik) O grad g [n x (n x B_inc)] . dl
 *     B' = 2 SS (n x B_inc) x grad g dS
 *   - Sec. II, Eq. 2: g = exp(ik|r - r'|) / (4 pi |r - r'|)
 *   - Sec. II, Eq. 10 (label eq:theory.stratton-chu-poa) with the dyadic of
 *     Appendix A (eq:singularInt.doubleGradientExp): the "double-gradient"
 *     form, kept here as an independent second oracle.
 *   - Sec. III.A: incident field on the mirror, beam travelling along -z,
 *     mirror given as z = F(r, theta) in cylindrical coordinates.
 *   - Sec. III.B, Eqs. 12-18: Fourier convention exp(-ikt), semi-discrete
 *     inverse transform, per-component amplitude from a power spectrum
 *     (Eq. 16) and a spectral phase map (Eq. 18).
 *   - Sec. II, eq:theory.mfie with its Liouville-Neumann series: the first
 *     correction beyond physical optics (eq:theory.poa), and Appendix A's
 *     singular limits (the principal value of the on-surface integral).
 *   - Sec. III.C.1, Eq. 21: the paraboloid z = r^2/(4f) - f with its focus at
 *     the origin; Sec. III.C.1: tensor-product quadrature, Gauss-Legendre or
 *     composite Simpson in r (the two rules it names), trapezoid in theta.
 *   - Sec. IV.B, Eq. 27: super-Gaussian power spectrum in wavelength.
 *
 * Readings of passages the paper leaves open (its Supplementary Material,
 * which holds the explicit incident fields, is not available):
 *   R1  grad acts on the surface variable r: grad g = (ik - 1/R) g (r-r')/R
 *       (Appendix A defines R = r - r').
 *   R2  the unit normal points to the illuminated side (+z at the vertex).
 *   R3  the boundary curve is oriented counter-clockwise seen from the side
 *       the normal points to (Stokes' theorem), so the outer rim runs with
 *       increasing theta and an inner rim (r_min > 0) with decreasing theta.
 *   R4  the incident beam is collimated: E_inc = A(rho) p(theta)
 *       exp(-ik(z + z_ref)) exp(ik W), B_inc = (-z) x E_inc, with
 *       z_ref = 2f for the paraboloid (so the geometric focal arrival is at
 *       t = 0) and z_ref = -z0 for the flat test mirror.  A is Gaussian
 *       exp(-rho^2/w0^2), super-Gaussian exp(-(rho/w0)^(2N)) or a top-hat of
 *       radius w0;
 *       p is a fixed linear direction, rho_hat (radial) or theta_hat
 *       (azimuthal), the last two times rho/w0.  W is the optical path
 *       difference of a Zernike expansion (Noll ordering) on the unit disk
 *       rho / r_norm, coefficients in waves at lambda0.
 *   R5  the super-Gaussian of Eq. 27 carries a minus sign in its exponent;
 *       energy per unit k includes |d lambda / dk| = lambda^2 / (2 pi).
 *   R6  units: lambda0 = c = 1, k = 2 pi omega with omega in units of
 *       omega0 = 2 pi c / lambda0; time in lambda0 / c.
 *   R15 frequency-dependent incident envelopes (profiles 3 and 4): the beam
 *       is E_inc = e_perp(x, y, z; k) exp(-ik(z + z_ref)) exp(ikW), B_inc =
 *       (-z) x E_inc, with a complex transverse envelope e_perp that may
 *       depend on k.  Profile 3 is the Laguerre-Gauss mode (p, l) of the
 *       paraxial wave equation travelling along -z with its waist at
 *       z = z_waist (Sec. III.A's beam basis): with zeta = z_waist - z,
 *       z_R = k w0^2 / 2, w = w0 sqrt(1 + zeta^2/z_R^2),
 *       1/R = zeta / (zeta^2 + z_R^2), psi = atan(zeta / z_R),
 *         u = (w0/w)^(|l|+1) (rho/w0)^|l| L_p^|l|(2 rho^2/w^2)
 *             exp(-rho^2/w^2) exp(ik rho^2 / (2R)) exp(-i(2p+|l|+1) psi),
 *       e_perp = u exp(i l theta) p_lin (linear), u rho_hat (radial) or
 *       u theta_hat (azimuthal), the last two with |l| = 1; as z_R -> oo it
 *       is the collimated beam of R4.  The constant phase exp(ik(z_waist +
 *       z_ref)) is dropped, so t = 0 stays the geometric focal arrival.
 *       Profile 4 takes e_perp from a caller's function (measured maps,
 *       spatio-temporal couplings), sampled once per frequency and node.
 *   R16 NEXT-4, an ellipsoidal mirror and a point source: surface 2 is the
 *       lower cap of the ellipsoid of revolution with semi-axis c along z
 *       and focal half-distance e < c, its lower focus F2 at the origin and
 *       its upper focus F1 at (0, 0, 2e): z = e - c sqrt(1 - r^2/a^2),
 *       a^2 = c^2 - e^2, vertex at z = -(c - e) (as e -> oo with c - e = f
 *       fixed it is the paraboloid of focal length f, F1 going to infinity
 *       above it).  Profile 5 is the exact field of an electric
 *       dipole p at F1 (time factor exp(-i omega t), c = 1),
 *         E = e^{ikr} [k^2 (n x p) x n / r + (3 n (n.p) - p)(1/r^3 - ik/r^2)],
 *         B = e^{ikr} (n x p) (k^2/r + ik/r^2),
 *       r = |P - F1|, n = (P - F1)/r, times exp(-ik 2c) (every ray F1 ->
 *       mirror -> F2 has length 2c, so t = 0 is the focal arrival at F2).
 *       Collimated beams on the ellipsoid use z_ref = -2 z_vertex = 2(c - e),
 *       as z_ref = 2f for the paraboloid.
 *   R14 first-order incident field (beam order 1): the collimated beam of R4
 *       is not divergence-free at O(eps), eps = lambda / (pi w0) (Sec. III.A).
 *       Order 1 adds the longitudinal terms that make div E = div B = 0 and
 *       leave Faraday's and Ampere's laws violated only at O(eps^2):
 *         E_z = -(i/k) div_perp(e_perp exp(ikW)) exp(-ik(z + z_ref)),
 *         B_z = -(i/k) div_perp(b_perp exp(ikW)) exp(-ik(z + z_ref)),
 *       b_perp = (-z) x e_perp; B_perp stays (-z) x E_perp.  Here the
 *       transverse divergences are taken by fourth-order central
 *       differences of step 1e-3 w0 (the library uses closed forms).
 *   R17 the first correction beyond physical optics (NEXT-4): the
 *       Liouville-Neumann series of the MFIE (Sec. II) starts at J0 = 2 J_inc
 *       and its next term adds dJ = 2 n_t x PV SS J0 x grad g dS.  The
 *       integrand is O(1/R) at the target on a smooth surface, so the
 *       principal value is the improper integral, taken in polar coordinates
 *       about the target (Gauss-Legendre in rho to the rim, trapezoid in phi).
 *       The corrected field adds the field of dJ from Sancer's representation
 *       with n x E = 0 (Eq. 10's form for a general current) on the mirror's
 *       nodes.  Disks (r_min = 0) and collimated beams of order 0 only.
 *
 * Output layout: E[n_omega][n_pts][3] complex, stored as interleaved doubles
 * (re, im); same for B.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Parameter blocks (mirrored by ctypes structures in oracle/__init__.py).   */

typedef struct {
    int surface;      /* 0: paraboloid z = r^2/(4f) - f; 1: flat disk z = z0 */
    int n_r;          /* nodes in r on [r_min, r_max] (rule: `radial` below)  */
    int n_theta;      /* trapezoid nodes in theta, theta_l = 2 pi l / n_theta  */
    int rim;          /* 1: include the boundary line integral of Eq. 11      */
    double f;         /* focal length                                          */
    double z0;        /* plane height of the flat test mirror                  */
    double r_min;
    double r_max;
    double c_ell, e_ell; /* ellipsoid (surface 2): semi-axis along z, focal half-distance */
    int radial;       /* radial rule: 0 Gauss-Legendre, 1 composite Simpson (n_r odd)   */
} or_mirror;

typedef struct {
    int profile;      /* 0 Gaussian, 1 super-Gaussian, 2 top-hat              */
    int sg_order;     /* N of exp(-(rho/w0)^(2N))                              */
    int pol;          /* 0 linear, 1 radial, 2 azimuthal                      */
    int n_zern;       /* number of Zernike coefficients, Noll j = 2 ..         */
    double w0;
    double pol_angle; /* direction of linear polarisation in the xy-plane      */
    double r_norm;    /* radius of the Zernike unit disk                       */
    const double* zern;
    int order;        /* 0: collimated beam (R4); 1: plus the O(eps) terms (R14) */
    int lg_p, lg_l;   /* Laguerre-Gauss indices (profile 3)                   */
    double z_waist;   /* waist plane of the Laguerre-Gauss beam               */
    /* profile 4: fn(user, n, xyz[n][3], k, e[n][2][2]) writes e_perp (re, im) */
    void (*env_fn)(void* user, int n, const double* xyz, double k, double* e);
    void* env_user;
    double dip[3];    /* profile 5: dipole moment and position, and the path */
    double src[3];    /* length removed from its phase (R16)                  */
    double phase_ref;
} or_beam;

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre rule on [a, b] (the quadrature named in Sec. III.C.1):     */
/* nodes are the roots of the Legendre polynomial P_n, found by Newton's    */
/* method from the three-term recurrence; w_i = 2 / ((1 - x^2) P_n'(x)^2).   */

int or_gauss_legendre(int n, double a, double b, double* x, double* w)
{
    if (n < 1) return 1;
    for (int i = 0; i < n; ++i) {
        double t = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            /* P_n(t) = p1, P_{n-1}(t) = p0 */
            dp = n * (t * p1 - p0) / (t * t - 1.0);
            double dt = p1 / dp;
            t -= dt;
            if (fabs(dt) < 1e-16) break;
        }
        /* recompute the derivative at the converged root */
        {
            double p0 = 1.0, p1 = t;
            for (int j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * t * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = t; p0 = 1.0; }
            dp = n * (t * p1 - p0) / (t * t - 1.0);
        }
        double wi = 2.0 / ((1.0 - t * t) * dp * dp);
        /* roots come out in decreasing t; store ascending */
        int k = n - 1 - i;
        x[k] = 0.5 * (a + b) + 0.5 * (b - a) * t;
        w[k] = 0.5 * (b - a) * wi;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Composite Simpson rule on [a, b] (the other rule Sec. III.C.1 names): the */
/* n = 2m + 1 equally spaced nodes form m panels of two intervals, and each  */
/* panel [x_2p, x_2p+2] adds Simpson's (h/3)(f_2p + 4 f_2p+1 + f_2p+2).      */

int or_simpson(int n, double a, double b, double* x, double* w)
{
    if (n < 3 || n % 2 == 0) return 1;
    const int intervals = n - 1;
    const double h = (b - a) / intervals;
    for (int i = 0; i < n; ++i) {
        x[i] = a + (b - a) * ((double)i / intervals);
        w[i] = 0.0;
    }
    for (int panel = 0; 2 * panel + 2 < n; ++panel) {
        w[2 * panel] += h / 3.0;
        w[2 * panel + 1] += 4.0 * h / 3.0;
        w[2 * panel + 2] += h / 3.0;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Zernike polynomials, Noll (1976) ordering and normalisation.              */

static void noll_to_nm(int j, int* n_out, int* m_out)
{
    int jj = 1;
    for (int n = 0;; ++n) {
        for (int am = n % 2; am <= n; am += 2) {
            if (am == 0) {
                if (jj == j) { *n_out = n; *m_out = 0; return; }
                jj += 1;
            } else {
                /* the even index of the pair carries cos (m > 0), the odd sin */
                if (jj == j) { *n_out = n; *m_out = (jj % 2 == 0) ? am : -am; return; }
                if (jj + 1 == j) { *n_out = n; *m_out = ((jj + 1) % 2 == 0) ? am : -am; return; }
                jj += 2;
            }
        }
    }
}

static double factorial(int n)
{
    double r = 1.0;
    for (int i = 2; i <= n; ++i) r *= i;
    return r;
}

double or_zernike(int j, double rho, double theta)
{
    int n, m;
    noll_to_nm(j, &n, &m);
    int am = abs(m);
    double radial = 0.0;
    for (int s = 0; s <= (n - am) / 2; ++s) {
        double c = factorial(n - s) /
                   (factorial(s) * factorial((n + am) / 2 - s) * factorial((n - am) / 2 - s));
        radial += ((s % 2) ? -c : c) * pow(rho, n - 2 * s);
    }
    if (m == 0) return sqrt(n + 1.0) * radial;
    double ang = (m > 0) ? cos(am * theta) : sin(am * theta);
    return sqrt(2.0 * (n + 1.0)) * radial * ang;
}

/* ------------------------------------------------------------------------ */
/* Incident field model (reading R4).                                        */

static double beam_amplitude(const or_beam* bm, double rho)
{
    switch (bm->profile) {
    case 0: return exp(-(rho * rho) / (bm->w0 * bm->w0));
    case 1: return exp(-pow(rho / bm->w0, 2.0 * bm->sg_order));
    default: return (rho <= bm->w0) ? 1.0 : 0.0;
    }
}

/* spatial part of E_inc at (x, y): A(rho) p(theta), a real transverse vector */
static void beam_field(const or_beam* bm, double x, double y, double e[3])
{
    double rho = sqrt(x * x + y * y);
    double a = beam_amplitude(bm, rho);
    double th = atan2(y, x);
    if (bm->pol == 0) {
        e[0] = a * cos(bm->pol_angle);
        e[1] = a * sin(bm->pol_angle);
    } else if (bm->pol == 1) {
        double s = a * rho / bm->w0;
        e[0] = s * cos(th);
        e[1] = s * sin(th);
    } else {
        double s = a * rho / bm->w0;
        e[0] = -s * sin(th);
        e[1] = s * cos(th);
    }
    e[2] = 0.0;
}

/* optical path difference W(x, y) = sum_j c_j Z_j(rho / r_norm, theta) */
static double beam_opd(const or_beam* bm, double x, double y)
{
    if (bm->n_zern <= 0) return 0.0;
    double rho = sqrt(x * x + y * y) / bm->r_norm;
    double th = atan2(y, x);
    double w = 0.0;
    for (int i = 0; i < bm->n_zern; ++i) w += bm->zern[i] * or_zernike(i + 2, rho, th);
    return w;
}

/* Exact field of the dipole of profile 5 at (x, y, z) (R16), including its
 * phase exp(ik (r - phase_ref)) and the extra phase exp(ik extra). */
static void dipole_field(const or_beam* bm, double k, double x, double y, double z, double extra,
                         cplx E[3], cplx B[3])
{
    const double d[3] = {x - bm->src[0], y - bm->src[1], z - bm->src[2]};
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    const double n[3] = {d[0] / r, d[1] / r, d[2] / r};
    const double* p = bm->dip;
    const double np = n[0] * p[0] + n[1] * p[1] + n[2] * p[2];
    const double nxp[3] = {n[1] * p[2] - n[2] * p[1], n[2] * p[0] - n[0] * p[2], n[0] * p[1] - n[1] * p[0]};
    const cplx ph = cexp(I * k * (r - bm->phase_ref + extra));
    const cplx near = 1.0 / (r * r * r) - I * k / (r * r);
    for (int c = 0; c < 3; ++c) {
        const double far = p[c] - n[c] * np; /* (n x p) x n */
        E[c] = ph * (k * k * far / r + (3.0 * n[c] * np - p[c]) * near);
        B[c] = ph * nxp[c] * (k * k / r + I * k / (r * r));
    }
}

/* generalised Laguerre polynomial L_p^a(x) by its three-term recurrence */
static double laguerre(int p, int a, double x)
{
    double l0 = 1.0, l1 = 1.0 + a - x;
    if (p == 0) return l0;
    for (int n = 1; n < p; ++n) {
        double l2 = ((2.0 * n + 1.0 + a - x) * l1 - (n + a) * l0) / (n + 1.0);
        l0 = l1;
        l1 = l2;
    }
    return l1;
}

/* Laguerre-Gauss envelope e_perp (complex x, y) of reading R15 at (x, y, z) */
static void lg_envelope(const or_beam* bm, double k, double x, double y, double z, cplx e[2])
{
    const double w0 = bm->w0, zr = 0.5 * k * w0 * w0, zeta = bm->z_waist - z;
    const double w = w0 * sqrt(1.0 + (zeta / zr) * (zeta / zr));
    const double invR = zeta / (zeta * zeta + zr * zr), psi = atan(zeta / zr);
    const double rho2 = x * x + y * y, rho = sqrt(rho2), th = atan2(y, x);
    const int al = (bm->pol == 0) ? abs(bm->lg_l) : 1;
    const double amp = pow(w0 / w, al + 1.0) * pow(rho / w0, al) *
                       laguerre(bm->lg_p, al, 2.0 * rho2 / (w * w)) * exp(-rho2 / (w * w));
    const cplx u = amp * cexp(I * (0.5 * k * rho2 * invR - (2.0 * bm->lg_p + al + 1.0) * psi));
    if (bm->pol == 0) {
        const cplx v = u * cexp(I * (double)bm->lg_l * th);
        e[0] = v * cos(bm->pol_angle);
        e[1] = v * sin(bm->pol_angle);
    } else if (bm->pol == 1) {
        e[0] = u * cos(th);
        e[1] = u * sin(th);
    } else {
        e[0] = -u * sin(th);
        e[1] = u * cos(th);
    }
}

/* Transverse envelope component c of the incident beam at (x, y), with the
 * aberration phase: c = 0, 1 the x, y components of e_perp exp(ikW), c = 2, 3
 * those of b_perp exp(ikW), b_perp = (-z) x e_perp = (e_y, -e_x). */
static cplx envelope(const or_beam* bm, double k, double x, double y, int c)
{
    double es[3];
    beam_field(bm, x, y, es);
    cplx ph = cexp(I * k * beam_opd(bm, x, y));
    switch (c) {
    case 0: return es[0] * ph;
    case 1: return es[1] * ph;
    case 2: return es[1] * ph;
    default: return -es[0] * ph;
    }
}

/* d/dx of component cx plus d/dy of component cy, fourth-order central
 * differences of step h = 1e-3 w0 (truncation ~ h^4, far below FP64 needs) */
static cplx div_perp(const or_beam* bm, double k, double x, double y, int cx, int cy)
{
    const double h = 1e-3 * bm->w0;
    cplx dx = (-envelope(bm, k, x + 2 * h, y, cx) + 8.0 * envelope(bm, k, x + h, y, cx) -
               8.0 * envelope(bm, k, x - h, y, cx) + envelope(bm, k, x - 2 * h, y, cx)) / (12.0 * h);
    cplx dy = (-envelope(bm, k, x, y + 2 * h, cy) + 8.0 * envelope(bm, k, x, y + h, cy) -
               8.0 * envelope(bm, k, x, y - h, cy) + envelope(bm, k, x, y - 2 * h, cy)) / (12.0 * h);
    return dx + dy;
}

/* longitudinal terms of reading R14 without the phase exp(-ik(z + z_ref)) */
static void longitudinal(const or_beam* bm, double k, double x, double y, cplx* ez, cplx* bz)
{
    *ez = -(I / k) * div_perp(bm, k, x, y, 0, 1);
    *bz = -(I / k) * div_perp(bm, k, x, y, 2, 3);
}

/* beam power integral SS |f_E|^2 dA over the transverse plane (Eq. 16 with
 * Re(f_E x f_B*) . dA = |f_E|^2 dA for the collimated beam), by plain
 * trapezoid quadrature in rho on a fine grid -- deliberately numerical. */
double or_beam_power(const or_beam* bm)
{
    if (bm->profile >= 4) return -1.0; /* a caller's envelope or a dipole: no beam power */
    double rmax;
    if (bm->profile == 2) rmax = bm->w0;
    else rmax = 12.0 * bm->w0;
    int n = 400000;
    double h = rmax / n, s = 0.0;
    for (int i = 0; i <= n; ++i) {
        double rho = i * h;
        double v;
        if (bm->profile == 3) {
            /* at the waist plane the envelope does not depend on k */
            cplx e[2];
            lg_envelope(bm, 1.0, rho, 0.0, bm->z_waist, e);
            v = (creal(e[0] * conj(e[0])) + creal(e[1] * conj(e[1]))) * 2.0 * OR_PI * rho;
        } else {
            double e[3];
            beam_field(bm, rho, 0.0, e);
            v = (e[0] * e[0] + e[1] * e[1]) * 2.0 * OR_PI * rho;
        }
        s += (i == 0 || i == n) ? 0.5 * v : v;
    }
    return s * h;
}

/* ------------------------------------------------------------------------ */
/* Mirror geometry (Sec. III.A, Eq. 21).                                     */

static double surf_z(const or_mirror* m, double r)
{
    if (m->surface == 2) {
        const double a2 = m->c_ell * m->c_ell - m->e_ell * m->e_ell;
        return m->e_ell - m->c_ell * sqrt(1.0 - r * r / a2);
    }
    return (m->surface == 0) ? (r * r / (4.0 * m->f) - m->f) : m->z0;
}

/* reference of the incident phase: E_inc ~ exp(-ik(z + z_ref)) */
static double surf_zref(const or_mirror* m)
{
    if (m->surface == 2) return 2.0 * (m->c_ell - m->e_ell); /* -2 z_vertex */
    return (m->surface == 0) ? 2.0 * m->f : -m->z0;
}

/* unnormalised normal (-dz/dx, -dz/dy, 1); its length is the area factor */
static void surf_normal(const or_mirror* m, double x, double y, double nvec[3])
{
    if (m->surface == 2) {
        /* dz/dx = c x / (a^2 sqrt(1 - r^2/a^2)) */
        const double a2 = m->c_ell * m->c_ell - m->e_ell * m->e_ell;
        const double s = m->c_ell / (a2 * sqrt(1.0 - (x * x + y * y) / a2));
        nvec[0] = -x * s;
        nvec[1] = -y * s;
    } else if (m->surface == 0) {
        nvec[0] = -x / (2.0 * m->f);
        nvec[1] = -y / (2.0 * m->f);
    } else {
        nvec[0] = 0.0;
        nvec[1] = 0.0;
    }
    nvec[2] = 1.0;
}

/* ------------------------------------------------------------------------ */
/* Small complex-vector helpers.                                             */

static void ccross(const cplx a[3], const cplx b[3], cplx c[3])
{
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* ------------------------------------------------------------------------ */
/* One frequency, one observation point.                                     */

/* Eq. 11 (form 0) or Eq. 10 with the Appendix-A dyadic (form 1). */
/* env_s, env_r (nullable): the sampled envelope e_perp at this k for the
 * surface nodes [n_r][n_theta][2] and the rim nodes [edge][n_theta][2]
 * (profiles 3 and 4); NULL for the real profiles 0-2. */
static void field_at(const or_mirror* m, const or_beam* bm, int form, double k,
                     const double* gl_r, const double* gl_w, const double rp[3],
                     const cplx* env_s, const cplx* env_r, cplx E[3], cplx B[3])
{
    for (int c = 0; c < 3; ++c) { E[c] = 0.0; B[c] = 0.0; }
    const double dth = 2.0 * OR_PI / m->n_theta;
    const double zref = surf_zref(m);

    /* surface integrals */
    for (int i = 0; i < m->n_r; ++i) {
        double r = gl_r[i];
        for (int l = 0; l < m->n_theta; ++l) {
            double th = l * dth;
            double x = r * cos(th), y = r * sin(th), z = surf_z(m, r);
            double nv[3];
            surf_normal(m, x, y, nv);
            double nlen = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
            double nhat[3] = {nv[0] / nlen, nv[1] / nlen, nv[2] / nlen};
            /* dS = |N| r dr dtheta for z = F(r, theta) */
            double dS = nlen * r * gl_w[i] * dth;

            cplx es[2];
            if (env_s) {
                es[0] = env_s[2 * ((long)i * m->n_theta + l)];
                es[1] = env_s[2 * ((long)i * m->n_theta + l) + 1];
            } else {
                double er[3];
                beam_field(bm, x, y, er);
                es[0] = er[0];
                es[1] = er[1];
            }
            double W = beam_opd(bm, x, y);
            double d[3] = {x - rp[0], y - rp[1], z - rp[2]};
            double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            double Rh[3] = {d[0] / R, d[1] / R, d[2] / R};
            /* exp(ikR) of g and exp(-ik(z + z_ref)) exp(ikW) of E_inc, joined in
             * one exponential so that the FP64 phase keeps its accuracy */
            cplx ph = cexp(I * k * (R - (z + zref) + W));
            /* E_inc and B_inc = (-z) x E_inc at the node, with g's phase attached */
            cplx Einc[3] = {es[0] * ph, es[1] * ph, 0.0};
            cplx Binc[3] = {es[1] * ph, -es[0] * ph, 0.0};
            if (bm->order >= 1) {
                cplx ez, bz;
                longitudinal(bm, k, x, y, &ez, &bz);
                cplx pp = cexp(I * k * (R - (z + zref)));
                Einc[2] = ez * pp;
                Binc[2] = bz * pp;
            }
            if (bm->profile == 5) dipole_field(bm, k, x, y, z, R, Einc, Binc);
            cplx nh[3] = {nhat[0], nhat[1], nhat[2]};
            cplx J[3];
            ccross(nh, Binc, J); /* n x B_inc */
            double g0 = 1.0 / (4.0 * OR_PI * R); /* |g| */
            cplx dg = (I * k - 1.0 / R) * g0;    /* grad g = dg * Rhat */

            if (form == 0) {
                cplx sigma = nh[0] * Einc[0] + nh[1] * Einc[1] + nh[2] * Einc[2];
                for (int c = 0; c < 3; ++c)
                    E[c] += 2.0 * (I * k * J[c] * g0 + sigma * dg * Rh[c]) * dS;
            } else {
                /* (i/k) grad grad g . J with the Appendix-A dyadic */
                cplx a_iso = -(-I * k / R + 1.0 / (R * R)) * g0;
                cplx a_rr = (3.0 / (R * R) - 3.0 * I * k / R - k * k) * g0;
                cplx RJ = Rh[0] * J[0] + Rh[1] * J[1] + Rh[2] * J[2];
                for (int c = 0; c < 3; ++c)
                    E[c] += 2.0 * (I * k * J[c] * g0 +
                                   (I / k) * (a_iso * J[c] + a_rr * Rh[c] * RJ)) * dS;
            }
            cplx gg[3] = {dg * Rh[0], dg * Rh[1], dg * Rh[2]};
            cplx JxG[3];
            ccross(J, gg, JxG);
            for (int c = 0; c < 3; ++c) B[c] += 2.0 * JxG[c] * dS;
        }
    }

    /* boundary line integral of Eq. 11, -(2/ik) O grad g [n x (n x B_inc)] . dl */
    if (form == 0 && m->rim) {
        for (int edge = 0; edge < 2; ++edge) {
            double r = (edge == 0) ? m->r_max : m->r_min;
            double orient = (edge == 0) ? 1.0 : -1.0; /* reading R3 */
            if (r <= 0.0) continue;
            for (int l = 0; l < m->n_theta; ++l) {
                double th = l * dth;
                double x = r * cos(th), y = r * sin(th), z = surf_z(m, r);
                double nv[3];
                surf_normal(m, x, y, nv);
                double nlen = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
                cplx nh[3] = {nv[0] / nlen, nv[1] / nlen, nv[2] / nlen};
                /* tangent dP/dtheta = (-r sin, r cos, 0); dl = tangent * dtheta */
                double dl[3] = {-r * sin(th) * dth * orient, r * cos(th) * dth * orient, 0.0};

                cplx es[2];
                if (env_r) {
                    es[0] = env_r[2 * ((long)edge * m->n_theta + l)];
                    es[1] = env_r[2 * ((long)edge * m->n_theta + l) + 1];
                } else {
                    double er[3];
                    beam_field(bm, x, y, er);
                    es[0] = er[0];
                    es[1] = er[1];
                }
                double W = beam_opd(bm, x, y);
                double d[3] = {x - rp[0], y - rp[1], z - rp[2]};
                double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                double Rh[3] = {d[0] / R, d[1] / R, d[2] / R};
                cplx ph = cexp(I * k * (R - (z + zref) + W));
                cplx Binc[3] = {es[1] * ph, -es[0] * ph, 0.0};
                if (bm->order >= 1) {
                    cplx ez, bz;
                    longitudinal(bm, k, x, y, &ez, &bz);
                    Binc[2] = bz * cexp(I * k * (R - (z + zref)));
                }
                if (bm->profile == 5) {
                    cplx Ed[3];
                    dipole_field(bm, k, x, y, z, R, Ed, Binc);
                }
                cplx t1[3], t2[3];
                ccross(nh, Binc, t1);
                ccross(nh, t1, t2); /* n x (n x B_inc) */
                cplx proj = t2[0] * dl[0] + t2[1] * dl[1] + t2[2] * dl[2];
                cplx dg = (I * k - 1.0 / R) / (4.0 * OR_PI * R);
                for (int c = 0; c < 3; ++c) E[c] += -(2.0 / (I * k)) * dg * Rh[c] * proj;
            }
        }
    }
}

/*
 * Transverse envelope e_perp (complex x, y) of the incident beam at
 * arbitrary points and one k, without the phases exp(-ik(z + z_ref)) and
 * exp(ikW): R4's real profiles (0-2) or the Laguerre-Gauss mode (3).
 * Output e[n][2] complex as interleaved doubles.  Returns 0, or 1 for a
 * caller's envelope (4), which the caller already has.
 */
int or_envelope(const or_beam* bm, double k, int n, const double* xyz, double* e)
{
    if (bm->profile == 4) return 1;
    for (int j = 0; j < n; ++j) {
        cplx v[2];
        if (bm->profile == 3) {
            lg_envelope(bm, k, xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], v);
        } else {
            double er[3];
            beam_field(bm, xyz[3 * j], xyz[3 * j + 1], er);
            v[0] = er[0];
            v[1] = er[1];
        }
        for (int c = 0; c < 2; ++c) {
            e[4 * j + 2 * c] = creal(v[c]);
            e[4 * j + 2 * c + 1] = cimag(v[c]);
        }
    }
    return 0;
}

/*
 * Incident field E_inc, B_inc of readings R4 / R14 at arbitrary points for
 * n_omega frequencies (unit a_n), phase reference exp(-ik(z + z_ref)).
 * Layout as or_field's outputs.  Returns 0.
 */
int or_incident(const or_beam* bm, double zref, int n_omega, const double* omega, int n_pts,
                const double* pts, double* E_out, double* B_out)
{
    for (int n = 0; n < n_omega; ++n) {
        double k = 2.0 * OR_PI * omega[n];
        for (int p = 0; p < n_pts; ++p) {
            double x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
            double es[3];
            beam_field(bm, x, y, es);
            cplx ph = cexp(I * k * (beam_opd(bm, x, y) - (z + zref)));
            cplx E[3] = {es[0] * ph, es[1] * ph, 0.0}, B[3] = {es[1] * ph, -es[0] * ph, 0.0};
            if (bm->profile == 5) dipole_field(bm, k, x, y, z, 0.0, E, B);
            if (bm->order >= 1) {
                cplx ez, bz;
                longitudinal(bm, k, x, y, &ez, &bz);
                cplx pp = cexp(-I * k * (z + zref));
                E[2] = ez * pp;
                B[2] = bz * pp;
            }
            for (int c = 0; c < 3; ++c) {
                long o = 2 * (((long)n * n_pts + p) * 3 + c);
                E_out[o] = creal(E[c]);
                E_out[o + 1] = cimag(E[c]);
                B_out[o] = creal(B[c]);
                B_out[o + 1] = cimag(B[c]);
            }
        }
    }
    return 0;
}

/*
 * Reflected spectral field at n_pts observation points for n_omega
 * frequencies.  amp (nullable) holds complex a_n = E0^n exp(i phi) as
 * interleaved doubles; NULL means a_n = 1 (the spatial integrals alone).
 * form 0 = Eq. 11 (with its line integral when mirror->rim), form 1 = Eq. 10.
 * Returns 0 on success, nonzero on invalid input.
 */
int or_field(const or_mirror* m, const or_beam* bm, int form, int n_omega, const double* omega,
             const double* amp, int n_pts, const double* pts, double* E_out, double* B_out,
             int nthreads)
{
    if (m->n_r < 1 || m->n_theta < 1 || m->r_max <= m->r_min || m->r_min < 0.0) return 1;
    if (m->surface == 0 && m->f <= 0.0) return 1;
    if (m->surface == 2 && !(m->e_ell > 0.0 && m->e_ell < m->c_ell &&
                             m->r_max * m->r_max < m->c_ell * m->c_ell - m->e_ell * m->e_ell))
        return 1;
    if (bm->order >= 1 && bm->profile >= 2) return 1; /* needs a smooth real profile (R14) */
    if (bm->profile == 4 && !bm->env_fn) return 1;
    if (m->radial != 0 && (m->radial != 1 || m->n_r < 3 || m->n_r % 2 == 0)) return 1;
    double* gl_r = (double*)malloc(sizeof(double) * m->n_r);
    double* gl_w = (double*)malloc(sizeof(double) * m->n_r);
    if (m->radial == 1) or_simpson(m->n_r, m->r_min, m->r_max, gl_r, gl_w);
    else or_gauss_legendre(m->n_r, m->r_min, m->r_max, gl_r, gl_w);
    /* profiles 3 and 4: the envelope at every (omega, node), sampled up front
     * on this thread (a caller's function is not called from worker threads) */
    const long n_s = (long)m->n_r * m->n_theta, n_rim = 2L * m->n_theta, n_nd = n_s + n_rim;
    cplx* env = NULL;
    if (bm->profile == 3 || bm->profile == 4) {
        env = (cplx*)malloc(sizeof(cplx) * 2 * n_nd * n_omega);
        double* xyz = (double*)malloc(sizeof(double) * 3 * n_nd);
        double* e = (double*)malloc(sizeof(double) * 4 * n_nd);
        const double dth = 2.0 * OR_PI / m->n_theta;
        for (long j = 0; j < n_nd; ++j) {
            double r;
            long l;
            if (j < n_s) {
                r = gl_r[j / m->n_theta];
                l = j % m->n_theta;
            } else {
                r = ((j - n_s) / m->n_theta == 0) ? m->r_max : m->r_min;
                l = (j - n_s) % m->n_theta;
            }
            xyz[3 * j] = r * cos(l * dth);
            xyz[3 * j + 1] = r * sin(l * dth);
            xyz[3 * j + 2] = surf_z(m, r);
        }
        for (int n = 0; n < n_omega; ++n) {
            const double k = 2.0 * OR_PI * omega[n];
            cplx* en = env + 2 * n_nd * n;
            if (bm->profile == 3) {
                for (long j = 0; j < n_nd; ++j) lg_envelope(bm, k, xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], en + 2 * j);
            } else {
                bm->env_fn(bm->env_user, (int)n_nd, xyz, k, e);
                for (long j = 0; j < 2 * n_nd; ++j) en[j] = e[2 * j] + I * e[2 * j + 1];
            }
        }
        free(xyz);
        free(e);
    }
    long total = (long)n_omega * n_pts;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long idx = 0; idx < total; ++idx) {
        int n = (int)(idx / n_pts), p = (int)(idx % n_pts);
        double k = 2.0 * OR_PI * omega[n];
        cplx E[3], B[3];
        const cplx* es = env ? env + 2 * n_nd * n : NULL;
        field_at(m, bm, form, k, gl_r, gl_w, pts + 3 * p, es, es ? es + 2 * n_s : NULL, E, B);
        cplx a = 1.0;
        if (amp) a = amp[2 * n] + I * amp[2 * n + 1];
        for (int c = 0; c < 3; ++c) {
            cplx e = a * E[c], b = a * B[c];
            long o = 2 * ((idx) * 3 + c);
            E_out[o] = creal(e);
            E_out[o + 1] = cimag(e);
            B_out[o] = creal(b);
            B_out[o + 1] = cimag(b);
        }
    }
    free(env);
    free(gl_r);
    free(gl_w);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Spectrum (Sec. III.B, Eqs. 14-18; Sec. IV.B, Eq. 27).                     */

/* power spectrum per unit k, unnormalised */
static double spectrum_shape(int kind, double k, double fwhm_t, double lambda_c, double dlambda,
                             int sg_n)
{
    double kc = 2.0 * OR_PI / lambda_c;
    if (kind == 1) {
        /* Gaussian pulse of intensity FWHM fwhm_t: field spectrum
         * exp(-(k-kc)^2 tau^2 / (8 ln 2)), power its square */
        double s = exp(-(k - kc) * (k - kc) * fwhm_t * fwhm_t / (8.0 * log(2.0)));
        return s * s;
    }
    if (kind == 2) {
        /* Eq. 27 with the minus sign (reading R5), times |d lambda/dk| */
        if (k <= 0.0) return 0.0;
        double lam = 2.0 * OR_PI / k;
        double u = (lam - lambda_c) / dlambda;
        return exp(-pow(u * u, (double)sg_n)) * lam * lam / (2.0 * OR_PI);
    }
    return 0.0;
}

/*
 * Complex amplitudes a_n = E0^n exp(i phi(k_n)) at the given omegas.
 * kind: 0 monochromatic (E0 = 1), 1 Gaussian in time, 2 super-Gaussian in
 * lambda, 3 sampled (amp_in holds the amplitudes).  For kinds 1 and 2 the
 * power spectrum is normalised to int eps(k) dk = energy (Eq. 17, by
 * numerical quadrature) and E0^n = sqrt(eps(k_n) / (4 pi P)) (Eq. 16) with
 * P = beam_power.  phi(k) = sum_j phi_j (k - kc)^j / j!  (Eq. 18).
 */
int or_spectrum(int kind, double fwhm_t, double lambda_c, double dlambda, int sg_n, double energy,
                double beam_power, int n_phi, const double* phi, int n, const double* omega,
                const double* amp_in, double* amp_out)
{
    double kc = 2.0 * OR_PI / lambda_c;
    double norm = 1.0;
    if (kind == 1 || kind == 2) {
        /* trapezoid over a wide k window */
        double k_lo = 1e-3 * kc, k_hi = 6.0 * kc;
        int m = 2000000;
        double h = (k_hi - k_lo) / m, s = 0.0;
        for (int i = 0; i <= m; ++i) {
            double v = spectrum_shape(kind, k_lo + i * h, fwhm_t, lambda_c, dlambda, sg_n);
            s += (i == 0 || i == m) ? 0.5 * v : v;
        }
        norm = s * h;
        if (!(norm > 0.0)) return 1;
    }
    for (int i = 0; i < n; ++i) {
        double k = 2.0 * OR_PI * omega[i];
        cplx a;
        if (kind == 0) a = 1.0;
        else if (kind == 3) a = amp_in[2 * i] + I * amp_in[2 * i + 1];
        else {
            double eps = energy * spectrum_shape(kind, k, fwhm_t, lambda_c, dlambda, sg_n) / norm;
            a = sqrt(eps / (4.0 * OR_PI * beam_power));
        }
        double ph = 0.0, term = 1.0;
        for (int j = 0; j < n_phi; ++j) {
            if (j > 0) term *= (k - kc) / j;
            ph += phi[j] * term;
        }
        a *= cexp(I * ph);
        amp_out[2 * i] = creal(a);
        amp_out[2 * i + 1] = cimag(a);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Semi-discrete inverse transform (Sec. III.B, Eq. 13).                      */
/* F(t) = sum_{n=-N..N} F_n exp(-i k_n t) dk over a real field, i.e.          */
/* 2 Re sum_{n>=1} F_n exp(-i k_n t) dk for positive k_n; dk = k_1 - k_0      */
/* (uniform grid) or 1 for a single frequency.                                */

int or_time_domain(int n_omega, const double* omega, long n_vals, const double* F, int n_t,
                   const double* t, double* out, int nthreads)
{
    double dk = (n_omega > 1) ? 2.0 * OR_PI * (omega[1] - omega[0]) : 1.0;
    long total = (long)n_t * n_vals;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(static)
#endif
    for (long idx = 0; idx < total; ++idx) {
        int m = (int)(idx / n_vals);
        long v = idx % n_vals;
        cplx s = 0.0;
        for (int n = 0; n < n_omega; ++n) {
            double k = 2.0 * OR_PI * omega[n];
            cplx Fn = F[2 * (n * n_vals + v)] + I * F[2 * (n * n_vals + v) + 1];
            s += Fn * cexp(-I * k * t[m]);
        }
        out[idx] = 2.0 * creal(s) * dk;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* First correction of the Liouville-Neumann series of the MFIE (Sec. II,   */
/* eq:theory.mfie; reading R17).                                             */
/*                                                                           */
/*   (1/2) J = J_inc + n x PV SS J x grad g dS,   J_inc = n x B_inc.         */
/*                                                                           */
/* The first term of the series is physical optics, J0 = 2 J_inc            */
/* (eq:theory.poa).  The next iterate is J1 = J0 + dJ with                   */
/*   dJ(r_t) = 2 n_t x PV SS J0(r) x grad g(r, r_t) dS(r),                   */
/* grad acting on the surface variable r (reading R1), n_t the unit normal   */
/* at the target r_t on the mirror.  Near r_t the integrand is O(1/R): both  */
/* n_t . (r - r_t) and n_t . J0(r) vanish like R on a smooth surface (J0 is  */
/* tangent at r), so the principal value is the ordinary improper integral.  */
/* It is taken in polar coordinates (rho, phi) about the target's projection */
/* (x_t, y_t) on the plane of the mirror's parametrisation z = F(x, y):      */
/* dS = |N| dx dy = |N| rho drho dphi, and the factor rho cancels the 1/R.   */
/* Each ray phi runs from the target to the rim r = r_max (a disk,           */
/* r_min = 0): Gauss-Legendre in rho on [0, rho_max(phi)], periodic          */
/* trapezoid in phi.  The field of the corrected current adds the field of   */
/* dJ to the physical-optics field; dJ does not come from a Maxwell          */
/* incident field, so its field is the general representation behind        */
/* Eq. 10 (Sancer's form with n x E = 0 and n x B = J),                       */
/*   E' += SS { ik dJ g + (i/k) grad grad g . dJ } dS,  B' += SS dJ x grad g dS, */
/* on the mirror's own quadrature nodes, with the Appendix-A dyadic.         */

/* SS J x grad g(r, r_t) dS for one source point: adds J x grad g * dS to acc.
 * The incident phase of J (phi_in) joins the phase of g in one exponential. */
static void mfie_term(double k, const double r[3], const double rt[3], const cplx Jt[3], double phi_in,
                      double dS, cplx acc[3])
{
    const double d[3] = {r[0] - rt[0], r[1] - rt[1], r[2] - rt[2]};
    const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    if (!(R > 0.0)) return; /* the target itself carries weight rho = 0 */
    const cplx dg = (I * k - 1.0 / R) * cexp(I * (k * R + phi_in)) / (4.0 * OR_PI * R);
    const cplx G[3] = {dg * d[0] / R, dg * d[1] / R, dg * d[2] / R};
    cplx c[3];
    ccross(Jt, G, c);
    for (int q = 0; q < 3; ++q) acc[q] += c[q] * dS;
}

/* PO current J0 = 2 n x B_inc at the mirror point above (x, y), without its
 * phase, which goes to phi_in: B_inc = (-z) x E_inc of reading R4. */
static void mfie_po_current(const or_mirror* m, const or_beam* bm, double k, double x, double y, cplx J[3],
                            double* phi_in, double* area)
{
    double nv[3];
    surf_normal(m, x, y, nv);
    const double nlen = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    double es[3];
    beam_field(bm, x, y, es);
    const cplx nh[3] = {nv[0] / nlen, nv[1] / nlen, nv[2] / nlen};
    const cplx Bt[3] = {es[1], -es[0], 0.0};
    cplx c[3];
    ccross(nh, Bt, c);
    for (int q = 0; q < 3; ++q) J[q] = 2.0 * c[q];
    const double z = surf_z(m, sqrt(x * x + y * y));
    *phi_in = k * (beam_opd(bm, x, y) - (z + surf_zref(m)));
    *area = nlen;
}

/* dJ at the mirror point above (xt, yt), polar rule of n_rho x n_phi points;
 * gx, gw: Gauss-Legendre nodes and weights on [0, 1]. */
static void mfie_dj(const or_mirror* m, const or_beam* bm, double k, double xt, double yt, int n_rho,
                    const double* gx, const double* gw, int n_phi, cplx dJ[3])
{
    const double rt[3] = {xt, yt, surf_z(m, sqrt(xt * xt + yt * yt))};
    double nv[3];
    surf_normal(m, xt, yt, nv);
    const double nlen = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    const cplx nt[3] = {nv[0] / nlen, nv[1] / nlen, nv[2] / nlen};
    cplx acc[3] = {0.0, 0.0, 0.0};
    const double dphi = 2.0 * OR_PI / n_phi;
    for (int j = 0; j < n_phi; ++j) {
        const double ux = cos(j * dphi), uy = sin(j * dphi);
        /* rho_max: |(xt, yt) + rho u| = r_max */
        const double b = xt * ux + yt * uy, c = xt * xt + yt * yt - m->r_max * m->r_max;
        const double rho_max = -b + sqrt(b * b - c);
        for (int i = 0; i < n_rho; ++i) {
            const double rho = rho_max * gx[i];
            const double x = xt + rho * ux, y = yt + rho * uy;
            cplx J[3];
            double phi_in, area;
            mfie_po_current(m, bm, k, x, y, J, &phi_in, &area);
            const double r[3] = {x, y, surf_z(m, sqrt(x * x + y * y))};
            mfie_term(k, r, rt, J, phi_in, area * rho * gw[i] * rho_max * dphi, acc);
        }
    }
    cplx c[3];
    ccross(nt, acc, c);
    for (int q = 0; q < 3; ++q) dJ[q] = 2.0 * c[q];
}

static int mfie_supported(const or_mirror* m, const or_beam* bm)
{
    if (m->r_min != 0.0 || m->n_r < 1 || m->n_theta < 1 || !(m->r_max > 0.0)) return 0;
    if (m->surface == 0 && !(m->f > 0.0)) return 0;
    return bm->profile <= 2 && bm->order == 0;
}

/* dJ at n_t targets (x, y) on the mirror for one wavenumber, out[n_t][3]
 * complex.  Returns 0, or 1 if the mirror or beam is not supported (an
 * annulus, a beam of order 1, profiles 3-5). */
int or_mfie_current(const or_mirror* m, const or_beam* bm, double k, int n_t, const double* xy, int n_rho,
                    int n_phi, double* out)
{
    if (!mfie_supported(m, bm) || n_rho < 1 || n_phi < 1) return 1;
    double* gx = (double*)malloc(sizeof(double) * n_rho);
    double* gw = (double*)malloc(sizeof(double) * n_rho);
    or_gauss_legendre(n_rho, 0.0, 1.0, gx, gw);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int t = 0; t < n_t; ++t) {
        cplx dJ[3];
        mfie_dj(m, bm, k, xy[2 * t], xy[2 * t + 1], n_rho, gx, gw, n_phi, dJ);
        for (int q = 0; q < 3; ++q) {
            out[6 * t + 2 * q] = creal(dJ[q]);
            out[6 * t + 2 * q + 1] = cimag(dJ[q]);
        }
    }
    free(gx);
    free(gw);
    return 0;
}

/* The physical-optics field (Eq. 11, or_field form 0) plus the field of the
 * first MFIE correction dJ, evaluated at the mirror's surface nodes (its
 * Gauss-Legendre x trapezoid rule) with the polar rule n_rho x n_phi.
 * Layouts and amp as or_field.  Returns 0, or nonzero on invalid input. */
int or_field_mfie(const or_mirror* m, const or_beam* bm, int n_omega, const double* omega, const double* amp,
                  int n_pts, const double* pts, int n_rho, int n_phi, double* E_out, double* B_out, int nthreads)
{
    if (!mfie_supported(m, bm) || n_rho < 1 || n_phi < 1) return 1;
    int rc = or_field(m, bm, 0, n_omega, omega, amp, n_pts, pts, E_out, B_out, nthreads);
    if (rc) return rc;
    const int nr = m->n_r, nt = m->n_theta;
    double* rr = (double*)malloc(sizeof(double) * nr);
    double* rw = (double*)malloc(sizeof(double) * nr);
    if (m->radial == 1) or_simpson(nr, m->r_min, m->r_max, rr, rw);
    else or_gauss_legendre(nr, m->r_min, m->r_max, rr, rw);
    double* gx = (double*)malloc(sizeof(double) * n_rho);
    double* gw = (double*)malloc(sizeof(double) * n_rho);
    or_gauss_legendre(n_rho, 0.0, 1.0, gx, gw);
    const long ns = (long)nr * nt;
    const double dth = 2.0 * OR_PI / nt;
    cplx* dJ = (cplx*)malloc(sizeof(cplx) * 3 * ns * n_omega);
    /* dJ at every surface node and frequency */
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long idx = 0; idx < ns * n_omega; ++idx) {
        const int n = (int)(idx / ns);
        const long s = idx % ns;
        const double r = rr[s / nt], th = (s % nt) * dth;
        mfie_dj(m, bm, 2.0 * OR_PI * omega[n], r * cos(th), r * sin(th), n_rho, gx, gw, n_phi, dJ + 3 * idx);
    }
    /* the field of dJ at the observation points */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (long idx = 0; idx < (long)n_omega * n_pts; ++idx) {
        const int n = (int)(idx / n_pts), p = (int)(idx % n_pts);
        const double k = 2.0 * OR_PI * omega[n];
        const double* rp = pts + 3 * p;
        cplx E[3] = {0.0, 0.0, 0.0}, B[3] = {0.0, 0.0, 0.0};
        for (long s = 0; s < ns; ++s) {
            const double r = rr[s / nt], th = (s % nt) * dth;
            const double x = r * cos(th), y = r * sin(th), z = surf_z(m, r);
            double nv[3];
            surf_normal(m, x, y, nv);
            const double dS = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]) * r * rw[s / nt] * dth;
            const cplx* J = dJ + 3 * ((long)n * ns + s);
            const double d[3] = {x - rp[0], y - rp[1], z - rp[2]};
            const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double Rh[3] = {d[0] / R, d[1] / R, d[2] / R};
            const cplx g = cexp(I * k * R) / (4.0 * OR_PI * R);
            const cplx a_iso = -(-I * k / R + 1.0 / (R * R)) * g;
            const cplx a_rr = (3.0 / (R * R) - 3.0 * I * k / R - k * k) * g;
            const cplx RJ = Rh[0] * J[0] + Rh[1] * J[1] + Rh[2] * J[2];
            const cplx dg = (I * k - 1.0 / R) * g;
            const cplx G[3] = {dg * Rh[0], dg * Rh[1], dg * Rh[2]};
            cplx JxG[3];
            ccross(J, G, JxG);
            for (int c = 0; c < 3; ++c) {
                E[c] += (I * k * J[c] * g + (I / k) * (a_iso * J[c] + a_rr * Rh[c] * RJ)) * dS;
                B[c] += JxG[c] * dS;
            }
        }
        const cplx a = amp ? amp[2 * n] + I * amp[2 * n + 1] : 1.0;
        for (int c = 0; c < 3; ++c) {
            const long o = 2 * (idx * 3 + c);
            E_out[o] += creal(a * E[c]);
            E_out[o + 1] += cimag(a * E[c]);
            B_out[o] += creal(a * B[c]);
            B_out[o + 1] += cimag(a * B[c]);
        }
    }
    free(dJ);
    free(gx);
    free(gw);
    free(rr);
    free(rw);
    return 0;
}

/* Pin of the MFIE operator itself on a sphere of radius a (a closed surface,
 * used only by the tests): K[J](r_t) = n_t x PV SS J(r) x grad g(r, r_t) dS
 * for the current J = (z x r^) (K0 = 1), evaluated at n_t targets (unit
 * vectors) in geodesic polar coordinates about each target: the angle psi
 * from the target (Gauss-Legendre on [0, pi], n_psi) and the azimuth around
 * it (trapezoid, n_phi); dS = a^2 sin psi dpsi dphi, whose sin psi cancels
 * the 1/R of the integrand.  out[n_t][3] complex.  Returns 0. */
int or_mfie_sphere_te1(double a, double k, int n_t, const double* tgt, int n_psi, int n_phi, double* out)
{
    double* gx = (double*)malloc(sizeof(double) * n_psi);
    double* gw = (double*)malloc(sizeof(double) * n_psi);
    or_gauss_legendre(n_psi, 0.0, OR_PI, gx, gw);
    const double dphi = 2.0 * OR_PI / n_phi;
    for (int t = 0; t < n_t; ++t) {
        const double* e3 = tgt + 3 * t;
        /* an orthonormal frame (e1, e2, e3) about the target direction */
        double h[3] = {1.0, 0.0, 0.0};
        if (fabs(e3[0]) > 0.9) { h[0] = 0.0; h[1] = 1.0; }
        double e1[3] = {h[1] * e3[2] - h[2] * e3[1], h[2] * e3[0] - h[0] * e3[2], h[0] * e3[1] - h[1] * e3[0]};
        const double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        for (int q = 0; q < 3; ++q) e1[q] /= l1;
        const double e2[3] = {e3[1] * e1[2] - e3[2] * e1[1], e3[2] * e1[0] - e3[0] * e1[2],
                              e3[0] * e1[1] - e3[1] * e1[0]};
        const double rt[3] = {a * e3[0], a * e3[1], a * e3[2]};
        cplx acc[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < n_phi; ++j) {
            const double cp = cos(j * dphi), sp = sin(j * dphi);
            for (int i = 0; i < n_psi; ++i) {
                const double ps = gx[i];
                double u[3];
                for (int q = 0; q < 3; ++q) u[q] = sin(ps) * (cp * e1[q] + sp * e2[q]) + cos(ps) * e3[q];
                const double r[3] = {a * u[0], a * u[1], a * u[2]};
                const cplx J[3] = {-u[1], u[0], 0.0}; /* z x r^ */
                mfie_term(k, r, rt, J, 0.0, a * a * sin(ps) * gw[i] * dphi, acc);
            }
        }
        const cplx nt[3] = {e3[0], e3[1], e3[2]};
        cplx c[3];
        ccross(nt, acc, c);
        for (int q = 0; q < 3; ++q) {
            out[6 * t + 2 * q] = creal(c[q]);
            out[6 * t + 2 * q + 1] = cimag(c[q]);
        }
    }
    free(gx);
    free(gw);
    return 0;
}
