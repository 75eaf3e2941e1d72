// sc_mfie.cu -- the first correction beyond physical optics (FP64 kernels).
//
// Sec. II writes the current on a perfectly conducting mirror as the
// solution of the magnetic-field integral equation
//     (1/2) J = J_inc + n x PV SS J x grad g dS,      J_inc = n x B_inc,
// and solves it by its Liouville-Neumann series, whose first term is
// physical optics, J0 = 2 J_inc.  The next term adds
//     dJ(r_t) = 2 n_t x PV SS J0(r) x grad g(r, r_t) dS(r),
// grad acting on the surface variable r, g = e^{ikR} / (4 pi R).  On a
// smooth surface the integrand is only O(1/R) at the target (n_t . (r - r_t)
// and n_t . J0(r) both vanish like R), so the principal value is the
// improper integral; it is taken in polar coordinates (rho, phi) about the
// target's projection (x_t, y_t) on the plane of the mirror's
// parametrisation z = F(x, y), where dS = |N| rho drho dphi and the factor
// rho cancels the 1/R: Gauss-Legendre in rho from the target to the rim,
// periodic trapezoid in phi.  The incident field is evaluated at every polar
// point on the device (the collimated beams of the library: Gaussian,
// super-Gaussian or top-hat amplitude, linear, radial or azimuthal
// polarisation, Zernike optical path), since the rays meet the mirror
// between its quadrature nodes.
//
// The corrected current's field adds the field of dJ, which does not come
// from a Maxwell incident field, so it is Sancer's representation with
// n x E = 0 (the form of Eq. 10 for a general current):
//     E += SS { ik dJ g + (i/k) grad grad g . dJ } dS,   B += SS dJ x grad g dS,
// with the dyadic of Appendix A, on the mirror's own quadrature nodes.
//
// Both sums run in FP64: the phases k R between two mirror points are not
// compensated by any geometric identity (unlike the focal sum), and the
// correction is a small part of the field.
//
// Kernels:
//   mfie_current_kernel  one CTA per (target node, omega); its threads share
//                        the polar points and reduce with warp shuffles and
//                        one shared-memory step;
//   mfie_field_kernel    one thread per (point, omega); node tiles of (x, y,
//                        z, dS, dJ) are staged in shared memory and reused by
//                        the CTA's 256 points.
#include <cuda_runtime.h>
#include <stdint.h>

#include "sc_internal.h"

namespace sc {

namespace {

constexpr double kPi = 3.141592653589793;

struct C3 {
    double2 v[3];
};

__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Surface z = F(r) and the unnormalised normal N = (-F_x, -F_y, 1).
__device__ __forceinline__ void surface_at(const MfieLaunch& p, double x, double y, double& z, double& nx,
                                           double& ny)
{
    const double r2 = x * x + y * y;
    if (p.surface == 2) {
        const double a2 = p.c_ell * p.c_ell - p.e_ell * p.e_ell;
        const double q = sqrt(1.0 - r2 / a2);
        z = p.e_ell - p.c_ell * q;
        const double s = p.c_ell / (a2 * q);
        nx = -x * s;
        ny = -y * s;
    } else {
        z = r2 / (4.0 * p.f) - p.f;
        nx = -x / (2.0 * p.f);
        ny = -y / (2.0 * p.f);
    }
}

// Optical path difference W = sum_j c_j Z_j(u, v), u + iv = (x + iy)/r_norm:
// Z_j = N_j P_j(u^2 + v^2) {1, Re, Im}((u + iv)^|m|), coefficients of P_j
// (times c_j N_j) prepared on the host.
__device__ __forceinline__ double opd(const MfieLaunch& p, double x, double y)
{
    if (p.n_zern == 0) return 0.0;
    const double u = x / p.r_norm, v = y / p.r_norm, s = u * u + v * v;
    double W = 0.0;
    for (int j = 0; j < p.n_zern; ++j) {
        const MfieZern& z = p.zern[j];
        double P = 0.0;
        for (int d = z.deg; d >= 0; --d) P = fma(P, s, z.p[d]);
        double zr = 1.0, zi = 0.0;
        for (int m = 0; m < z.m; ++m) {
            const double t = zr * u - zi * v;
            zi = zr * v + zi * u;
            zr = t;
        }
        W += P * (z.kind == 0 ? 1.0 : (z.kind == 1 ? zr : zi));
    }
    return W;
}

// Transverse incident field e = A p at (x, y) (reading R4), no phase.
__device__ __forceinline__ void beam_e(const MfieLaunch& p, double x, double y, double& ex, double& ey)
{
    const double r2 = x * x + y * y;
    double A;
    if (p.profile == 0) A = exp(-r2 / (p.w0 * p.w0));
    else if (p.profile == 1) A = exp(-pow(r2 / (p.w0 * p.w0), (double)p.sg_order));
    else A = r2 <= p.w0 * p.w0 ? 1.0 : 0.0;
    if (p.pol == 0) {
        ex = A * p.cos_a;
        ey = A * p.sin_a;
    } else if (p.pol == 1) {  // rho_hat rho/w0 = (x, y)/w0
        ex = A * x / p.w0;
        ey = A * y / p.w0;
    } else {                  // theta_hat rho/w0 = (-y, x)/w0
        ex = -A * y / p.w0;
        ey = A * x / p.w0;
    }
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(256) mfie_current_kernel(MfieLaunch p)
{
    __shared__ double red[8][6];
    const int t = blockIdx.x, n = blockIdx.y;
    const double k = p.kval[n];
    const double4 gt = p.geo[t];
    const double xt = gt.x, yt = gt.y, zt = gt.z;
    const int n_pts = p.n_rho * p.n_phi;
    const double dphi = 2.0 * kPi / p.n_phi;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int q = threadIdx.x; q < n_pts; q += blockDim.x) {
        const int j = q / p.n_rho, i = q % p.n_rho;
        double uy, ux;
        sincospi(2.0 * j / p.n_phi, &uy, &ux);
        // rho_max: |(xt, yt) + rho u| = r_max
        const double b = xt * ux + yt * uy, c = xt * xt + yt * yt - p.r_max * p.r_max;
        const double rho_max = -b + sqrt(b * b - c);
        const double rho = rho_max * p.gx[i];
        const double x = xt + rho * ux, y = yt + rho * uy;
        double z, Nx, Ny;
        surface_at(p, x, y, z, Nx, Ny);
        const double nlen = sqrt(1.0 + Nx * Nx + Ny * Ny);
        double ex, ey;
        beam_e(p, x, y, ex, ey);
        // J0 = 2 n x B~, B~ = (e_y, -e_x, 0):  N x B~ = (e_x, e_y, -(N . e))
        const double s = 2.0 / nlen;
        const double J[3] = {s * ex, s * ey, -s * (Nx * ex + Ny * ey)};
        const double d[3] = {x - xt, y - yt, z - zt};
        const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        if (!(R > 0.0)) continue;
        const double iR = 1.0 / R;
        // e^{i(kR + k(W - z - zref))} (ik - 1/R) / (4 pi R) times the rule's weight
        double sn, cs;
        sincos(k * (R + opd(p, x, y) - (z + p.zref)), &sn, &cs);
        const double wgt = nlen * rho * p.gw[i] * rho_max * dphi * iR * iR / (4.0 * kPi);
        // dg R^ = (ik - 1/R) e^{i phi} / (4 pi R) * d / R
        const double gr = wgt * (-iR * cs - k * sn), gi = wgt * (-iR * sn + k * cs);
        // J x d (real), times (gr + i gi)
        const double cx = J[1] * d[2] - J[2] * d[1], cy = J[2] * d[0] - J[0] * d[2], cz = J[0] * d[1] - J[1] * d[0];
        acc[0] += cx * gr;
        acc[1] += cx * gi;
        acc[2] += cy * gr;
        acc[3] += cy * gi;
        acc[4] += cz * gr;
        acc[5] += cz * gi;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < 6; ++c) acc[c] = warp_sum(acc[c]);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < 6; ++c) red[warp][c] = acc[c];
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
#pragma unroll
        for (int c = 0; c < 6; ++c) acc[c] = warp_sum(lane < nw ? red[lane][c] : 0.0);
        if (lane == 0) {
            // dJ = 2 n_t x acc, n_t the unit normal at the target
            double z, Nx, Ny;
            surface_at(p, xt, yt, z, Nx, Ny);
            const double il = 1.0 / sqrt(1.0 + Nx * Nx + Ny * Ny);
            const double nt[3] = {Nx * il, Ny * il, il};
            C3 out;
            for (int h = 0; h < 2; ++h) {  // real, imaginary part
                const double a0 = acc[h], a1 = acc[2 + h], a2 = acc[4 + h];
                const double r0 = 2.0 * (nt[1] * a2 - nt[2] * a1);
                const double r1 = 2.0 * (nt[2] * a0 - nt[0] * a2);
                const double r2 = 2.0 * (nt[0] * a1 - nt[1] * a0);
                if (h == 0) {
                    out.v[0].x = r0; out.v[1].x = r1; out.v[2].x = r2;
                } else {
                    out.v[0].y = r0; out.v[1].y = r1; out.v[2].y = r2;
                }
            }
            C3* dst = reinterpret_cast<C3*>(p.dJ) + (size_t)n * p.n_surf + t;
            *dst = out;
        }
    }
}

constexpr int kFieldTile = 128;

__global__ void __launch_bounds__(256) mfie_field_kernel(MfieFieldLaunch p)
{
    __shared__ double4 sgeo[kFieldTile];
    __shared__ C3 sJ[kFieldTile];
    const int n = blockIdx.y;
    const int pt = blockIdx.x * blockDim.x + threadIdx.x;
    const double k = p.kval[n];
    double rx = 0, ry = 0, rz = 0;
    if (pt < p.n_pts) {
        rx = p.pts[3 * pt];
        ry = p.pts[3 * pt + 1];
        rz = p.pts[3 * pt + 2];
    }
    double E[6] = {0, 0, 0, 0, 0, 0}, B[6] = {0, 0, 0, 0, 0, 0};
    const C3* dJn = reinterpret_cast<const C3*>(p.dJ) + (size_t)n * p.n_surf;
    for (int s0 = 0; s0 < p.n_surf; s0 += kFieldTile) {
        const int ns = min(kFieldTile, p.n_surf - s0);
        __syncthreads();
        for (int i = threadIdx.x; i < ns; i += blockDim.x) {
            sgeo[i] = p.geo[s0 + i];
            sJ[i] = dJn[s0 + i];
        }
        __syncthreads();
        if (pt >= p.n_pts) continue;
        for (int i = 0; i < ns; ++i) {
            const double4 g4 = sgeo[i];
            const double d[3] = {g4.x - rx, g4.y - ry, g4.z - rz};
            const double R = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            const double iR = 1.0 / R;
            const double h[3] = {d[0] * iR, d[1] * iR, d[2] * iR};
            double sn, cs;
            sincos(k * R, &sn, &cs);
            const double2 g = make_double2(g4.w * cs * iR / (4.0 * kPi), g4.w * sn * iR / (4.0 * kPi));  // g dS
            // Appendix A: grad grad g = a_iso I + a_rr R^R^,
            //   a_iso = -(-ik/R + 1/R^2) g,  a_rr = (3/R^2 - 3ik/R - k^2) g
            const double2 a_iso = cmul(make_double2(-iR * iR, k * iR), g);
            const double2 a_rr = cmul(make_double2(3.0 * iR * iR - k * k, -3.0 * k * iR), g);
            const double2 dg = cmul(make_double2(-iR, k), g);  // (ik - 1/R) g
            const C3& J = sJ[i];
            const double2 RJ = make_double2(h[0] * J.v[0].x + h[1] * J.v[1].x + h[2] * J.v[2].x,
                                            h[0] * J.v[0].y + h[1] * J.v[1].y + h[2] * J.v[2].y);
            const double2 ikg = make_double2(-k * g.y, k * g.x);
            const double ik_inv = 1.0 / k;
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                // ik J g + (i/k)(a_iso J + a_rr R^ (R^ . J))
                const double2 t = cmul(a_iso, J.v[c]);
                const double2 u = cmul(a_rr, make_double2(h[c] * RJ.x, h[c] * RJ.y));
                const double2 dy = make_double2(-(t.y + u.y) * ik_inv, (t.x + u.x) * ik_inv);
                const double2 a = cmul(ikg, J.v[c]);
                E[2 * c] += a.x + dy.x;
                E[2 * c + 1] += a.y + dy.y;
            }
            // J x (dg R^)
            const int c1[3] = {1, 2, 0}, c2[3] = {2, 0, 1};
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const double2 p1 = cmul(J.v[c1[c]], make_double2(dg.x * h[c2[c]], dg.y * h[c2[c]]));
                const double2 p2 = cmul(J.v[c2[c]], make_double2(dg.x * h[c1[c]], dg.y * h[c1[c]]));
                B[2 * c] += p1.x - p2.x;
                B[2 * c + 1] += p1.y - p2.y;
            }
        }
    }
    if (pt >= p.n_pts) return;
    const double2 a = make_double2(p.amp[2 * n], p.amp[2 * n + 1]);
    const size_t o = (size_t)n * p.out_stride_omega + (size_t)pt * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const double2 e = cmul(a, make_double2(E[2 * c], E[2 * c + 1]));
        const double2 bb = cmul(a, make_double2(B[2 * c], B[2 * c + 1]));
        if (p.f64) {
            double2* Eo = reinterpret_cast<double2*>(p.E) + o + c;
            *Eo = make_double2(Eo->x + e.x, Eo->y + e.y);
            if (p.B) {
                double2* Bo = reinterpret_cast<double2*>(p.B) + o + c;
                *Bo = make_double2(Bo->x + bb.x, Bo->y + bb.y);
            }
        } else {
            float2* Eo = reinterpret_cast<float2*>(p.E) + o + c;
            *Eo = make_float2((float)((double)Eo->x + e.x), (float)((double)Eo->y + e.y));
            if (p.B) {
                float2* Bo = reinterpret_cast<float2*>(p.B) + o + c;
                *Bo = make_float2((float)((double)Bo->x + bb.x), (float)((double)Bo->y + bb.y));
            }
        }
    }
}

}  // namespace

int launch_mfie_current(const MfieLaunch& p, cudaStream_t s)
{
    if (p.n_surf < 1 || p.n_omega < 1) return 0;
    mfie_current_kernel<<<dim3((unsigned)p.n_surf, (unsigned)p.n_omega), 256, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int launch_mfie_field(const MfieFieldLaunch& p, cudaStream_t s)
{
    if (p.n_pts < 1 || p.n_omega < 1) return 0;
    mfie_field_kernel<<<dim3((unsigned)((p.n_pts + 255) / 256), (unsigned)p.n_omega), 256, 0, s>>>(p);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace sc
