// sc_f64_idft.cu -- the plain FP64 field sum and the inverse-transform stage.
//
// field_f64_kernel: the same quadrature of Sec. II Eq. 11 as the FP32 kernel,
// written the plain way: FP64 throughout, phase R - (z + 2f) + W formed by a
// direct difference and one sincos per (point, node, omega).  It is both a
// second parity check and the FP64 GPU baseline.  An incident with several
// node tables runs one launch per table, the later ones adding to E and B.
//
// idft: Sec. III.B Eq. 13 for a real field sampled at positive k_n,
// F(t_m) = 2 dk Re sum_n F_n e^{-i k_n t_m}, as a phasor table
// M[n][m] = e^{-i k_n t_m} (built in FP64, stored as float2) contracted with
// the spectra by a shared-memory tiled FP32 kernel.
#include <cuda_runtime.h>
#include <math.h>

#include "sc_internal.h"

namespace sc {

namespace {

__global__ void field_f64_kernel(Field64Launch a)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long total = (long long)a.n_pts * a.n_omega;
    if (idx >= total) return;
    const int n = (int)(idx / a.n_pts), pt = (int)(idx % a.n_pts);
    const double k = a.kval[n];
    const double x = a.pts[3 * pt], y = a.pts[3 * pt + 1], z = a.pts[3 * pt + 2];
    double sE[6] = {0, 0, 0, 0, 0, 0}, sB[6] = {0, 0, 0, 0, 0, 0}, sR[6] = {0, 0, 0, 0, 0, 0};
    for (int pass = 0; pass < 2; ++pass) {
        const Node64* nodes = pass == 0 ? a.surf : a.rim;
        const int nn = pass == 0 ? a.n_surf : a.n_rim;
        for (int j = 0; j < nn; ++j) {
            const Node64 nd = nodes[j];
            const double dx = nd.px - x, dy = nd.py - y, dz = nd.pz - z;
            const double R = sqrt(dx * dx + dy * dy + dz * dz);
            const double ir = 1.0 / R;
            const double phi = (R - nd.pn) + nd.w;
            double s, c;
            sincos(k * phi, &s, &c);
            const double qr = -k * s, qi = k * c;
            const double zr = qr - ir * c, zi = qi - ir * s;
            const double rx = dx * ir, ry = dy * ir, rz = dz * ir;
            const double ux = nd.jx * ir, uy = nd.jy * ir, uz = nd.jz * ir;
            const double av = nd.rho * ir;
            const double v[3] = {av * rx, av * ry, av * rz};
            const double u[3] = {ux, uy, uz};
            const double w[3] = {uy * rz - uz * ry, uz * rx - ux * rz, ux * ry - uy * rx};
            if (pass == 0) {
                for (int cc = 0; cc < 3; ++cc) {
                    sE[2 * cc] += u[cc] * qr + v[cc] * zr;
                    sE[2 * cc + 1] += u[cc] * qi + v[cc] * zi;
                    sB[2 * cc] += w[cc] * zr;
                    sB[2 * cc + 1] += w[cc] * zi;
                }
            } else {
                for (int cc = 0; cc < 3; ++cc) {
                    sR[2 * cc] += v[cc] * zr;
                    sR[2 * cc + 1] += v[cc] * zi;
                }
            }
        }
    }
    const double ar = a.amp[2 * n], ai = a.amp[2 * n + 1], ik = 1.0 / k;
    double2* E = a.E + ((size_t)n * a.n_pts + pt) * 3;
    // amp (S + (i/k) rim); later table parts add to the earlier ones
    for (int cc = 0; cc < 3; ++cc) {
        const double er = sE[2 * cc] - ik * sR[2 * cc + 1];
        const double ei = sE[2 * cc + 1] + ik * sR[2 * cc];
        double2 v = make_double2(ar * er - ai * ei, ar * ei + ai * er);
        if (a.accumulate) v = make_double2(v.x + E[cc].x, v.y + E[cc].y);
        E[cc] = v;
    }
    if (a.B) {
        double2* B = a.B + ((size_t)n * a.n_pts + pt) * 3;
        for (int cc = 0; cc < 3; ++cc) {
            const double br = sB[2 * cc], bi = sB[2 * cc + 1];
            double2 v = make_double2(ar * br - ai * bi, ar * bi + ai * br);
            if (a.accumulate) v = make_double2(v.x + B[cc].x, v.y + B[cc].y);
            B[cc] = v;
        }
    }
}

__global__ void phasor_kernel(const double* kval, int n_omega, const double* t, int n_t,
                              float2* M)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)n_omega * n_t) return;
    const int n = (int)(idx / n_t), m = (int)(idx % n_t);
    double s, c;
    sincos(kval[n] * t[m], &s, &c);
    M[idx] = make_float2((float)c, (float)-s);
}

__device__ __forceinline__ float2 load_c(const float2* F, size_t i) { return F[i]; }
__device__ __forceinline__ float2 load_c(const double2* F, size_t i)
{
    const double2 v = F[i];
    return make_float2((float)v.x, (float)v.y);
}

// out[m][v] = scale * sum_n Re(F[n][v] M[n][m]); 64 x 64 output tile per
// CTA (16 x 16 threads, 4 x 4 outputs each), 8 frequencies per smem stage.
template <typename T>
__global__ void __launch_bounds__(256) idft_kernel(const T* F, int n_omega, long long n_vals,
                                                   const float2* M, int n_t, float scale,
                                                   float* out, int accumulate)
{
    __shared__ float2 Ms[8][64];
    __shared__ float2 Fs[8][64];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    const int m0 = blockIdx.y * 64;
    const long long v0 = (long long)blockIdx.x * 64;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int n0 = 0; n0 < n_omega; n0 += 8) {
        for (int e = threadIdx.x; e < 8 * 64; e += 256) {
            const int nn = e / 64, c = e % 64;
            const int n = n0 + nn;
            const int m = m0 + c;
            const long long v = v0 + c;
            Ms[nn][c] = (n < n_omega && m < n_t) ? M[(size_t)n * n_t + m] : make_float2(0.f, 0.f);
            Fs[nn][c] = (n < n_omega && v < n_vals) ? load_c(F, (size_t)n * n_vals + v)
                                                    : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll
        for (int nn = 0; nn < 8; ++nn) {
            float2 mv[4], fv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) mv[i] = Ms[nn][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; ++j) fv[j] = Fs[nn][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    acc[i][j] = fmaf(fv[j].x, mv[i].x, fmaf(-fv[j].y, mv[i].y, acc[i][j]));
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + ty + 16 * i;
        if (m >= n_t) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const long long v = v0 + tx + 16 * j;
            if (v < n_vals) {
                float* o = out + (size_t)m * n_vals + v;
                *o = accumulate ? *o + scale * acc[i][j] : scale * acc[i][j];
            }
        }
    }
}

}  // namespace

int launch_field_f64(const Field64Launch& a, cudaStream_t s)
{
    const long long total = (long long)a.n_pts * a.n_omega;
    field_f64_kernel<<<(unsigned)((total + 127) / 128), 128, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int launch_idft(const IdftLaunch& p, cudaStream_t s)
{
    const long long nm = (long long)p.n_omega * p.n_t;
    phasor_kernel<<<(unsigned)((nm + 255) / 256), 256, 0, s>>>(p.kval, p.n_omega, p.t, p.n_t,
                                                               p.phasor);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return -(int)e;
    dim3 grid((unsigned)((p.n_vals + 63) / 64), (unsigned)((p.n_t + 63) / 64));
    const float scale = (float)(2.0 * p.dk);
    if (p.f64)
        idft_kernel<double2><<<grid, 256, 0, s>>>((const double2*)p.F, p.n_omega, p.n_vals,
                                                  p.phasor, p.n_t, scale, p.out, p.accumulate);
    else
        idft_kernel<float2><<<grid, 256, 0, s>>>((const float2*)p.F, p.n_omega, p.n_vals,
                                                 p.phasor, p.n_t, scale, p.out, p.accumulate);
    e = cudaGetLastError();
    return e == cudaSuccess ? 2 : -(int)e;
}

}  // namespace sc
