// sc_reduce.cu -- FP64 cross-split reduction and epilogue of the FP32 path.
//
// The field kernels leave, per node table, split and (point, omega), the
// compensated float-float partials of the 12 sums of Sec. II Eq. 11's
// summand (E: U q + V z, B: Wv z) and a rim slot with the E sums of the
// boundary nodes.  One thread per (point, omega) adds the splits in FP64 in
// a fixed order (so results are deterministic), multiplies the rim sum by
// i/k_n (the factor of the line integral), and sums the node tables with
// their amplitudes a_n w_p(omega_n):
//     E = sum_p amp_p (S_p + (i/k) rim_p),   B = sum_p amp_p S_p^B.
#include <cuda_runtime.h>

#include "sc_internal.h"

namespace sc {

namespace {

// Sum one (point, omega) entry of a workspace over its surface splits (s)
// and read its rim slot (rim, the E sums only), in FP64, in split order.
__device__ __forceinline__ void section_sums(const float2* ws, int n_splits, size_t stride, size_t at,
                                             double s[kAcc], double rim[6])
{
#pragma unroll
    for (int c = 0; c < kAcc; ++c) s[c] = 0.0;
    const float2* base = ws + at;
    for (int sp = 0; sp < n_splits; ++sp) {
        const float4* v = reinterpret_cast<const float4*>(base + sp * stride);
#pragma unroll
        for (int c = 0; c < kAcc / 2; ++c) {
            const float4 h = v[c];
            s[2 * c] += (double)h.x + (double)h.y;
            s[2 * c + 1] += (double)h.z + (double)h.w;
        }
    }
    const float4* v = reinterpret_cast<const float4*>(base + (size_t)n_splits * stride);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float4 h = v[c];
        rim[2 * c] = (double)h.x + (double)h.y;
        rim[2 * c + 1] = (double)h.z + (double)h.w;
    }
}

__device__ __forceinline__ void reduce_one(const ReduceLaunch& r, long long idx)
{
    const int pt = (int)(idx / r.n_omega), n = (int)(idx % r.n_omega);
    const size_t stride = (size_t)r.n_pts * r.n_omega * kAcc;
    const size_t at = ((size_t)pt * r.n_omega + n) * kAcc;
    const double ik = 1.0 / r.kval[n];
    double er[3] = {0, 0, 0}, ei[3] = {0, 0, 0}, br[3] = {0, 0, 0}, bi[3] = {0, 0, 0};
    for (int p = 0; p < r.n_parts; ++p) {
        double s[kAcc], rim[6];
        section_sums(r.ws + (size_t)p * (r.n_splits + 1) * stride, r.n_splits, stride, at, s, rim);
        const double ar = r.amp[p * r.amp_stride + 2 * n], ai = r.amp[p * r.amp_stride + 2 * n + 1];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            // T = S + (i/k) rim: the rim slot's E sum carries the factor i/k
            // of the line integral; the part adds amp_p T
            const double tr = s[2 * c] - ik * rim[2 * c + 1], ti = s[2 * c + 1] + ik * rim[2 * c];
            er[c] += ar * tr - ai * ti;
            ei[c] += ar * ti + ai * tr;
            const double ur = s[6 + 2 * c], ui = s[6 + 2 * c + 1];
            br[c] += ar * ur - ai * ui;
            bi[c] += ar * ui + ai * ur;
        }
    }
    float2* E = r.E + (size_t)n * r.out_pt_stride_omega + (size_t)pt * 3;
#pragma unroll
    for (int c = 0; c < 3; ++c) E[c] = make_float2((float)er[c], (float)ei[c]);
    if (r.B) {
        float2* B = r.B + (size_t)n * r.out_pt_stride_omega + (size_t)pt * 3;
#pragma unroll
        for (int c = 0; c < 3; ++c) B[c] = make_float2((float)br[c], (float)bi[c]);
    }
}

__global__ void reduce_kernel(ReduceLaunch r)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (long long)r.n_pts * r.n_omega) return;
    reduce_one(r, idx);
}

__global__ void reduce_batch_kernel(const ReduceLaunch* reqs, int n_req, long long total)
{
    const long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= total) return;
    int lo = 0, hi = n_req - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (reqs[mid].off <= idx) lo = mid; else hi = mid - 1;
    }
    const ReduceLaunch& r = reqs[lo];
    reduce_one(r, idx - r.off);
}

}  // namespace

int launch_reduce_f32(const ReduceLaunch& r, cudaStream_t s)
{
    const long long total = (long long)r.n_pts * r.n_omega;
    const int nb = (int)((total + 255) / 256);
    reduce_kernel<<<nb, 256, 0, s>>>(r);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int launch_reduce_batch(const ReduceLaunch* reqs, int n_req, long long total, cudaStream_t s)
{
    if (total <= 0) return 0;
    reduce_batch_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(reqs, n_req, total);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace sc
