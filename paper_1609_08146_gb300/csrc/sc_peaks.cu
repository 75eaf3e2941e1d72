// Arithmetic-unit throughput probes for the roofline of the field sum.
//
// The field sum of Eq. 11 is bound by the FP32 FMA pipe (the per-pair rsqrt,
// rcp and seed sincos use the MUFU pipe).  These kernels measure what each
// pipe sustains on this device with instruction streams that have nothing
// else in them: every thread runs kChains independent dependency chains, so
// latency is hidden and only issue and pipe throughput remain.  A value that
// is never true guards the final store, which keeps the chains live without
// writing anything.
#include <cuda_runtime.h>

#include "sc_internal.h"

namespace sc {
namespace {

constexpr int kChains = 8;
constexpr int kUnroll = 16;

// x <- x a + b: one FP32 FMA (one lane-op) per chain step.  With a < 1 the
// chains settle at b / (1 - a) and stay finite.
__global__ void __launch_bounds__(512) fma_probe_kernel(float* sink, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = 1e-3f * (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = fmaf(x[j], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// The packed form: one FFMA2 is two lane-ops.
__global__ void __launch_bounds__(512) fma2_probe_kernel(float* sink, int iters, float a, float b)
{
    float2 x[kChains / 2];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) x[j] = make_float2(1e-3f * (float)(threadIdx.x + j), 1e-3f * (float)j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kChains / 2; ++j) x[j] = __ffma2_rn(x[j], a2, b2);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains / 2; ++j) s += x[j].x + x[j].y;
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// x <- rsqrt(x): one MUFU operation per chain step (the fixed point is 1).
__device__ __forceinline__ float rsqrt_approx(float x)
{
    float y;
    asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__global__ void __launch_bounds__(512) mufu_probe_kernel(float* sink, int iters, float a, float b)
{
    float x[kChains];
#pragma unroll
    for (int j = 0; j < kChains; ++j) x[j] = a + b * (float)(threadIdx.x + j);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u)
#pragma unroll
            for (int j = 0; j < kChains; ++j) x[j] = rsqrt_approx(x[j]);
    }
    float s = 0.f;
#pragma unroll
    for (int j = 0; j < kChains; ++j) s += x[j];
    if (s == -1.0f) sink[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

int launch_alu_probe(int kind, int iters, float* sink, int grid, int block, cudaStream_t s)
{
    switch (kind) {
    case 0: fma_probe_kernel<<<grid, block, 0, s>>>(sink, iters, 0.999f, 1e-3f); break;
    case 1: fma2_probe_kernel<<<grid, block, 0, s>>>(sink, iters, 0.999f, 1e-3f); break;
    default: mufu_probe_kernel<<<grid, block, 0, s>>>(sink, iters, 1.5f, 1e-4f); break;
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

int alu_probe_grid(int kind, int device)
{
    int sms = 0, per_sm = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    if (kind == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel, 512, 0);
    else if (kind == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma2_probe_kernel, 512, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, mufu_probe_kernel, 512, 0);
    return (sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
}

long long alu_probe_ops_per_thread(int iters)
{
    return (long long)iters * kUnroll * kChains;
}

}  // namespace sc
