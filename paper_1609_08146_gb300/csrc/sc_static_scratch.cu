// sc_static_scratch.cu -- fixed, library-owned device scratch for the
// allocation-free evaluation entry point (sc_eval_fp32_static in sc.h).
//
// Some callers cannot allocate device memory at the moment they evaluate the
// field: services that reserve all device memory up front for their own pools
// (a cudaMalloc would fail or break their accounting), and real-time or
// latency-bound loops that forbid cudaMalloc and cudaFree because those calls
// can block on the whole device.  For them the FP32 field sum can take its
// split partials (and the wavenumbers k_n, written here by a small kernel)
// from this file-scope array instead of a cudaMalloc'ed workspace.
//
// The array is static device memory of the library's module: every GPU that
// loads the library holds kStaticScratchBytes of it until the process exits.
// In host code its name is only a host-side stand-in for the symbol, never a
// device address, so the device address is looked up once per device, with
// that device current, by cudaGetSymbolAddress and then passed to kernels as a
// plain pointer.  The first call of the entry point on a device does that
// lookup (which may load the module) and restores the caller's current
// device; that first call should come before any stream capture begins.
#include <cuda_runtime.h>

#include <mutex>

#include "sc_internal.h"

namespace sc {

namespace {

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_ptr[kMaxDevices] = {};

}  // namespace

cudaError_t static_scratch(int device, void** ptr)
{
    *ptr = nullptr;
    if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ptr[device]) {
        int prev = 0;
        cudaError_t e = cudaGetDevice(&prev);
        if (e != cudaSuccess) return e;
        e = cudaSetDevice(device);
        if (e != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        const cudaError_t e2 = cudaSetDevice(prev);  // the caller's device, as it was
        if (e != cudaSuccess) return e;
        if (e2 != cudaSuccess) return e2;
        g_ptr[device] = p;
    }
    *ptr = g_ptr[device];
    return cudaSuccess;
}

namespace {

// k_n = 2 pi (omega0 + n domega), the wavenumbers of the uniform grid, in FP64
__global__ void kgrid_kernel(double* k, double omega0, double domega, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) k[i] = 6.283185307179586 * (omega0 + (double)i * domega);
}

}  // namespace

int launch_kgrid(double* k, double omega0, double domega, int n, cudaStream_t s)
{
    if (n < 1) return 0;
    kgrid_kernel<<<(n + 255) / 256, 256, 0, s>>>(k, omega0, domega, n);
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace sc
