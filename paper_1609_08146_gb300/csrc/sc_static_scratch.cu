// sc_static_scratch.cu -- fixed, library-owned device scratch for the
// allocation-free evaluation entry point (sc_eval_fp32_static in sc.h).
//
// Some callers cannot allocate device memory at the moment they evaluate the
// field: code that runs while a stream is being captured into a CUDA graph in
// global capture mode, services that reserve all device memory up front into
// their own pools, or hosts that forbid allocation on their latency path.  For
// them the FP32 field sum can take its split partials from this file-scope
// array instead of a cudaMalloc'ed workspace.
//
// The array is static device memory of the library's module: every GPU that
// loads the library holds kStaticScratchBytes of it until the process exits.
// In host code its name is only a host-side stand-in for the symbol, never a
// device address, so the device address is looked up once per device, with
// that device current, by cudaGetSymbolAddress and then passed to kernels as a
// plain pointer.  The first lookup on a device may load the module; it should
// therefore happen before any stream capture begins.
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
        cudaError_t e = cudaSetDevice(device);
        if (e != cudaSuccess) return e;
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_static_scratch);
        if (e != cudaSuccess) return e;
        g_ptr[device] = p;
    }
    *ptr = g_ptr[device];
    return cudaSuccess;
}

}  // namespace sc
