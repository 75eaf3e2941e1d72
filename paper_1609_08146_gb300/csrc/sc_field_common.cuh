// sc_field_common.cuh -- device helpers of the FP32 field-sum kernels
// (sc_field.cu: the grouped kernel, many omegas per point; sc_field_direct.cu:
// the direct kernel, few): mbarrier and bulk-copy wrappers with bounded
// waits, the reduced phasor e^{i pi x}, the pair geometry and coefficients of
// Eq. 11's summand, the packed accumulation step, the compensated fold, and
// the persistent work-item loop.  Included by those two files only.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sc_internal.h"

namespace sc {

namespace {

constexpr int kB = 8;                 // omegas per thread in the grouped kernel
constexpr unsigned kSpinLimit = 1u << 26;       // bounded mbarrier waits: polls
constexpr uint64_t kWaitNs = 1000000000ull;     // ... and wall time (1 s)
constexpr unsigned kSuspendNs = 20000;          // suspend-time hint per poll

// ------------------------------------------------------------------------
// mbarrier / bulk-copy helpers (inline PTX)

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_fence_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
            "r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void fence_proxy_async()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait on phase `parity`: gives up after about one second of wall
// time (or kSpinLimit polls) and returns WAIT_EXPIRED, so a copy or a
// hand-over that never lands turns into an error flag instead of a hung
// kernel.  With an abort flag (the CTA's shared word, set by the first of its
// waits that expires) the wait also returns WAIT_ABORTED as soon as the flag
// is set, so one expired wait ends every later one at once.  Each poll may
// suspend the warp for up to kSuspendNs until the phase completes, and the
// clock is read only every 64 polls, so waiting warps take few issue slots
// from working ones.
enum : int { WAIT_ABORTED = -1, WAIT_EXPIRED = 0, WAIT_DONE = 1 };

__device__ __forceinline__ int mbar_wait(uint64_t* bar, unsigned parity, const volatile int* abort = nullptr)
{
    const uint32_t addr = smem_u32(bar);
    uint64_t t0 = 0;
    for (unsigned it = 0; it < kSpinLimit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(addr), "r"(parity), "n"(kSuspendNs)
            : "memory");
        if (done) return WAIT_DONE;
        if (abort && *abort) return WAIT_ABORTED;
        if ((it & 63) == 0) {
            const uint64_t now = global_ns();
            if (it == 0) t0 = now;
            else if (now - t0 > kWaitNs) return WAIT_EXPIRED;
        }
    }
    return WAIT_EXPIRED;
}

// A main-loop wait of a field kernel: on expiry latch the CTA's abort flag
// and the launch's, and note the timeout for the error word.
__device__ __forceinline__ int field_wait(uint64_t* bar, unsigned parity, volatile int* s_abort, int* launch_abort,
                                          bool& timed_out)
{
    const int w = mbar_wait(bar, parity, s_abort);
    if (w == WAIT_EXPIRED) {
        *s_abort = 1;
        timed_out = true;
        if (launch_abort) atomicExch(launch_abort, 1);
    }
    return w;
}

// Failure-path test hook: leave this copy unissued (see BatchLaunch).
__device__ __forceinline__ bool skip_copy(const BatchLaunch& b, long long item, int tile)
{
    return b.fail_tile >= 0 && item == 0 && tile == b.fail_tile;
}

// ------------------------------------------------------------------------
// e^{i pi x} with x = 2 omega Phi, omega given as a float-float pair: the
// product keeps its rounding residual, and x is reduced by the nearest even
// integer n (e^{i pi x} has period 2) to r in [-1, 1] half-turns before
// sincospif; xh - n is exact (Sterbenz) since |xh - n| <= 1.

__device__ __forceinline__ float2 phasor_2wphi(float w_hi, float w_lo, float phi)
{
    const float a = 2.0f * w_hi;
    const float xh = a * phi;
    const float xl = fmaf(a, phi, -xh) + 2.0f * w_lo * phi;
    const float n = 2.0f * rintf(0.5f * xh);
    const float r = (xh - n) + xl;
    float s, c;
    sincospif(r, &s, &c);
    return make_float2(c, s);
}

// The same phasor from the MUFU sine and cosine (__sincosf, absolute error
// about 4e-7 on [-pi, pi], where the reduced argument pi r lies).  Used only
// for the direct kernel's seed, whose error is a constant factor on the
// phasors derived from it: it does not compound along the recurrence, unlike
// the rotation's, which stays on sincospif.  There the seed is a large share
// of the per-pair work (the small-omega classes got 2-27% faster).  The
// grouped kernel keeps sincospif for its seeds: with a MUFU seed one
// Laguerre-Gauss configuration of the seeded random tests went from under
// 5e-6 to 1.005e-5 of the gate metric, for 1.2% of speed.
__device__ __forceinline__ float2 phasor_2wphi_mufu(float w_hi, float w_lo, float phi)
{
    const float a = 2.0f * w_hi;
    const float xh = a * phi;
    const float xl = fmaf(a, phi, -xh) + 2.0f * w_lo * phi;
    const float n = 2.0f * rintf(0.5f * xh);
    const float r = (xh - n) + xl;
    float s, c;
    __sincosf(3.14159265358979f * r, &s, &c);
    return make_float2(c, s);
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}

// Pair geometry and coefficients from a staged tile (field f of node j at
// nb[f * 32 + j]) and a point (x, y, z, |r'|^2).  co[0..8] = U, V, Wv;
// co[9] = 1/R; returns Phi.
__device__ __forceinline__ float pair_coefs(const float* nb, int j, float4 pt, float co[10])
{
    const float px = nb[F_PX * kTile + j], py = nb[F_PY * kTile + j], pz = nb[F_PZ * kTile + j];
    const float pn = nb[F_PN * kTile + j], wo = nb[F_W * kTile + j];
    const float jx = nb[F_JX * kTile + j], jy = nb[F_JY * kTile + j], jz = nb[F_JZ * kTile + j];
    const float rho = nb[F_RHO * kTile + j];
    const float dx = px - pt.x, dy = py - pt.y, dz = pz - pt.z;
    const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    const float ir = rsqrtf(r2);
    const float R = r2 * ir;
    // |r'|^2 - 2 P.r'  (= R^2 - |P|^2 without the cancellation)
    const float D = fmaf(-2.0f * pt.x, px, fmaf(-2.0f * pt.y, py, fmaf(-2.0f * pt.z, pz, pt.w)));
    const float phi = __fdividef(D, R + pn) + wo;
    const float rx = dx * ir, ry = dy * ir, rz = dz * ir;
    const float ux = jx * ir, uy = jy * ir, uz = jz * ir;
    const float a = rho * ir;
    co[0] = ux; co[1] = uy; co[2] = uz;
    co[3] = a * rx; co[4] = a * ry; co[5] = a * rz;
    co[6] = fmaf(uy, rz, -uz * ry);
    co[7] = fmaf(uz, rx, -ux * rz);
    co[8] = fmaf(ux, ry, -uy * rx);
    co[9] = ir;
    return phi;
}

// One (point, node, omega) evaluation, packed: accumulators as (re, im) pairs
// and coefficients pre-duplicated as (c, c) pairs, so the 18 accumulation
// FMAs issue as 9 FFMA2 and z as one more: 22 FP32 lane-ops in 12 issued
// instructions, plus the phasor step.  QFIRST adds the U q term before the
// V z term so that it does not wait for z (the chain from the phasor to the
// last update of an E accumulator is three dependent steps instead of four):
// 2% faster in the grouped kernel, 10% slower in the direct kernel, whose
// register allocation it changes, so each kernel takes its faster order.
struct AccX2 {
    float2 v[6];  // E_x, E_y, E_z, B_x, B_y, B_z as (re, im)
};

template <bool QFIRST>
__device__ __forceinline__ void eval_x2(AccX2& a, const float2* cp, float k, float2 ph)
{
    const float2 q = make_float2(-k * ph.y, k * ph.x);  // q = ik ph
    const float2 z = __ffma2_rn(cp[9], ph, q);           // z = q - ph/R  (cp[9] = (-1/R, -1/R))
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        if (QFIRST)
            a.v[c] = __ffma2_rn(cp[3 + c], z, __ffma2_rn(cp[c], q, a.v[c]));
        else
            a.v[c] = __ffma2_rn(cp[c], q, __ffma2_rn(cp[3 + c], z, a.v[c]));
        a.v[3 + c] = __ffma2_rn(cp[6 + c], z, a.v[3 + c]);
    }
}

// Fold one thread's FP32 sums for omegas [n0, n0 + nb) into its compensated
// partials: (hi, lo) <- (hi, lo) + acc by TwoSum, or a plain store on the
// first fold.  Slots j with j & 2 set hold the negated sums (the sign that the
// phasor recurrence carries) and are folded with the sign taken out.  Each
// (split, point, omega) entry belongs to exactly one thread.
template <int NB>
__device__ __forceinline__ void fold(float2* dst, AccX2* acc, int nb, bool first)
{
#pragma unroll
    for (int j = 0; j < NB; ++j) {
        if (j < nb) {
            float4* d4 = reinterpret_cast<float4*>(dst + (size_t)j * kAcc);
            const float sg = (j & 2) ? -1.f : 1.f;  // sign carried by the phasor recurrence
            if (first) {
#pragma unroll
                for (int c = 0; c < kAcc / 2; ++c)
                    d4[c] = make_float4(sg * acc[j].v[c].x, 0.f, sg * acc[j].v[c].y, 0.f);
            } else {
                float4 h[kAcc / 2];
#pragma unroll
                for (int c = 0; c < kAcc / 2; ++c) h[c] = d4[c];  // six loads in flight together
#pragma unroll
                for (int c = 0; c < kAcc / 2; ++c) {
                    const float a0 = sg * acc[j].v[c].x, a1 = sg * acc[j].v[c].y;
                    const float s0 = h[c].x + a0, b0 = s0 - h[c].x;
                    const float e0 = (h[c].x - (s0 - b0)) + (a0 - b0);
                    const float s1 = h[c].z + a1, b1 = s1 - h[c].z;
                    const float e1 = (h[c].z - (s1 - b1)) + (a1 - b1);
                    d4[c] = make_float4(s0, h[c].y + e0, s1, h[c].w + e1);
                }
            }
            // one omega at a time: keeps the register footprint of the fold small
            asm volatile("" ::: "memory");
        }
#pragma unroll
        for (int c = 0; c < kAcc / 2; ++c) acc[j].v[c] = make_float2(0.f, 0.f);
    }
}

// Split -> node tile range.
__device__ __forceinline__ void split_range(const FieldLaunch& p, int split, int& t0, int& t1)
{
    if (split < p.n_splits) {
        t0 = split * p.tiles_per_split;
        t1 = min(t0 + p.tiles_per_split, p.n_surf_tiles);
    } else {
        t0 = p.n_surf_tiles;
        t1 = p.n_surf_tiles + p.n_rim_tiles;
    }
}

__device__ __forceinline__ void load_point(const double* pts, int n_pts, int p, float4& out)
{
    if (p < n_pts) {
        const double x = pts[3 * p], y = pts[3 * p + 1], z = pts[3 * p + 2];
        out = make_float4((float)x, (float)y, (float)z, (float)(x * x + y * y + z * z));
    } else {
        out = make_float4(0.f, 0.f, 0.f, 0.f);  // padding lane: computed, never stored
    }
}

// ------------------------------------------------------------------------
// Work items.  Every kernel below loops over work items (request, point
// block, split): in grid mode the item is blockIdx.x of a single request, in
// queue mode CTAs stay resident and take items from a device counter until
// the batch is exhausted (persistent scheduling across requests of uneven
// size).  Items of one request are numbered point block fastest, so CTAs that
// run at the same time share node tiles in L2.  The arithmetic of an item
// never depends on the other requests of a batch.

struct Item {
    const WorkReq* r;
    int pbi, split;
};

__device__ __forceinline__ const WorkReq* find_req(const BatchLaunch& b, long long item)
{
    if (!b.reqs) return &b.one;
    int lo = 0, hi = b.n_req - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (b.reqs[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    return &b.reqs[lo];
}

// next item for the whole CTA (thread 0 takes it, everyone reads it); none
// once this CTA or another of the launch has aborted on an expired wait
__device__ __forceinline__ long long next_item(const BatchLaunch& b, long long* slot, long long prev,
                                               const volatile int* s_abort)
{
    __syncthreads();  // everyone is done with the previous item (and its slot value)
    if (threadIdx.x == 0) {
        const bool stop = *s_abort || (b.abort && *(const volatile int*)b.abort);
        *slot = stop ? b.n_items
                     : (b.queue ? (long long)atomicAdd(b.queue, 1) : (prev < 0 ? (long long)blockIdx.x : b.n_items));
    }
    __syncthreads();
    return *slot;
}

__device__ __forceinline__ Item decode(const BatchLaunch& b, long long item)
{
    Item it;
    it.r = find_req(b, item);
    const long long local = item - it.r->item0;
    it.pbi = (int)(local % it.r->pb);
    it.split = (int)(local / it.r->pb);
    return it;
}

// ------------------------------------------------------------------------
// Resident CTAs of a kernel on the device (occupancy x SMs).

template <typename K>
int resident(K kern, int threads, size_t smem, int device)
{
    int per_sm = 0, sms = 0;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem) != cudaSuccess)
        per_sm = 1;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) sms = 1;
    cudaGetLastError();
    return std::max(1, per_sm) * std::max(1, sms);
}

}  // namespace

}  // namespace sc
