// sc_field_direct.cu -- the direct FP32 field-sum kernel: chunks of up to
// 256 omegas (the grouped kernel of sc_field.cu takes larger ones).  The quadrature of Sec. II, Eq. 11 over
// the node table of the paraboloid (Eq. 21) with the compensated phase of
// Sec. III.C.1; see sc_field.cu for the summand and the shared structure.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sc_field_common.cuh"
#include "sc_internal.h"

namespace sc {

namespace {

// ------------------------------------------------------------------------
// Direct kernel: n_omega <= 256.  GP threads per point (1 to 32, all in one
// warp), each owning NB consecutive omegas (NB = ceil(n_omega / GP) up to 24
// omegas, so no omega slot is wasted beyond the last thread's; 8 for 25..32,
// 5 to 8 for 33..64; 8 on 16 and 32 threads for up to 128 and 256).  The CTA shares the bulk-copied node tiles; 256 threads, 256 / GP
// points per item.  The accumulation is the packed (FFMA2) form with the
// three-term phasor recurrence, as in the grouped kernel.
//   GP = 1: each thread computes the geometry and phasors of its pairs
//   itself (with so few omegas per pair a shared table would not pay for
//   warps of its own); with two or three omegas every phasor comes from the
//   MUFU directly, no rotation (19% and 9% faster than the recurrence).
//   GP > 1: the GP threads of a point (neighbouring lanes of one warp) share
//   the pair geometry instead of each computing it: per sub-tile of 2 GP
//   nodes, each thread computes two pairs' coefficients, rotation e^{i dk
//   Phi} and Phi into a row of the point's shared-memory area, and after a
//   warp barrier every thread reads all 2 GP rows and takes only its own
//   seed phasor (the MUFU sine and cosine of its first omega).  Per-pair
//   work per thread drops from a full pair to 2/GP of one plus a seed.

// Two CTAs per SM (three for NB = 2, 3): the 128-register cap costs the
// NB >= 6 instantiations a few spilled registers, but the doubled warp count
// hides latency better; measured 2-19% faster per class than one CTA per SM.
// Threads per CTA and CTAs per SM of a class.
__host__ __device__ constexpr int direct_threads(int NB, int GP) { return 256; }
__host__ __device__ constexpr int direct_min_blocks(int NB, int GP) { return (NB == 2 || NB == 3) ? 3 : 2; }

template <int NB, int GP>
__global__ void __launch_bounds__(direct_threads(NB, GP), direct_min_blocks(NB, GP)) field_direct_kernel(BatchLaunch b)
{
    constexpr int NT = direct_threads(NB, GP);
    constexpr bool kQFirst = GP >= 2 && !(GP == 8 && NB == 6);
    constexpr int PPI = NT / GP;  // points per item
    // shared pair rows (GP > 1): per point TS rows of 16 floats (10
    // coefficients, rotation, Phi, pad) and a 16-byte pad, so that the
    // points of one warp read from different banks
    constexpr int TS = GP < 32 ? 2 * GP : 32;  // nodes per sub-tile
    constexpr int RPT = TS / GP;               // rows computed by each thread
    constexpr int ROW = 16;
    constexpr int PSTRIDE = TS * ROW + 4;
    // Loop unrolling, measured per class: the shared rows of a sub-tile 4
    // deep for NB <= 4 and 2 deep for NB = 5, 6 (so the next row's loads and
    // seed overlap this row's evaluations: 1-3% faster), not at all for
    // NB = 7, 8 (2-5% slower: their registers are already at the cap); the
    // nodes of a one-thread-per-point tile 2 deep for NB = 1, 2, 4 (3-8%
    // faster; 3-7% slower for NB = 3, 7, whose extra registers spill).
    constexpr int kRowUnroll = NB <= 4 ? 4 : (NB <= 6 ? 2 : 1);
    constexpr int kNodeUnroll = (NB == 1 || NB == 2 || NB == 4) ? 2 : 1;
    __shared__ __align__(16) float rows[GP > 1 ? PPI * PSTRIDE : 4];
    __shared__ __align__(128) float nodebuf[2 * kTileFloats];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ long long slot;
    __shared__ int abort_word;
    // per node buffer: warps done with it (mod 8) and copies issued into it this item
    __shared__ unsigned s_arrive[2], s_issued[2];
    constexpr unsigned kWarps = NT / 32;
    constexpr bool kLastWarpRefill = !(NB == 1 && GP == 1);
    static_assert((kWarps & (kWarps - 1)) == 0, "warps per CTA must be a power of two");
    volatile int* s_abort = &abort_word;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        s_arrive[0] = s_arrive[1] = 0;
        *s_abort = 0;
        mbar_fence_init();
    }
    bool timed_out = false;
    long long tbase = 0;
    for (long long item = next_item(b, &slot, -1, s_abort); item < b.n_items;
         item = next_item(b, &slot, item, s_abort)) {
        const Item w = decode(b, item);
        const FieldLaunch& p = w.r->f;
        const int pt = w.pbi * PPI + tid / GP;
        const int g = tid % GP;
        const int split = w.split;
        int t0, t1;
        split_range(p, split, t0, t1);
        const double om0 = (double)p.om_hi0 + (double)p.om_lo0;
        const double dom = (double)p.dom_hi + (double)p.dom_lo;
        float4 P;
        load_point(p.pts, p.n_pts, pt, P);
        float kv[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) kv[j] = (float)(6.283185307179586 * (om0 + (double)(g * NB + j) * dom));
        const double wg = om0 + (double)(g * NB) * dom;  // first omega of this thread
        const float wgh = (float)wg, wgl = (float)(wg - (double)wgh);
        // every omega of the thread as a float-float pair (the two- and three-omega classes)
        float wjh[NB], wjl[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j) {
            const double wj = om0 + (double)(g * NB + j) * dom;
            wjh[j] = (float)wj;
            wjl[j] = (float)(wj - (double)wjh[j]);
        }
        const float d1h = p.dom_hi, d1l = p.dom_lo;
        const int nt = t1 - t0;
        // copies issued into each buffer this item: counted by thread 0 alone with
        // the per-tile barrier, in shared memory by whichever warp issues otherwise
        unsigned issued[2] = {0, 0}, waited[2] = {0, 0};
        if (tid == 0) {
            if constexpr (kLastWarpRefill) s_issued[0] = s_issued[1] = 0;
            for (int s = 0; s < 2 && s < nt; ++s) {
                if (skip_copy(b, item, s)) continue;
                const int nbi = (int)((tbase + s) & 1);
                mbar_expect_tx(&bar[nbi], kTileBytes);
                bulk_g2s(nodebuf + nbi * kTileFloats, p.nodes + (size_t)(t0 + s) * kTileFloats,
                         kTileBytes, &bar[nbi]);
                if constexpr (kLastWarpRefill) s_issued[nbi]++; else issued[nbi]++;
            }
        }
        AccX2 acc[NB];
#pragma unroll
        for (int j = 0; j < NB; ++j)
#pragma unroll
            for (int c = 0; c < kAcc / 2; ++c) acc[j].v[c] = make_float2(0.f, 0.f);
        const bool pt_ok = pt < p.n_pts && g * NB < p.n_omega;
        const int nb_ok = min(NB, p.n_omega - g * NB);
        auto fold_now = [&](bool first) {
            if (pt_ok) {
                float2* dst = p.ws + (((size_t)split * p.n_pts + pt) * (size_t)p.n_omega + (size_t)g * NB) * kAcc;
                fold<NB>(dst, acc, nb_ok, first);
            }
        };
        for (int it = 0; it < nt; ++it) {
            const long long tg = tbase + it;
            const int nbi = (int)(tg & 1);
            // only a wait that saw the copy land counts it as drained; after an
            // abort the waits return at once and the item's rest is discarded
            if (field_wait(&bar[nbi], (unsigned)((tg >> 1) & 1), s_abort, b.abort, timed_out) == WAIT_DONE &&
                tid == 0)
                waited[nbi]++;
            const float* nb = nodebuf + nbi * kTileFloats;
            // one pair's evaluations from its coefficients co[0..9], rotation and Phi;
            // with shared pair rows (GP > 1) adding U q before V z is 0.7-3.4%
            // faster per class (2.4% at 256 omegas), except for 8 threads of 6
            // omegas (1.9% slower); one thread per point keeps V z first
            auto pair_evals = [&](const float co[10], float2 rot, float phi) {
                const float2 cp[10] = {make_float2(co[0], co[0]), make_float2(co[1], co[1]),
                                       make_float2(co[2], co[2]), make_float2(co[3], co[3]),
                                       make_float2(co[4], co[4]), make_float2(co[5], co[5]),
                                       make_float2(co[6], co[6]), make_float2(co[7], co[7]),
                                       make_float2(co[8], co[8]), make_float2(-co[9], -co[9])};
                const float2 pe = phasor_2wphi_mufu(wgh, wgl, phi);
                if (NB == 1) {
                    eval_x2<kQFirst>(acc[0], cp, kv[0], pe);
                } else {
                    const float2 cc = make_float2(2.f * rot.x, 2.f * rot.x);
                    const float2 ncc = make_float2(-2.f * rot.x, -2.f * rot.x);
                    float2 p0 = pe;
                    float2 p1 = cmul(pe, rot);
                    eval_x2<kQFirst>(acc[0], cp, kv[0], p0);
                    eval_x2<kQFirst>(acc[1], cp, kv[1], p1);
#pragma unroll
                    for (int jj = 2; jj < NB; ++jj) {
                        const float2 pn = __ffma2_rn((jj & 1) ? cc : ncc, p1, p0);
                        eval_x2<kQFirst>(acc[jj], cp, kv[jj], pn);
                        p0 = p1;
                        p1 = pn;
                    }
                }
            };
            if constexpr (GP == 1 && (NB == 2 || NB == 3)) {
                // two or three omegas: each phasor straight from the MUFU (its error,
                // like the seed's, is a constant factor that does not compound),
                // cheaper than a sincospif rotation and the recurrence
#pragma unroll kNodeUnroll
                for (int j = 0; j < kTile; ++j) {
                    float co[10];
                    const float phi = pair_coefs(nb, j, P, co);
                    const float2 cp[10] = {make_float2(co[0], co[0]), make_float2(co[1], co[1]),
                                           make_float2(co[2], co[2]), make_float2(co[3], co[3]),
                                           make_float2(co[4], co[4]), make_float2(co[5], co[5]),
                                           make_float2(co[6], co[6]), make_float2(co[7], co[7]),
                                           make_float2(co[8], co[8]), make_float2(-co[9], -co[9])};
#pragma unroll
                    for (int jj = 0; jj < NB; ++jj) {
                        float2 ph = phasor_2wphi_mufu(wjh[jj], wjl[jj], phi);
                        if (jj & 2) ph = make_float2(-ph.x, -ph.y);  // the slot sign fold() removes
                        eval_x2<false>(acc[jj], cp, kv[jj], ph);
                    }
                }
            } else if constexpr (GP == 1) {
#pragma unroll kNodeUnroll
                for (int j = 0; j < kTile; ++j) {
                    float co[10];
                    const float phi = pair_coefs(nb, j, P, co);
                    const float2 rot = NB > 1 ? phasor_2wphi(d1h, d1l, phi) : make_float2(1.f, 0.f);
                    pair_evals(co, rot, phi);
                }
            } else {
                float* prow = rows + (tid / GP) * PSTRIDE;
#pragma unroll 1
                for (int j0 = 0; j0 < kTile; j0 += TS) {
                    // this thread's rows of the sub-tile
#pragma unroll
                    for (int h = 0; h < RPT; ++h) {
                        const int q = g + h * GP;
                        float co[10];
                        const float phi = pair_coefs(nb, j0 + q, P, co);
                        const float2 rot = phasor_2wphi(d1h, d1l, phi);
                        float4* r4 = reinterpret_cast<float4*>(prow + q * ROW);
                        r4[0] = make_float4(co[0], co[1], co[2], co[3]);
                        r4[1] = make_float4(co[4], co[5], co[6], co[7]);
                        r4[2] = make_float4(co[8], co[9], rot.x, rot.y);
                        r4[3] = make_float4(phi, 0.f, 0.f, 0.f);
                    }
                    __syncwarp();
#pragma unroll kRowUnroll
                    for (int q = 0; q < TS; ++q) {
                        const float4* r4 = reinterpret_cast<const float4*>(prow + q * ROW);
                        const float4 a0 = r4[0], a1 = r4[1], a2 = r4[2];
                        const float co[10] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w, a2.x, a2.y};
                        pair_evals(co, make_float2(a2.z, a2.w), r4[3].x);
                    }
                    __syncwarp();  // rows are rewritten by the next sub-tile
                }
            }
            if ((it + 1) % p.flush_tiles == 0 || it + 1 == nt) fold_now(it + 1 <= p.flush_tiles);
            // The last warp to finish this tile refills its buffer with tile it + 2:
            // no CTA-wide barrier per tile (0.3-4% faster per class, except one
            // omega per thread on its own, 4% slower, which keeps the barrier).  A
            // warp waits for every tile's copy to land, so none runs more than two
            // tiles ahead of the slowest, and the buffer's mbarrier parity cannot
            // alias.
            if constexpr (!kLastWarpRefill) {
                __syncthreads();
                if (tid == 0 && it + 2 < nt && !*s_abort && !skip_copy(b, item, it + 2)) {
                    fence_proxy_async();
                    mbar_expect_tx(&bar[nbi], kTileBytes);
                    bulk_g2s(nodebuf + nbi * kTileFloats, p.nodes + (size_t)(t0 + it + 2) * kTileFloats,
                             kTileBytes, &bar[nbi]);
                    issued[nbi]++;
                }
            } else {
                __syncwarp();
                if ((tid & 31) == 0) {
                    __threadfence_block();  // this warp's reads of the buffer come first
                    const unsigned n = atomicAdd(&s_arrive[nbi], 1u);
                    if ((n & (kWarps - 1)) == kWarps - 1 && it + 2 < nt && !*s_abort &&
                        !skip_copy(b, item, it + 2)) {
                        __threadfence_block();
                        fence_proxy_async();
                        mbar_expect_tx(&bar[nbi], kTileBytes);
                        bulk_g2s(nodebuf + nbi * kTileFloats, p.nodes + (size_t)(t0 + it + 2) * kTileFloats,
                                 kTileBytes, &bar[nbi]);
                        s_issued[nbi]++;
                    }
                }
            }
        }
        if constexpr (kLastWarpRefill) {
            __syncthreads();  // every copy of this item is issued (and counted) by now
            if (tid == 0) issued[0] = s_issued[0], issued[1] = s_issued[1];
        }
        if (tid == 0) {
            // drain (waits that ignore the abort flag, each bounded)
            for (int s = 0; s < 2; ++s)
                while (waited[s] < issued[s]) {
                    const long long first = tbase + ((s - (int)(tbase & 1)) & 1);
                    if (mbar_wait(&bar[s], (unsigned)(((first >> 1) + waited[s]) & 1)) != WAIT_DONE) {
                        timed_out = true;
                        break;
                    }
                    waited[s]++;
                }
        }
        if (nt == 0) fold_now(true);
        tbase += nt;
    }
    if (timed_out) atomicOr(b.err, ERR_TIMEOUT);
}

template <int NB, int GP>
int launch_direct(const BatchLaunch& b, int grid, cudaStream_t s)
{
    field_direct_kernel<NB, GP><<<grid, direct_threads(NB, GP), 0, s>>>(b);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

template <int NB, int GP>
void direct_shape(int device, int* ppc, int* slots)
{
    *ppc = direct_threads(NB, GP) / GP;
    *slots = resident(field_direct_kernel<NB, GP>, direct_threads(NB, GP), 0, device);
}

}  // namespace

void direct_field_shape(int cls, int device, int* ppc, int* slots)
{
    switch (cls) {
    case 0: return direct_shape<1, 1>(device, ppc, slots);
    case 1: return direct_shape<2, 1>(device, ppc, slots);
    case 2: return direct_shape<3, 1>(device, ppc, slots);
    case 3: return direct_shape<4, 1>(device, ppc, slots);
    case 4: return direct_shape<5, 1>(device, ppc, slots);
    case 5: return direct_shape<6, 1>(device, ppc, slots);
    case 6: return direct_shape<7, 1>(device, ppc, slots);
    case 7: return direct_shape<4, 2>(device, ppc, slots);
    case 8: return direct_shape<5, 2>(device, ppc, slots);
    case 9: return direct_shape<6, 2>(device, ppc, slots);
    case 10: return direct_shape<7, 2>(device, ppc, slots);
    case 11: return direct_shape<8, 2>(device, ppc, slots);
    case 12: return direct_shape<5, 4>(device, ppc, slots);
    case 13: return direct_shape<6, 4>(device, ppc, slots);
    case 14: return direct_shape<8, 4>(device, ppc, slots);
    case 15: return direct_shape<5, 8>(device, ppc, slots);
    case 16: return direct_shape<6, 8>(device, ppc, slots);
    case 17: return direct_shape<7, 8>(device, ppc, slots);
    case 18: return direct_shape<8, 8>(device, ppc, slots);
    case 19: return direct_shape<8, 16>(device, ppc, slots);
    case 20: return direct_shape<8, 32>(device, ppc, slots);
    case 24: return direct_shape<8, 1>(device, ppc, slots);
    case 25: return direct_shape<3, 4>(device, ppc, slots);
    case 26: return direct_shape<4, 4>(device, ppc, slots);
    case 27: return direct_shape<3, 16>(device, ppc, slots);
    case 28: return direct_shape<4, 16>(device, ppc, slots);
    case 29: return direct_shape<4, 32>(device, ppc, slots);
    default: *ppc = 1; *slots = 1;
    }
}

int launch_direct_field(int cls, const BatchLaunch& b, int grid, cudaStream_t s)
{
    switch (cls) {
    case 0: return launch_direct<1, 1>(b, grid, s);
    case 1: return launch_direct<2, 1>(b, grid, s);
    case 2: return launch_direct<3, 1>(b, grid, s);
    case 3: return launch_direct<4, 1>(b, grid, s);
    case 4: return launch_direct<5, 1>(b, grid, s);
    case 5: return launch_direct<6, 1>(b, grid, s);
    case 6: return launch_direct<7, 1>(b, grid, s);
    case 7: return launch_direct<4, 2>(b, grid, s);
    case 8: return launch_direct<5, 2>(b, grid, s);
    case 9: return launch_direct<6, 2>(b, grid, s);
    case 10: return launch_direct<7, 2>(b, grid, s);
    case 11: return launch_direct<8, 2>(b, grid, s);
    case 12: return launch_direct<5, 4>(b, grid, s);
    case 13: return launch_direct<6, 4>(b, grid, s);
    case 14: return launch_direct<8, 4>(b, grid, s);
    case 15: return launch_direct<5, 8>(b, grid, s);
    case 16: return launch_direct<6, 8>(b, grid, s);
    case 17: return launch_direct<7, 8>(b, grid, s);
    case 18: return launch_direct<8, 8>(b, grid, s);
    case 19: return launch_direct<8, 16>(b, grid, s);
    case 20: return launch_direct<8, 32>(b, grid, s);
    case 24: return launch_direct<8, 1>(b, grid, s);
    case 25: return launch_direct<3, 4>(b, grid, s);
    case 26: return launch_direct<4, 4>(b, grid, s);
    case 27: return launch_direct<3, 16>(b, grid, s);
    case 28: return launch_direct<4, 16>(b, grid, s);
    case 29: return launch_direct<4, 32>(b, grid, s);
    default: return -(int)cudaErrorInvalidValue;
    }
}

}  // namespace sc
