// sc_field.cu -- FP32 field-sum kernels of libsc (the hot path): the grouped
// kernel and the class dispatch; the direct kernel of requests with few
// omegas is in sc_field_direct.cu, their shared device helpers in
// sc_field_common.cuh.
//
// Computes, for every observation point r' and frequency omega_n, the
// quadrature of Sec. II Eq. 11 (physical-optics Stratton-Chu integrals after
// Stokes' theorem) over a node table of the paraboloid of Eq. 21.  Per node j
// the table holds P_j, |P_j|, the aberration W_j, J_j = (N x B~) w_j / (2 pi)
// and rho_j = (N . E~) w_j / (2 pi), where N = (-x/2f, -y/2f, 1) is the
// un-normalised normal (n dS = N r dr dtheta) and w_j the quadrature weight
// times r.  With R = |P - r'|, R^ = (P - r')/R and the phase
//     Phi = R - (z + 2f) + W = (|r'|^2 - 2 P.r') / (R + |P|) + W
// (|P| = z + 2f on the paraboloid, so the large distances cancel exactly --
// the phase-cancellation analysis of Sec. III.C.1, Eqs. 20-21), the incident
// phase e^{-ik(z+2f)} e^{ikW} times g = e^{ikR}/(4 pi R) is ph/(4 pi R) with
// ph = e^{ik Phi}, and the summand of Eq. 11 becomes
//     E += U q + V z,   B += Wv z,
//     q = ik ph,  z = (ik - 1/R) ph,
//     U = J/R,  V = rho R^/R,  Wv = U x R^.
// On the uniform omega grid the phasors of consecutive omegas follow the
// three-term recurrence ph_{n+1} = c ph_n - ph_{n-1}, c = 2 cos(dk Phi), one
// packed FMA (2 lane-ops) per step instead of a sincos; a thread's first two
// phasors come from its seed and one complex rotation e^{i dk Phi}.  With 8
// omegas per thread that is 2 lane-ops per evaluation for the phasor, plus 2
// for q, 2 for z, 12 for E and 6 for B: 24 FP32 pipe operations per (point,
// node, omega).
// Boundary (rim) nodes carry U = 0 and rho = (J . m^) dl / (2 pi); their E sum
// is multiplied by i/k_n in the epilogue, which reproduces the line integral
// -(2/ik) O grad g [n x (n x B_inc)] . dl of Eq. 11.
//
// Kernel structure (sm_103a):
//   * node tiles of 32 nodes (1280 B) are staged into shared memory with 1-D
//     bulk copies (cp.async.bulk + mbarrier, double buffered, bounded waits);
//   * phase 1: one thread per (point, node) pair computes the pair geometry,
//     the 12 coefficients, the rotation e^{i dk Phi} and the seed phasor of
//     every omega group, into a shared-memory pair table (double buffered);
//   * phase 2: thread (point, group) owns 8 consecutive omegas of one point
//     and runs the 24-op inner loop over the tile's nodes, accumulators in
//     registers (12 per omega);
//   * each CTA sums one split of the node range.  Every flush_tiles tiles
//     (2048 nodes by default) the FP32 register sums are folded into a
//     compensated float-float (hi, lo) partial in the workspace (TwoSum on
//     the FP32 pipe) and restarted, so no FP32 running sum grows long; the
//     reduce kernel adds the splits' partials in FP64 in a fixed order, so
//     the result is deterministic.  Splits exist for load balance only.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "sc_field_common.cuh"
#include "sc_internal.h"

namespace sc {

namespace {

// ------------------------------------------------------------------------
// Grouped kernel: G = ceil(n_omega / 8) >= 2 omega groups per point.
// Warp-specialised, 384 threads:
//   consumers  warps 0-7 (256 threads): thread (point pl, group g) owns 8
//              consecutive omegas of one point and runs only the 24-op loop;
//              PPC = 256 / TPP points per item, TPP = threads per point
//              (power of two >= G, <= 256);
//   producers  warps 8-11 (128 threads): stage node tiles with bulk copies and
//              build the pair table of the next compute tile (geometry,
//              coefficients, rotation, per-group seed phasors).
// Pair tables are double buffered; `full` mbarriers (128 producer arrivals)
// hand a table to the consumers and `empty` mbarriers (8 consumer-warp
// arrivals) hand it back.  Buffer indices and phase parities come from
// counters that run on across items, so the barriers are initialised once.
// Every wait is bounded.  Each 32-node tile is processed as CPT compute
// tiles of TC nodes so that two tables fit in shared memory for every TPP.

template <int TPP>
struct Grouped {
    static constexpr int NC = 256;                 // consumer threads
    static constexpr int NPROD = 128;              // producer threads
    static constexpr int NT = NC + NPROD;
    static constexpr int PPC = NC / TPP;
    static constexpr int TC = TPP == 2 ? 4 : (TPP == 4 ? 8 : (TPP <= 16 ? 16 : 32));
    static constexpr int CPT = kTile / TC;
    static constexpr int SEG = TPP >= 32 ? TPP / 32 : 1;  // seed segments of 32 groups per pair
    static constexpr int NPAIR = PPC * TC;
    static constexpr int NITEM = NPAIR * SEG;
    // floats per pair row: 10 duplicated pairs, rotation, rotation^2, pad to 28 so
    // that consecutive producer lanes store to different banks
    static constexpr int COEF = 28;
    // shared layout (bytes): node tiles | coefs | seeds | points | segment omegas | mbarriers | item
    static constexpr size_t OFF_NODE = 0;
    static constexpr size_t OFF_COEF = OFF_NODE + 2 * kTileBytes;
    static constexpr size_t COEF_BYTES = (size_t)NPAIR * COEF * 4;
    static constexpr size_t OFF_SEED = OFF_COEF + 2 * COEF_BYTES;
    // seed rows padded by one entry: producer lanes (consecutive pairs) write
    // rows TPP + 1 apart, so their stores fall in different banks
    static constexpr int SROW = TPP + 1;
    static constexpr size_t SEED_BYTES = (size_t)NPAIR * SROW * 8;
    static constexpr size_t OFF_PTS = OFF_SEED + 2 * SEED_BYTES;
    static constexpr size_t OFF_OMS = OFF_PTS + PPC * 16;
    static constexpr size_t NOMS = (TPP + 15) / 16;  // omegas of every 16th group (every 32nd used)
    static constexpr size_t OFF_BAR = (OFF_OMS + NOMS * 8 + 15) / 16 * 16;
    static constexpr size_t SMEM = OFF_BAR + 8 * 8;  // node[2], full[2], empty[2], item slot, abort
    static_assert(SMEM <= 227 * 1024, "shared memory");
    static_assert(NC % TPP == 0 && kTile % TC == 0, "shape");
};

template <int TPP>
__global__ void __launch_bounds__(Grouped<TPP>::NT, 1) field_grouped_kernel(BatchLaunch b)
{
    using L = Grouped<TPP>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* nodebuf = reinterpret_cast<float*>(smem + L::OFF_NODE);
    float* coefbuf = reinterpret_cast<float*>(smem + L::OFF_COEF);
    float2* seedbuf = reinterpret_cast<float2*>(smem + L::OFF_SEED);
    float4* spts = reinterpret_cast<float4*>(smem + L::OFF_PTS);
    float2* soms = reinterpret_cast<float2*>(smem + L::OFF_OMS);
    uint64_t* nbar = reinterpret_cast<uint64_t*>(smem + L::OFF_BAR);
    uint64_t* full = nbar + 2;
    uint64_t* empty = nbar + 4;
    long long* slot = reinterpret_cast<long long*>(nbar + 6);
    volatile int* s_abort = reinterpret_cast<volatile int*>(nbar + 7);

    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&nbar[0], 1);
        mbar_init(&nbar[1], 1);
        mbar_init(&full[0], L::NPROD);
        mbar_init(&full[1], L::NPROD);
        mbar_init(&empty[0], L::NC / 32);
        mbar_init(&empty[1], L::NC / 32);
        *s_abort = 0;
        mbar_fence_init();
    }
    bool timed_out = false;
    long long cbase = 0, tbase = 0;  // compute tiles and node tiles done by this CTA

    for (long long item = next_item(b, slot, -1, s_abort); item < b.n_items;
         item = next_item(b, slot, item, s_abort)) {
        const Item w = decode(b, item);
        const FieldLaunch& p = w.r->f;
        const int p0 = w.pbi * L::PPC;
        const int split = w.split;
        int t0, t1;
        split_range(p, split, t0, t1);
        const int G = (p.n_omega + kB - 1) / kB;
        const double om0 = (double)p.om_hi0 + (double)p.om_lo0;
        const double dom = (double)p.dom_hi + (double)p.dom_lo;
        const int nt = t1 - t0;        // bulk-copied tiles
        const int nct = nt * L::CPT;   // compute tiles

        for (int i = tid; i < L::PPC; i += L::NT) load_point(p.pts, p.n_pts, p0 + i, spts[i]);
        if (tid < (int)L::NOMS) {
            const double wv = om0 + (double)(tid * 16 * kB) * dom;
            const float hi = (float)wv;
            soms[tid] = make_float2(hi, (float)(wv - (double)hi));
        }
        __syncthreads();

        if (tid < L::NC) {
            // ---------------- consumers ----------------
            const int pl = tid / TPP;   // local point
            const int g = tid % TPP;    // omega group
            float kv[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j)
                kv[j] = (float)(6.283185307179586 * (om0 + (double)(g * kB + j) * dom));
            AccX2 acc[kB];
#pragma unroll
            for (int j = 0; j < kB; ++j)
#pragma unroll
                for (int c = 0; c < kAcc / 2; ++c) acc[j].v[c] = make_float2(0.f, 0.f);
            auto fold_now = [&](bool first) {
                if (p0 + pl < p.n_pts && g < G) {
                    float2* dst = p.ws + (((size_t)split * p.n_pts + (p0 + pl)) * (size_t)p.n_omega +
                                          (size_t)g * kB) * kAcc;
                    fold<kB>(dst, acc, min(kB, p.n_omega - g * kB), first);
                }
            };
            const int flush_ct = p.flush_tiles * L::CPT;
            for (int c = 0; c < nct; ++c) {
                const long long cg = cbase + c;
                const int pb = (int)(cg & 1);
                // after an abort this wait returns at once and the rest of the
                // item (microseconds of work on stale tables) is discarded
                field_wait(&full[pb], (unsigned)((cg >> 1) & 1), s_abort, b.abort, timed_out);
                const float* cb = coefbuf + (size_t)pb * L::NPAIR * L::COEF + (size_t)pl * L::TC * L::COEF;
                const float2* sb = seedbuf + (size_t)pb * L::NPAIR * L::SROW + (size_t)pl * L::TC * L::SROW + g;
#pragma unroll 1
                for (int j = 0; j < L::TC; ++j) {
                    const float4* c4 = reinterpret_cast<const float4*>(cb + j * L::COEF);
                    float2 cp[10];
                    float2 rot, cc, ncc;
                    {
                        const float4 a0 = c4[0], a1 = c4[1], a2 = c4[2], a3 = c4[3], a4 = c4[4], a5 = c4[5];
                        ncc = *reinterpret_cast<const float2*>(c4 + 6);
                        cp[0] = make_float2(a0.x, a0.y); cp[1] = make_float2(a0.z, a0.w);
                        cp[2] = make_float2(a1.x, a1.y); cp[3] = make_float2(a1.z, a1.w);
                        cp[4] = make_float2(a2.x, a2.y); cp[5] = make_float2(a2.z, a2.w);
                        cp[6] = make_float2(a3.x, a3.y); cp[7] = make_float2(a3.z, a3.w);
                        cp[8] = make_float2(a4.x, a4.y); cp[9] = make_float2(a4.z, a4.w);
                        rot = make_float2(a5.x, a5.y);
                        cc = make_float2(a5.z, a5.w);
                    }
                    // one phasor chain by the three-term recurrence; the phasors of
                    // slots 2, 3, 6, 7 carry a minus sign so that every step is a
                    // single FFMA2 with no negated operand (c' alternates -c, +c),
                    // and fold() takes the sign back out of those slots
                    float2 p0 = sb[j * L::SROW];
                    float2 p1 = cmul(p0, rot);
                    eval_x2<true>(acc[0], cp, kv[0], p0);
                    eval_x2<true>(acc[1], cp, kv[1], p1);
#pragma unroll
                    for (int jj = 2; jj < kB; ++jj) {
                        const float2 pn = __ffma2_rn((jj & 1) ? cc : ncc, p1, p0);
                        eval_x2<true>(acc[jj], cp, kv[jj], pn);
                        p0 = p1;
                        p1 = pn;
                    }
                }
                // hand the table back: one arrival per consumer warp, after the warp is done
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(&empty[pb]);
                if ((c + 1) % flush_ct == 0 || c + 1 == nct) fold_now(c + 1 <= flush_ct);
            }
            if (nct == 0) fold_now(true);  // e.g. the rim slot with the rim term off: zeros
        } else {
            // ---------------- producers ----------------
            const int ptid = tid - L::NC;
            const float d1h = p.dom_hi, d1l = p.dom_lo;
            unsigned issued[2] = {0, 0}, waited[2] = {0, 0};
            if (ptid == 0) {
                for (int s = 0; s < 2 && s < nt; ++s) {
                    if (skip_copy(b, item, s)) continue;
                    const int nbi = (int)((tbase + s) & 1);
                    mbar_expect_tx(&nbar[nbi], kTileBytes);
                    bulk_g2s(nodebuf + nbi * kTileFloats, p.nodes + (size_t)(t0 + s) * kTileFloats,
                             kTileBytes, &nbar[nbi]);
                    issued[nbi]++;
                }
            }
            for (int c = 0; c < nct; ++c) {
                const long long cg = cbase + c;
                const int pb = (int)(cg & 1);
                const int it = c / L::CPT, sub = c % L::CPT;
                const long long tg = tbase + it;
                const int nbi = (int)(tg & 1);
                if (sub == 0) {
                    // only a wait that saw the copy land counts it as drained
                    if (field_wait(&nbar[nbi], (unsigned)((tg >> 1) & 1), s_abort, b.abort, timed_out) == WAIT_DONE &&
                        ptid == 0)
                        waited[nbi]++;
                }
                // the table pb was last used for compute tile cg - 2
                if (cg >= 2) field_wait(&empty[pb], (unsigned)(((cg >> 1) - 1) & 1), s_abort, b.abort, timed_out);
                const float* nb = nodebuf + nbi * kTileFloats;
                float* cb = coefbuf + (size_t)pb * L::NPAIR * L::COEF;
                float2* sb = seedbuf + (size_t)pb * L::NPAIR * L::SROW;
                for (int i = ptid; i < L::NITEM; i += L::NPROD) {
                    const int q = i / L::SEG, seg = i % L::SEG;
                    const int pq = q / L::TC, j = q % L::TC;
                    float co[10];
                    const float phi = pair_coefs(nb, sub * L::TC + j, spts[pq], co);
                    const float2 rot = phasor_2wphi(d1h, d1l, phi);
                    if (seg == 0) {
                        const float c2 = 2.f * rot.x;
                        float4* c4 = reinterpret_cast<float4*>(cb + (size_t)q * L::COEF);
                        c4[0] = make_float4(co[0], co[0], co[1], co[1]);
                        c4[1] = make_float4(co[2], co[2], co[3], co[3]);
                        c4[2] = make_float4(co[4], co[4], co[5], co[5]);
                        c4[3] = make_float4(co[6], co[6], co[7], co[7]);
                        c4[4] = make_float4(co[8], co[8], -co[9], -co[9]);
                        // rotation, and (c, c), (-c, -c) for the three-term recurrence
                        c4[5] = make_float4(rot.x, rot.y, c2, c2);
                        *reinterpret_cast<float2*>(c4 + 6) = make_float2(-c2, -c2);
                    }
                    const int g0 = seg * 32, g1 = min(G, g0 + 32);
                    if (g0 < g1) {
                        // e^{i 8 dk Phi} as the cube of squarings of e^{i dk Phi}
                        float2 rotB = cmul(rot, rot);
                        rotB = cmul(rotB, rotB);
                        rotB = cmul(rotB, rotB);
                        float2 sd = make_float2(1.f, 0.f);
                        for (int gg = g0; gg < g1; ++gg) {
                            if ((gg & 31) == 0) {  // one direct seed per 32 groups
                                const float2 wv = soms[gg >> 4];
                                sd = phasor_2wphi(wv.x, wv.y, phi);
                            } else {
                                sd = cmul(sd, rotB);
                            }
                            sb[(size_t)q * L::SROW + gg] = sd;
                        }
                    }
                }
                mbar_arrive(&full[pb]);  // release: this thread's table entries are written
                // node tile it fully read by all producers: refill its buffer with tile it + 2
                if (sub == L::CPT - 1) {
                    asm volatile("bar.sync 1, %0;" ::"n"(L::NPROD) : "memory");
                    if (ptid == 0 && it + 2 < nt && !*s_abort && !skip_copy(b, item, it + 2)) {
                        fence_proxy_async();
                        mbar_expect_tx(&nbar[nbi], kTileBytes);
                        bulk_g2s(nodebuf + nbi * kTileFloats, p.nodes + (size_t)(t0 + it + 2) * kTileFloats,
                                 kTileBytes, &nbar[nbi]);
                        issued[nbi]++;
                    }
                }
            }
            // drain: never leave a bulk copy in flight into shared memory that is
            // reused or released; these waits ignore the abort flag (each is
            // bounded), and at most one issued copy per buffer is still pending
            if (ptid == 0) {
                for (int s = 0; s < 2; ++s)
                    while (waited[s] < issued[s]) {
                        // the k-th tile of this item in buffer s has global index first + 2k
                        const long long first = tbase + ((s - (int)(tbase & 1)) & 1);
                        if (mbar_wait(&nbar[s], (unsigned)(((first >> 1) + waited[s]) & 1)) != WAIT_DONE) {
                            timed_out = true;
                            break;
                        }
                        waited[s]++;
                    }
            }
        }
        cbase += nct;
        tbase += nt;
    }
    if (timed_out) atomicOr(b.err, ERR_TIMEOUT);
}

// ------------------------------------------------------------------------
// Launchers and shapes

template <int TPP>
int launch_grouped(const BatchLaunch& b, int grid, cudaStream_t s)
{
    using L = Grouped<TPP>;
    auto kern = field_grouped_kernel<TPP>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::SMEM);
    if (e != cudaSuccess) return -(int)e;
    kern<<<grid, L::NT, L::SMEM, s>>>(b);
    e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

template <int TPP>
void grouped_shape(int device, int* ppc, int* slots)
{
    using L = Grouped<TPP>;
    *ppc = L::PPC;
    *slots = resident(field_grouped_kernel<TPP>, L::NT, L::SMEM, device);
}

}  // namespace

int field_class(int n_omega)
{
    // 0..6   direct, 1 thread per point, NB = n_omega (1..7)
    // 7      direct, 2 threads per point, NB = 4 (8 omegas: with the shared
    //        pair rows 3% faster than 1 thread of 8; slower below 8)
    // 8..11  direct, 2 threads per point, NB = ceil(n_omega / 2) (5..8)
    // 12..13 direct, 4 threads per point, NB = ceil(n_omega / 4) (5..6)
    // 14     direct, 4 threads per point, NB = 8 (25..32 omegas)
    // 15..18 direct, 8 threads per point, NB = ceil(n_omega / 8) (5..8)
    // 19     direct, 16 threads per point, NB = 8 (65..128 omegas)
    // 20     direct, 32 threads per point, NB = 8 (129..256 omegas)
    //        (with the shared pair rows the direct kernel outruns the
    //        grouped kernel at every count up to 256 omegas)
    // 21..23 grouped, TPP = 64, 128, 256 threads per point (257..2048)
    if (n_omega <= 7) return std::max(1, n_omega) - 1;
    if (n_omega == 8) return 7;
    if (n_omega <= 16) return 8 + (n_omega + 1) / 2 - 5;
    if (n_omega <= 24) return 12 + (n_omega + 3) / 4 - 5;
    if (n_omega <= 32) return 14;
    if (n_omega <= 64) return 15 + (n_omega + 7) / 8 - 5;
    if (n_omega <= 128) return 19;
    if (n_omega <= 256) return 20;
    const int G = (n_omega + kB - 1) / kB;
    int cls = kFirstGroupedClass, tpp = 64;
    while (tpp < G) { tpp *= 2; ++cls; }
    return cls;
}

int alt_field_class(int n_omega)
{
    if (n_omega == 8) return 24;                         // 1 thread of 8
    if (n_omega >= 9 && n_omega <= 12) return 25;        // 4 threads of 3
    if (n_omega >= 13 && n_omega <= 16) return 26;       // 4 threads of 4
    if (n_omega >= 33 && n_omega <= 48) return 27;       // 16 threads of 3
    if (n_omega >= 49 && n_omega <= 64) return 28;       // 16 threads of 4
    if (n_omega >= 65 && n_omega <= 128) return 29;      // 32 threads of 4
    return -1;
}

void class_layout(int cls, int* tpp, int* opt)
{
    static const int kLayout[kNumClasses][2] = {
        {1, 1}, {1, 2}, {1, 3}, {1, 4}, {1, 5}, {1, 6}, {1, 7}, {2, 4},     // 0..7
        {2, 5}, {2, 6}, {2, 7}, {2, 8}, {4, 5}, {4, 6}, {4, 8},             // 8..14
        {8, 5}, {8, 6}, {8, 7}, {8, 8}, {16, 8}, {32, 8},                   // 15..20
        {64, 8}, {128, 8}, {256, 8},                                        // 21..23 grouped
        {1, 8}, {4, 3}, {4, 4}, {16, 3}, {16, 4}, {32, 4}};                 // 24..29
    const int c = cls < 0 || cls >= kNumClasses ? 0 : cls;
    *tpp = kLayout[c][0];
    *opt = kLayout[c][1];
}

void field_shape(int cls, int device, int* ppc, int* slots)
{
    if (is_direct_class(cls)) return direct_field_shape(cls, device, ppc, slots);
    switch (cls) {
    case 21: return grouped_shape<64>(device, ppc, slots);
    case 22: return grouped_shape<128>(device, ppc, slots);
    default: return grouped_shape<256>(device, ppc, slots);
    }
}

int launch_field_batch(int cls, const BatchLaunch& b, int grid, cudaStream_t s)
{
    if (grid < 1) return 0;
    if (is_direct_class(cls)) return launch_direct_field(cls, b, grid, s);
    switch (cls) {
    case 21: return launch_grouped<64>(b, grid, s);
    case 22: return launch_grouped<128>(b, grid, s);
    case 23: return launch_grouped<256>(b, grid, s);
    default: return -(int)cudaErrorInvalidValue;
    }
}

int launch_field_f32(const FieldLaunch& p, cudaStream_t s)
{
    const int cls = field_class(p.n_omega);
    int ppc = 1, slots = 1;
    int dev = 0;
    cudaGetDevice(&dev);
    field_shape(cls, dev, &ppc, &slots);
    BatchLaunch b{};
    b.reqs = nullptr;
    b.one.f = p;
    b.one.pb = (p.n_pts + ppc - 1) / ppc;
    b.one.cls = cls;
    b.one.item0 = 0;
    b.n_req = 1;
    b.n_items = (long long)b.one.pb * (p.n_splits + 1);
    b.queue = nullptr;
    b.err = p.err;
    b.abort = nullptr;  // grid mode: one item per CTA, nothing to stop early
    b.fail_tile = -1;
    return launch_field_batch(cls, b, (int)b.n_items, s);
}

namespace {

// One bounded wait on an mbarrier that nothing ever arrives on: the wait must
// give up after its wall-time limit and raise ERR_TIMEOUT.
__global__ void wait_selftest_kernel(int* err)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0 && mbar_wait(&bar, 0) != WAIT_DONE) atomicOr(err, ERR_TIMEOUT);
}

}  // namespace

int launch_wait_selftest(int* err, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(err);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 1 : -(int)e;
}

}  // namespace sc
