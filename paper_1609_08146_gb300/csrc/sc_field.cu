// sc_field.cu -- FP32 field-sum kernels of libsc (the hot path).
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
// Direct kernel: n_omega <= 48.  GP threads per point (1, 2, 4 or 8), each
// owning NB consecutive omegas (NB = ceil(n_omega / GP) up to 24 omegas, so
// no omega slot is wasted beyond the last thread's; 8 for 25..32, 5 or 6 for
// 33..48); every thread computes the geometry and the
// phasors of its pairs itself (no pair table: with so few omegas per pair a
// shared table would not pay for its producers), and the CTA shares the
// bulk-copied node tiles.  256 threads, 256 / GP points per item.  The
// accumulation is the packed (FFMA2) form with the three-term phasor
// recurrence, as in the grouped kernel.

// Two CTAs per SM (three for NB = 2, 3): the 128-register cap costs the
// NB >= 6 instantiations a few spilled registers, but the doubled warp count
// hides latency better; measured 2-19% faster per class than one CTA per SM.
template <int NB, int GP>
__global__ void __launch_bounds__(256, (NB == 2 || NB == 3) ? 3 : 2) field_direct_kernel(BatchLaunch b)
{
    constexpr int PPI = 256 / GP;  // points per item
    __shared__ __align__(128) float nodebuf[2 * kTileFloats];
    __shared__ __align__(8) uint64_t bar[2];
    __shared__ long long slot;
    __shared__ int abort_word;
    volatile int* s_abort = &abort_word;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
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
        const float d1h = p.dom_hi, d1l = p.dom_lo;
        const int nt = t1 - t0;
        unsigned issued[2] = {0, 0}, waited[2] = {0, 0};
        if (tid == 0) {
            for (int s = 0; s < 2 && s < nt; ++s) {
                if (skip_copy(b, item, s)) continue;
                const int nbi = (int)((tbase + s) & 1);
                mbar_expect_tx(&bar[nbi], kTileBytes);
                bulk_g2s(nodebuf + nbi * kTileFloats, p.nodes + (size_t)(t0 + s) * kTileFloats,
                         kTileBytes, &bar[nbi]);
                issued[nbi]++;
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
#pragma unroll 1
            for (int j = 0; j < kTile; ++j) {
                float co[10];
                const float phi = pair_coefs(nb, j, P, co);
                const float2 cp[10] = {make_float2(co[0], co[0]), make_float2(co[1], co[1]),
                                       make_float2(co[2], co[2]), make_float2(co[3], co[3]),
                                       make_float2(co[4], co[4]), make_float2(co[5], co[5]),
                                       make_float2(co[6], co[6]), make_float2(co[7], co[7]),
                                       make_float2(co[8], co[8]), make_float2(-co[9], -co[9])};
                float2 pe = phasor_2wphi_mufu(wgh, wgl, phi);
                if (NB == 1) {
                    eval_x2<false>(acc[0], cp, kv[0], pe);
                } else {
                    const float2 rot = phasor_2wphi(d1h, d1l, phi);
                    const float2 cc = make_float2(2.f * rot.x, 2.f * rot.x);
                    const float2 ncc = make_float2(-2.f * rot.x, -2.f * rot.x);
                    float2 p0 = pe;
                    float2 p1 = cmul(pe, rot);
                    eval_x2<false>(acc[0], cp, kv[0], p0);
                    eval_x2<false>(acc[1], cp, kv[1], p1);
#pragma unroll
                    for (int jj = 2; jj < NB; ++jj) {
                        const float2 pn = __ffma2_rn((jj & 1) ? cc : ncc, p1, p0);
                        eval_x2<false>(acc[jj], cp, kv[jj], pn);
                        p0 = p1;
                        p1 = pn;
                    }
                }
            }
            if ((it + 1) % p.flush_tiles == 0 || it + 1 == nt) fold_now(it + 1 <= p.flush_tiles);
            __syncthreads();
            if (tid == 0 && it + 2 < nt && !*s_abort && !skip_copy(b, item, it + 2)) {
                fence_proxy_async();
                mbar_expect_tx(&bar[nbi], kTileBytes);
                bulk_g2s(nodebuf + nbi * kTileFloats, p.nodes + (size_t)(t0 + it + 2) * kTileFloats,
                         kTileBytes, &bar[nbi]);
                issued[nbi]++;
            }
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

// ------------------------------------------------------------------------
// Launchers and shapes

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

template <int NB, int GP>
int launch_direct(const BatchLaunch& b, int grid, cudaStream_t s)
{
    field_direct_kernel<NB, GP><<<grid, 256, 0, s>>>(b);
    cudaError_t e = cudaGetLastError();
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
    // 0..7   direct, 1 thread per point, NB = n_omega (1..8)
    // 8..11  direct, 2 threads per point, NB = ceil(n_omega / 2) (5..8)
    // 12..13 direct, 4 threads per point, NB = ceil(n_omega / 4) (5..6)
    // 14     direct, 4 threads per point, NB = 8 (25..32 omegas; at two
    //        CTAs per SM it is 10% faster here than the grouped kernel with
    //        4 threads per point)
    // 15..16 direct, 8 threads per point, NB = 5, 6 (33..48 omegas, where
    //        the grouped kernel would leave 2 or 3 of its 8 threads idle)
    // 17..22 grouped, TPP = 8, 16, ..., 256 threads per point
    if (n_omega <= 8) return std::max(1, n_omega) - 1;
    if (n_omega <= 16) return 8 + (n_omega + 1) / 2 - 5;
    if (n_omega <= 24) return 12 + (n_omega + 3) / 4 - 5;
    if (n_omega <= 32) return 14;
    if (n_omega <= 48) return 15 + (n_omega + 7) / 8 - 5;
    const int G = (n_omega + kB - 1) / kB;
    int cls = 17, tpp = 8;
    while (tpp < G) { tpp *= 2; ++cls; }
    return cls;
}

namespace {

template <int NB, int GP>
void direct_shape(int device, int* ppc, int* slots)
{
    *ppc = 256 / GP;
    *slots = resident(field_direct_kernel<NB, GP>, 256, 0, device);
}

}  // namespace

void field_shape(int cls, int device, int* ppc, int* slots)
{
    switch (cls) {
    case 0: return direct_shape<1, 1>(device, ppc, slots);
    case 1: return direct_shape<2, 1>(device, ppc, slots);
    case 2: return direct_shape<3, 1>(device, ppc, slots);
    case 3: return direct_shape<4, 1>(device, ppc, slots);
    case 4: return direct_shape<5, 1>(device, ppc, slots);
    case 5: return direct_shape<6, 1>(device, ppc, slots);
    case 6: return direct_shape<7, 1>(device, ppc, slots);
    case 7: return direct_shape<8, 1>(device, ppc, slots);
    case 8: return direct_shape<5, 2>(device, ppc, slots);
    case 9: return direct_shape<6, 2>(device, ppc, slots);
    case 10: return direct_shape<7, 2>(device, ppc, slots);
    case 11: return direct_shape<8, 2>(device, ppc, slots);
    case 12: return direct_shape<5, 4>(device, ppc, slots);
    case 13: return direct_shape<6, 4>(device, ppc, slots);
    case 14: return direct_shape<8, 4>(device, ppc, slots);
    case 15: return direct_shape<5, 8>(device, ppc, slots);
    case 16: return direct_shape<6, 8>(device, ppc, slots);
    case 17: return grouped_shape<8>(device, ppc, slots);
    case 18: return grouped_shape<16>(device, ppc, slots);
    case 19: return grouped_shape<32>(device, ppc, slots);
    case 20: return grouped_shape<64>(device, ppc, slots);
    case 21: return grouped_shape<128>(device, ppc, slots);
    default: return grouped_shape<256>(device, ppc, slots);
    }
}

int launch_field_batch(int cls, const BatchLaunch& b, int grid, cudaStream_t s)
{
    if (grid < 1) return 0;
    switch (cls) {
    case 0: return launch_direct<1, 1>(b, grid, s);
    case 1: return launch_direct<2, 1>(b, grid, s);
    case 2: return launch_direct<3, 1>(b, grid, s);
    case 3: return launch_direct<4, 1>(b, grid, s);
    case 4: return launch_direct<5, 1>(b, grid, s);
    case 5: return launch_direct<6, 1>(b, grid, s);
    case 6: return launch_direct<7, 1>(b, grid, s);
    case 7: return launch_direct<8, 1>(b, grid, s);
    case 8: return launch_direct<5, 2>(b, grid, s);
    case 9: return launch_direct<6, 2>(b, grid, s);
    case 10: return launch_direct<7, 2>(b, grid, s);
    case 11: return launch_direct<8, 2>(b, grid, s);
    case 12: return launch_direct<5, 4>(b, grid, s);
    case 13: return launch_direct<6, 4>(b, grid, s);
    case 14: return launch_direct<8, 4>(b, grid, s);
    case 15: return launch_direct<5, 8>(b, grid, s);
    case 16: return launch_direct<6, 8>(b, grid, s);
    case 17: return launch_grouped<8>(b, grid, s);
    case 18: return launch_grouped<16>(b, grid, s);
    case 19: return launch_grouped<32>(b, grid, s);
    case 20: return launch_grouped<64>(b, grid, s);
    case 21: return launch_grouped<128>(b, grid, s);
    case 22: return launch_grouped<256>(b, grid, s);
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
