// sc_batch.cpp -- batched FP32 execution (A8): chunks, the split autotuner,
// persistent launches per kernel class, CUDA graphs and the batched reduce.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sc_host.h"

namespace sch {

// ------------------------------------------------------------------------
// Batched FP32 execution (A8): requests are cut into chunks (<= 2048 omegas,
// points bounded by the workspace cap); chunks of one kernel class run in one
// persistent launch whose CTAs take (chunk, point block, split) items from a
// device queue; one batched FP64 reduce finishes every chunk.  The field
// launches of a batch are captured into a CUDA graph and replayed while the
// launch signature repeats.  Each chunk's split count comes from the
// autotuner cache (or the heuristic), never from the rest of the batch, so a
// request gives bitwise the same result alone or in a mix.

// Split a chunk's surface tiles S ways.  Every table part (same nodes) uses
// the same splits and a workspace section of its own.
void set_splits(Chunk& c, int S, int tiles)
{
    const int tps = (tiles + S - 1) / S;
    c.f.tiles_per_split = tps;
    c.f.n_splits = (tiles + tps - 1) / tps;
    c.rl.n_splits = c.f.n_splits;
    c.ws_elems = (size_t)(c.f.n_splits + 1) * c.f.n_pts * c.f.n_omega * sc::kAcc * c.n_parts;
}

// Largest work item the split heuristic aims for, in evaluations: about 6 ms
// of one CTA at the field kernels' rate (2 CTAs per SM).  Serving cuts a long
// request into launches of a few dozen milliseconds, and such a launch stays
// balanced only if each CTA takes several items.
constexpr double kMaxItemEvals = 2.5e7;

// items_evals: the evaluations of one item if the chunk had a single split
int heuristic_splits(int tiles, long long pb, int slots, double item_evals)
{
    // enough items for dynamic balance (about 16 per resident CTA), items of
    // at most kMaxItemEvals evaluations and at least 32 node tiles, at most
    // 64 splits
    long long s = (16LL * slots + pb - 1) / pb;
    s = std::max<long long>(s, (long long)std::ceil(item_evals / kMaxItemEvals));
    s = std::min<long long>(s, std::max(1, tiles / 32));
    return (int)std::max<long long>(1, std::min<long long>(64, s));
}

sc_status launch_chunks_direct(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, float2* ws, size_t ws_n);

// Time one chunk with split count S (the chunk's outputs are overwritten later).
float time_chunk(sc_ctx* ctx, Lane& ln, Chunk c, int S, const Table* tab, float2* ws)
{
    set_splits(c, S, tab->n_surf_tiles);
    std::vector<Chunk> one{c};
    cudaEvent_t a = take_event(ctx), b = take_event(ctx);
    cudaEventRecord(a, ln.stream);
    sc_status st = launch_chunks_direct(ctx, ln, one, ws, c.ws_elems);
    cudaEventRecord(b, ln.stream);
    float ms = 1e30f;
    if (st == SC_OK && cudaEventSynchronize(b) == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaGetLastError();
    ctx->pool.push_back(a);
    ctx->pool.push_back(b);
    return ms;
}

constexpr double kTuneMaxEvals = 1.2e12;

// Split count for a chunk shape: explicit option, tuned value, or heuristic
// (tuned on first sight when the autotuner is on).
sc_status choose_splits(sc_ctx* ctx, Lane& ln, Chunk& c, const Table* tab, int slots, int* S_out)
{
    const int tiles = tab->n_surf_tiles;
    if (ctx->nodes_per_split > 0) {
        const int tps = (int)std::max<long long>(1, ctx->nodes_per_split / sc::kTile);
        *S_out = (tiles + tps - 1) / tps;
        return SC_OK;
    }
    const auto key = std::make_tuple(c.cls, tiles, tab->n_rim_tiles, c.f.n_pts, c.f.n_omega, c.n_parts);
    auto hit = ctx->tuned.find(key);
    if (hit != ctx->tuned.end()) {
        *S_out = hit->second;
        return SC_OK;
    }
    // whole-request workspace of split count s
    auto ws_bytes = [&](int s) {
        const int tps = (tiles + s - 1) / s;
        const int ns = (tiles + tps - 1) / tps;
        return (size_t)(ns + 1) * c.f.n_pts * c.f.n_omega * sc::kAcc * c.n_parts * sizeof(float2);
    };
    int s0 = heuristic_splits(tiles, c.pb, slots, (double)c.ppc * tiles * sc::kTile * c.f.n_omega * c.n_parts);
    // the item-size bound never cuts into points a request that balance alone keeps in one launch
    const int sb = heuristic_splits(tiles, c.pb, slots, 0.0);
    if (ws_bytes(sb) <= ctx->ws_cap)
        while (s0 > sb && ws_bytes(s0) > ctx->ws_cap) --s0;
    int best = s0;
    if (ctx->autotune) {
        // candidates around the heuristic, each timed once on the real chunk
        std::vector<int> cand;
        for (int s : {s0 / 2, s0, 2 * s0, 4 * s0})
            if (s >= 1 && s <= std::min(64, tiles) &&
                std::find(cand.begin(), cand.end(), s) == cand.end())
                cand.push_back(s);
        // only candidates whose whole-request workspace fits under the cap
        size_t need = 0;
        std::vector<int> fit;
        for (int s : cand) {
            const int tps = (tiles + s - 1) / s;
            const int ns = (tiles + tps - 1) / tps;
            const size_t n = (size_t)(ns + 1) * c.f.n_pts * c.f.n_omega * sc::kAcc * c.n_parts;
            if (n * sizeof(float2) <= ctx->ws_cap) {
                fit.push_back(s);
                need = std::max(need, n);
            }
        }
        // Timing costs one run of the chunk per candidate.  A chunk of more
        // than kTuneMaxEvals evaluations (about a second) takes the most
        // splits that fit instead: at that size more, shorter items balance
        // the CTAs' tails better, and the extra partials cost little.
        const double chunk_evals = (double)c.f.n_pts * tiles * sc::kTile * c.f.n_omega * c.n_parts;
        if (chunk_evals > kTuneMaxEvals && !fit.empty()) {
            best = *std::max_element(fit.begin(), fit.end());
        } else if (fit.size() > 1) {
            sc_status st = ensure(ctx, ln.ws, need * sizeof(float2), ln.stream);
            if (st != SC_OK) return st;
            float best_ms = 1e30f;
            for (int s : fit) {
                const float ms = time_chunk(ctx, ln, c, s, tab, (float2*)ln.ws.p);
                if (ms < best_ms) { best_ms = ms; best = s; }
            }
        }
    }
    ctx->tuned[key] = best;
    *S_out = best;
    return SC_OK;
}

// Kernel class (tile shape: threads per point x omegas per thread) of a
// chunk.  field_class(n) is the layout measured fastest on GB300 for n
// omegas; where a second layout of the same n is close (alt_field_class), the
// autotuner times both on the real chunk, each with its own tuned split
// count, on the first request of each shape, and keeps the faster unless the
// default is within 1%.  Chunks above kTuneMaxEvals keep the default.
// SC_OPT_TILE_LAYOUT 0 / 1 pins the default / the alternative.
sc_status choose_class(sc_ctx* ctx, Lane& ln, Chunk& c, const Table* tab, int* cls_out)
{
    const int def = sc::field_class(c.f.n_omega);
    *cls_out = def;
    const int alt = sc::alt_field_class(c.f.n_omega);
    if (alt < 0 || ctx->tile_layout == 0) return SC_OK;
    if (ctx->tile_layout == 1) {
        *cls_out = alt;
        return SC_OK;
    }
    if (!ctx->autotune || ctx->nodes_per_split > 0) return SC_OK;
    const int tiles = tab->n_surf_tiles;
    const auto key = std::make_tuple(-1 - c.f.n_omega, tiles, tab->n_rim_tiles, c.f.n_pts, 0, c.n_parts);
    auto hit = ctx->tuned.find(key);
    if (hit != ctx->tuned.end()) {
        *cls_out = hit->second;
        return SC_OK;
    }
    const double chunk_evals = (double)c.f.n_pts * tiles * sc::kTile * c.f.n_omega * c.n_parts;
    if (chunk_evals > kTuneMaxEvals) {
        ctx->tuned[key] = def;
        return SC_OK;
    }
    float ms[2] = {1e30f, 1e30f};
    const int cand[2] = {def, alt};
    for (int i = 0; i < 2; ++i) {
        Chunk t = c;
        t.cls = cand[i];
        int slots = 1;
        sc::field_shape(t.cls, ctx->device, &t.ppc, &slots);
        t.pb = (t.f.n_pts + t.ppc - 1) / t.ppc;
        int S = 1;
        sc_status st = choose_splits(ctx, ln, t, tab, slots, &S);
        if (st != SC_OK) return st;
        set_splits(t, S, tiles);
        if (t.ws_elems * sizeof(float2) > ctx->ws_cap) continue;  // would need point chunks: not timed
        st = ensure(ctx, ln.ws, t.ws_elems * sizeof(float2), ln.stream);
        if (st != SC_OK) return st;
        ms[i] = time_chunk(ctx, ln, t, S, tab, (float2*)ln.ws.p);
    }
    const int best = (ms[1] < 0.99f * ms[0]) ? alt : def;
    ctx->tuned[key] = best;
    *cls_out = best;
    return SC_OK;
}

// Field-kernel throughput of one chunk, in 1e11 (point, node, omega)
// evaluations per second, measured on GB300 on the broadband mirror and beam
// at 256^2 nodes and 4160 focal points (tune_chunks.py in the package
// re-measures both tables): every omega count 1..64, and full grouped chunks
// of 64, 128, ..., 2048 omegas.  A grouped chunk of n > 64 omegas gives every
// point a power of two threads of 8 omegas, so it takes as long as a full
// chunk of its capacity (the next power of two >= n).
constexpr double kRateSmall[65] = {
    0.0,
    3.669, 4.907, 5.611, 6.067, 6.591, 7.171, 6.940, 7.982,  // 1..8
    7.440, 8.268, 8.135, 8.854, 8.567, 9.226, 8.795, 9.347,  // 9..16
    8.338, 8.819, 9.305, 9.805, 9.101, 9.525, 9.963, 10.373,  // 17..24
    8.348, 8.683, 9.015, 9.312, 9.663, 9.988, 10.337, 10.594,  // 25..32
    8.848, 9.108, 9.379, 9.639, 9.900, 10.170, 10.431, 10.707,  // 33..40
    9.547, 9.778, 10.006, 10.222, 10.465, 10.702, 10.916, 11.151,  // 41..48
    10.127, 10.333, 10.519, 10.727, 10.940, 11.126, 11.326, 11.552,  // 49..56
    10.336, 10.506, 10.692, 10.859, 11.060, 11.229, 11.408, 11.539,  // 57..64
};
constexpr double kRateFull[6] = {11.536, 12.204, 12.196, 10.848, 11.060, 10.884};  // 64 .. 2048

constexpr int kMaxChunk = 2048;

// Relative field time of one chunk of c omegas (per point-node pair).
double chunk_cost(int c)
{
    if (c <= 64) return c / kRateSmall[c];
    int cap = 128, i = 1;
    while (cap < c) {
        cap *= 2;
        ++i;
    }
    return cap / kRateFull[i];
}

// The omega chunks of a request: for every n <= 2048 the split that
// minimises the summed chunk times, charging each extra chunk 2% of a
// 32-omega chunk, as the first chunk of that split (the rest is looked up
// again).  Splits at any count up to 64 are allowed for requests large enough
// that an extra chunk's launch does not matter (`small`); otherwise only
// full grouped capacities (64, 128, ...) are cut off.  Computed once per
// process from the tables above; the result depends only on the request.
struct ChunkPlan {
    unsigned short first[2][kMaxChunk + 1];
};

const ChunkPlan& chunk_plan()
{
    static const ChunkPlan plan = [] {
        ChunkPlan p{};
        std::vector<double> best(kMaxChunk + 1, 0.0);
        const double extra = 0.02 * chunk_cost(32);
        for (int small = 0; small < 2; ++small) {
            for (int m = 1; m <= kMaxChunk; ++m) {
                double b = chunk_cost(m);
                int f = m;
                auto consider = [&](int c) {
                    const double v = chunk_cost(c) + best[m - c] + extra;
                    if (v < b) {
                        b = v;
                        f = c;
                    }
                };
                if (small)
                    for (int c = 1; c <= std::min(m - 1, 64); ++c) consider(c);
                else if (m > 64)
                    consider(64);
                for (int c = 128; c < m; c *= 2) consider(c);
                best[m] = b;
                p.first[small][m] = (unsigned short)f;
            }
        }
        return p;
    }();
    return plan;
}

// Omega count of the next chunk of a request with n omegas left.
int next_chunk(int n, bool small)
{
    return chunk_plan().first[small ? 1 : 0][std::min(n, kMaxChunk)];
}

// a launch bounded in evaluations still gives each resident CTA this many items
constexpr double kMinItemsPerCta = 4.0;

// requests of at least this many (point, node) pairs per omega take the
// splits at small omega counts
constexpr long long kSmallCutPairs = 1LL << 22;

// FP32 run length of tables fitted in k (see plan_request)
constexpr long long kFittedFlushNodes = 512;

// Cut one request into chunks.  d_amp / d_k point at this request's a_n, k_n.
sc_status plan_request(sc_ctx* ctx, Lane& ln, const Table* tab, const double* omegas, int n_omega,
                       double dom, const double* d_pts, int n_points, const double* d_amp,
                       const double* d_k, float2* dE, float2* dB, std::vector<Chunk>& out)
{
    if (!tab->fp32_ok)
        return fail(ctx, SC_ERR_INVALID,
                    "this mirror and beam do not focus on the origin (e.g. a collimated beam on an "
                    "ellipsoid): the compensated FP32 phase does not apply, use SC_FP64");
    // Beams expanded in Chebyshev terms of k sum their parts with weights of
    // alternating sign, which magnifies the FP32 rounding of each part's long
    // runs: they fold every 512 nodes (the worst of 1240 seeded random
    // configurations went from 9.7e-6 to 5.7e-6 of the 1e-5 gate).
    long long flush_nodes = ctx->flush_nodes;
    for (const auto& part : tab->parts)
        if (part.kind == PART_CHEB_RE || part.kind == PART_CHEB_IM)
            flush_nodes = std::min<long long>(flush_nodes, kFittedFlushNodes);
    const int flush_tiles = (int)std::max<long long>(1, flush_nodes / sc::kTile);
    const bool small_cuts = (long long)n_points * tab->n_surf >= kSmallCutPairs;
    for (int o0 = 0, no = 0; o0 < n_omega; o0 += no) {
        no = ctx->omega_chunks ? next_chunk(n_omega - o0, small_cuts) : std::min(kMaxChunk, n_omega - o0);
        Chunk c;
        const double w0 = omegas[o0];
        c.f.nodes = tab->d32;
        c.f.n_surf_tiles = tab->n_surf_tiles;
        c.f.n_rim_tiles = tab->n_rim_tiles;
        c.f.flush_tiles = flush_tiles;
        c.f.n_omega = no;
        c.f.om_hi0 = (float)w0;
        c.f.om_lo0 = (float)(w0 - (double)c.f.om_hi0);
        c.f.dom_hi = (float)dom;
        c.f.dom_lo = (float)(dom - (double)c.f.dom_hi);
        c.f.err = ctx->d_err;
        c.f.ws = nullptr;
        // the split count is chosen on the whole request's point count
        c.f.pts = d_pts;
        c.f.n_pts = n_points;
        c.rl.amp = d_amp + 2 * (size_t)o0;
        c.rl.kval = d_k + o0;
        c.rl.out_pt_stride_omega = (long long)n_points * 3;
        c.rl.E = dE + (size_t)o0 * n_points * 3;
        c.rl.B = dB ? dB + (size_t)o0 * n_points * 3 : nullptr;
        c.rl.n_pts = n_points;
        c.rl.n_omega = no;
        c.tab = tab;
        c.n_parts = (int)tab->parts.size();
        c.rl.n_parts = c.n_parts;
        c.rl.amp_stride = 2LL * n_omega;
        // tile shape: the measured default layout for this omega count, or the
        // autotuner's choice between it and an alternative
        sc_status st = choose_class(ctx, ln, c, tab, &c.cls);
        if (st != SC_OK) return st;
        int slots = 1;
        sc::field_shape(c.cls, ctx->device, &c.ppc, &slots);
        c.pb = (n_points + c.ppc - 1) / c.ppc;
        int S = 1;
        st = choose_splits(ctx, ln, c, tab, slots, &S);
        if (st != SC_OK) return st;
        set_splits(c, S, tab->n_surf_tiles);
        const int n_splits = c.f.n_splits;
        // point chunks bounded by the workspace cap and, on a lane whose
        // launches are bounded (serving's long requests), by its evaluations
        // per launch; the split count above stays that of the whole request,
        // so every point's arithmetic is the same however the points are cut
        const size_t per_pt = (size_t)(n_splits + 1) * no * sc::kAcc * c.n_parts;
        long long pchunk = std::max<long long>(1, (long long)(ctx->ws_cap / sizeof(float2) / per_pt));
        if (ln.max_launch_evals > 0.0) {
            // never fewer than kMinItemsPerCta items per resident CTA, or the
            // launch's tail would idle most of the GPU
            const double pt_evals = (double)tab->n_surf_tiles * sc::kTile * no * c.n_parts;
            const double item = (double)c.ppc * c.f.tiles_per_split * sc::kTile * no * c.n_parts;
            const double g = std::max(ln.max_launch_evals, kMinItemsPerCta * slots * item);
            pchunk = std::min<long long>(pchunk, std::max<long long>(1, (long long)(g / pt_evals)));
        }
        if (pchunk < n_points) pchunk = std::max<long long>(c.ppc, pchunk / c.ppc * c.ppc);
        for (int p0 = 0; p0 < n_points; p0 += (int)pchunk) {
            const int np = (int)std::min<long long>(pchunk, n_points - p0);
            Chunk d = c;
            d.f.pts = d_pts + 3 * (size_t)p0;
            d.f.n_pts = np;
            d.pb = (np + c.ppc - 1) / c.ppc;
            d.rl.n_pts = np;
            d.rl.E = c.rl.E + (size_t)p0 * 3;
            d.rl.B = c.rl.B ? c.rl.B + (size_t)p0 * 3 : nullptr;
            d.ws_elems = per_pt * np;
            out.push_back(d);
        }
    }
    return SC_OK;
}

// Launch a group of chunks whose workspaces fit in ws, with or without a
// CUDA graph.  Field kernels (one persistent launch per class present) go
// in the graph; the batched reduce follows on the stream.
sc_status launch_chunks(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, float2* ws, size_t ws_n, bool graph)
{
    // workspace offsets and reduce offsets
    size_t off = 0;
    long long roff = 0;
    for (auto& c : ch) {
        c.f.ws = ws + off;
        c.rl.ws = ws + off;
        c.rl.off = roff;
        off += c.ws_elems;
        roff += (long long)c.rl.n_pts * c.rl.n_omega;
    }
    if (off > ws_n) return fail(ctx, SC_ERR_OOM, "workspace plan exceeds its buffer");
    // per-class descriptor arrays
    constexpr int kClasses = sc::kNumClasses;
    std::vector<sc::WorkReq> reqs[kClasses];
    long long items[kClasses] = {};
    for (auto& c : ch)
        for (int t = 0; t < c.n_parts; ++t) {
            sc::WorkReq w;
            w.f = c.f;
            w.f.nodes = c.tab->parts[t].d32;
            w.f.n_rim_tiles = c.tab->parts[t].n_rim_tiles;
            w.f.ws = c.f.ws + (size_t)t * (c.ws_elems / c.n_parts);
            w.pb = c.pb;
            w.cls = c.cls;
            w.item0 = items[c.cls];
            items[c.cls] += (long long)c.pb * (w.f.n_splits + 1);
            reqs[c.cls].push_back(w);
        }
    std::vector<sc::ReduceLaunch> rls;
    for (auto& c : ch) rls.push_back(c.rl);
    // arena: queues and abort words (64 B per class) | WorkReq arrays | ReduceLaunch array
    size_t bytes = kClasses * 64;
    size_t req_off[kClasses];
    for (int k = 0; k < kClasses; ++k) {
        req_off[k] = bytes;
        bytes += (reqs[k].size() * sizeof(sc::WorkReq) + 255) / 256 * 256;
    }
    const size_t rl_off = bytes;
    bytes += rls.size() * sizeof(sc::ReduceLaunch);
    sc_status st = ensure(ctx, ln.desc, bytes, ln.stream);
    if (st != SC_OK) return st;
    unsigned char* arena = (unsigned char*)ln.desc.p;
    for (int k = 0; k < kClasses; ++k)
        if (!reqs[k].empty())
            SC_CUDA(cudaMemcpyAsync(arena + req_off[k], reqs[k].data(), reqs[k].size() * sizeof(sc::WorkReq),
                                    cudaMemcpyHostToDevice, ln.stream), "upload work descriptors");
    SC_CUDA(cudaMemcpyAsync(arena + rl_off, rls.data(), rls.size() * sizeof(sc::ReduceLaunch),
                            cudaMemcpyHostToDevice, ln.stream), "upload reduce descriptors");

    struct L { int cls; sc::BatchLaunch b; int grid; };
    std::vector<L> launches;
    for (int k = 0; k < kClasses; ++k) {
        if (reqs[k].empty()) continue;
        int ppc = 1, slots = 1;
        sc::field_shape(k, ctx->device, &ppc, &slots);
        sc::BatchLaunch b{};
        b.reqs = (const sc::WorkReq*)(arena + req_off[k]);
        b.n_req = (int)reqs[k].size();
        b.n_items = items[k];
        b.queue = (int*)(arena + 64 * k);
        b.abort = b.queue + 1;  // the launch's abort word, reset with its queue
        b.err = ctx->d_err;
        b.fail_tile = ctx->fail_tile;
        launches.push_back({k, b, (int)std::min<long long>(slots, items[k])});
    }
    // With several kernel classes, each persistent launch runs on a branch of
    // its own (forked from the lane's stream and joined back into it), so the
    // CTAs of one class fill the SMs that another class's tail leaves idle.
    // Every item writes only its own workspace section and its arithmetic does
    // not depend on scheduling, so results stay bitwise the same.
    const bool branches = ctx->class_streams && launches.size() > 1;
    if (branches) {
        if (!ln.fork_ev) SC_CUDA(cudaEventCreateWithFlags(&ln.fork_ev, cudaEventDisableTiming), "fork event");
        while (ln.side.size() < launches.size()) {
            cudaStream_t b = nullptr;
            cudaEvent_t e = nullptr;
            SC_CUDA(cudaStreamCreateWithPriority(&b, cudaStreamNonBlocking, ln.prio), "class stream");
            ln.side.push_back(b);
            SC_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming), "join event");
            ln.join_ev.push_back(e);
        }
    }
    auto issue = [&](cudaStream_t s) -> sc_status {
        SC_CUDA(cudaMemsetAsync(arena, 0, kClasses * 64, s), "reset work queues");
        if (!branches) {
            for (auto& l : launches) {
                const int r = sc::launch_field_batch(l.cls, l.b, l.grid, s);
                if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "field kernel launch");
            }
            return SC_OK;
        }
        SC_CUDA(cudaEventRecord(ln.fork_ev, s), "fork");
        for (size_t i = 0; i < launches.size(); ++i) {
            SC_CUDA(cudaStreamWaitEvent(ln.side[i], ln.fork_ev, 0), "fork wait");
            const int r = sc::launch_field_batch(launches[i].cls, launches[i].b, launches[i].grid, ln.side[i]);
            if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "field kernel launch");
            SC_CUDA(cudaEventRecord(ln.join_ev[i], ln.side[i]), "join");
            SC_CUDA(cudaStreamWaitEvent(s, ln.join_ev[i], 0), "join wait");
        }
        return SC_OK;
    };
    cudaEvent_t f0 = nullptr, f1 = nullptr;
    if (ctx->time_field) {
        f0 = take_event(ctx);
        f1 = take_event(ctx);
        cudaEventRecord(f0, ln.stream);
    }
    if (graph) {
        // signature: everything the captured launches depend on
        std::vector<unsigned char> sig;
        auto put = [&](const void* p, size_t n) {
            const unsigned char* q = (const unsigned char*)p;
            sig.insert(sig.end(), q, q + n);
        };
        put(&arena, sizeof arena);
        put(&branches, sizeof branches);
        for (auto& l : launches) {
            put(&l.cls, sizeof l.cls);
            put(&l.grid, sizeof l.grid);
            put(&l.b, sizeof l.b);
        }
        cudaGraphExec_t exec = nullptr;
        for (auto& g : ln.graphs)
            if (g.sig == sig) {
                exec = g.exec;
                g.last = ++ctx->graph_tick;
                ctx->graph_replays++;
            }
        if (!exec) {
            if (!ln.cap_stream)
                SC_CUDA(cudaStreamCreateWithPriority(&ln.cap_stream, cudaStreamNonBlocking, ln.prio),
                        "capture stream");
            SC_CUDA(cudaStreamBeginCapture(ln.cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
            st = issue(ln.cap_stream);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(ln.cap_stream, &g);
            if (st != SC_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
            e = cudaGraphInstantiate(&exec, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "graph instantiate");
            if (ln.graphs.size() >= 8) {
                auto it = std::min_element(ln.graphs.begin(), ln.graphs.end(),
                                           [](const GraphEntry& a, const GraphEntry& b) {
                                               return a.last < b.last;
                                           });
                cudaGraphExecDestroy(it->exec);
                ln.graphs.erase(it);
            }
            ln.graphs.push_back({sig, exec, ++ctx->graph_tick});
            ctx->graph_captures++;
        }
        SC_CUDA(cudaGraphLaunch(exec, ln.stream), "graph launch");
    } else {
        st = issue(ln.stream);
        if (st != SC_OK) return st;
    }
    if (ctx->time_field) {
        cudaEventRecord(f1, ln.stream);
        ctx->pending.push_back({f0, f1});
    }
    ctx->ctr.launches += launches.size();
    ctx->ctr.field_launches += launches.size();
    const int r = sc::launch_reduce_batch((const sc::ReduceLaunch*)(arena + rl_off), (int)rls.size(),
                                          roff, ln.stream);
    if (r < 0) return cuda_fail(ctx, (cudaError_t)(-r), "reduce launch");
    ctx->ctr.launches += r;
    return SC_OK;
}

sc_status launch_chunks_direct(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, float2* ws, size_t ws_n)
{
    const bool t = ctx->time_field;
    ctx->time_field = false;
    sc_status st = launch_chunks(ctx, ln, ch, ws, ws_n, false);
    ctx->time_field = t;
    return st;
}

// Evaluations of one chunk, every table part.
double chunk_evals(const Chunk& c)
{
    return (double)c.f.n_pts * c.f.n_surf_tiles * sc::kTile * c.f.n_omega * c.n_parts;
}

// Launch the group of chunks that starts at ch[i] -- as many as fit under
// the workspace cap (and, on a lane with bounded launches, under its bound
// on evaluations) -- and advance i past it.
sc_status run_chunk_group(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, size_t& i)
{
    const size_t cap = std::max<size_t>(ctx->ws_cap / sizeof(float2), 1);
    const double ecap = ln.max_launch_evals > 0.0 ? ln.max_launch_evals : 1e300;
    size_t j = i, tot = 0;
    double ev = 0.0;
    while (j < ch.size() && (j == i || (tot + ch[j].ws_elems <= cap && ev + chunk_evals(ch[j]) <= ecap))) {
        ev += chunk_evals(ch[j]);
        tot += ch[j++].ws_elems;
    }
    sc_status st = ensure(ctx, ln.ws, tot * sizeof(float2), ln.stream);
    if (st != SC_OK) return st;
    std::vector<Chunk> part(ch.begin() + i, ch.begin() + j);
    st = launch_chunks(ctx, ln, part, (float2*)ln.ws.p, tot, ctx->use_graphs && ln.use_graphs);
    if (st != SC_OK) return st;
    i = j;
    return SC_OK;
}

// Run every chunk, group by group.
sc_status run_chunks(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch)
{
    size_t i = 0;
    while (i < ch.size()) {
        const sc_status st = run_chunk_group(ctx, ln, ch, i);
        if (st != SC_OK) return st;
    }
    return SC_OK;
}

void free_lane(Lane& ln)
{
    if (ln.stream) cudaStreamSynchronize(ln.stream);
    for (DevBuf* b : {&ln.ws, &ln.desc, &ln.amp, &ln.kval})
        if (b->p) {
            cudaFree(b->p);
            b->p = nullptr;
            b->n = 0;
        }
    for (auto& g : ln.graphs) cudaGraphExecDestroy(g.exec);
    ln.graphs.clear();
    if (ln.cap_stream) cudaStreamDestroy(ln.cap_stream);
    ln.cap_stream = nullptr;
    for (cudaStream_t b : ln.side) cudaStreamDestroy(b);
    for (cudaEvent_t e : ln.join_ev) cudaEventDestroy(e);
    if (ln.fork_ev) cudaEventDestroy(ln.fork_ev);
    ln.side.clear();
    ln.join_ev.clear();
    ln.fork_ev = nullptr;
    if (ln.own_stream && ln.stream) cudaStreamDestroy(ln.stream);
    ln.stream = nullptr;
}

}  // namespace sch

extern "C" sc_status sc_plan_omega_chunks(sc_ctx* ctx, int n_omega, long long pairs_per_omega, int* sizes,
                                          int max_sizes, int* n_sizes)
{
    if (n_omega < 1 || pairs_per_omega < 0 || !n_sizes || (max_sizes > 0 && !sizes))
        return sch::fail(ctx, SC_ERR_INVALID, "invalid argument");
    const bool plan = ctx ? ctx->omega_chunks : true;
    const bool small = pairs_per_omega >= sch::kSmallCutPairs;
    int k = 0;
    for (int o0 = 0, no = 0; o0 < n_omega; o0 += no, ++k) {
        no = plan ? sch::next_chunk(n_omega - o0, small) : std::min(sch::kMaxChunk, n_omega - o0);
        if (k < max_sizes) sizes[k] = no;
    }
    *n_sizes = k;
    return k <= max_sizes ? SC_OK : sch::fail(ctx, SC_ERR_INVALID, "%d chunks do not fit in %d entries", k, max_sizes);
}
