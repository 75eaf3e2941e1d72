// sc_serve.cpp -- serving (A9): the server thread that admits, batches and
// completes submitted requests on four lanes (two for short requests, two for long ones).
#include <algorithm>

#include "sc_host.h"

namespace sch {

// ------------------------------------------------------------------------
// Serving (A9): continuous batching of submitted requests.  A server thread
// admits queued requests in arrival order while their device memory (staged
// points and server-owned outputs) fits the context's HBM budget, batches
// them and runs each batch on a free lane (a stream with its own buffers), so
// requests that arrive while others run overlap with them on the device.
// Completion is observed through an event per lane; memory returns to the
// budget when the caller releases the ticket.
//
// Short requests first.  A few long requests carry most of the work of a
// mixed stream, and under first-come-first-served every short request that
// arrives behind one waits for all of it.  So requests are classed by their
// evaluations (points x surface nodes x omegas):
//   * short ones (at most kLongEvals) run on two lanes whose streams have the
//     highest priority, batched until a batch holds kShortBatchEvals;
//   * long ones run one at a time on two lanes of the lowest priority, and
//     their chunks are cut by points into launches of about kGroupEvals
//     (more where that would leave fewer than 4 work items per resident CTA),
//     launched one after another as each completes.
// The field kernels are persistent (their CTAs stay until a launch's work
// is drained), so a running launch is never interrupted.  But when one of a
// long request's bounded launches ends, the block scheduler gives the freed
// SMs to pending high-priority work first: a short request waits for at most
// one such launch instead of a whole long request.  Two long lanes share the
// GPU launch by launch, so a long request does not wait for a longer one
// ahead of it either.  Cutting by points keeps every point's arithmetic (its
// split count is that of the whole request), so results stay bitwise the same
// as alone.  With SC_OPT_SERVE_PRIORITY = 0 the server uses two lanes of the
// default priority, first come first served, without bounded launches.
constexpr double kLongEvals = 1e11;        // about 90 ms of field work on one GB300
constexpr double kGroupEvals = 6e10;       // about 50 ms
constexpr double kShortBatchEvals = 3e10;

size_t ticket_bytes(const Ticket& t)
{
    size_t b = 0;
    if (t.own_pts) b += (size_t)t.n_points * 3 * sizeof(double);
    if (t.own_out) b += (size_t)2 * t.n_omega * t.n_points * 3 * sizeof(float2);
    return b;
}

sc_status launch_next_group(sc_ctx* ctx, Server* srv, int L);

// Ticket memory, stream-ordered, from the server's pool when it has one.
cudaError_t serve_alloc(Server* srv, void** p, size_t bytes, cudaStream_t s)
{
    return srv->pool ? cudaMallocFromPoolAsync(p, bytes, srv->pool, s) : cudaMallocAsync(p, bytes, s);
}

// Run one batch of admitted tickets on lane L (ctx->mu held).  A ticket
// whose node tables cannot be built (an envelope too rough to fit, a device
// allocation that failed) fails alone and leaves ids; the others run.
sc_status launch_batch(sc_ctx* ctx, Server* srv, int L, std::vector<uint64_t>& ids)
{
    Lane& ln = srv->lanes[L];
    ctx->tick++;
    std::vector<double> amp_all, k_all;
    std::vector<size_t> om_off, amp_off;
    std::vector<uint64_t> run;
    for (uint64_t id : ids) {
        Ticket& t = srv->tickets[id];
        t.lane = L;
        t.t_start = srv->now();
        std::vector<double> a;
        sc_status tst = get_table(ctx, t.mirror, t.incident, &t.tab, ln.stream);
        if (tst == SC_OK) tst = request_amps(ctx, t.incident, t.tab, t.omegas.data(), t.n_omega, a);
        if (tst != SC_OK) {
            t.tab = nullptr;
            t.state = 3;
            t.status = tst;
            t.t_done = srv->now();
            continue;
        }
        t.state = 1;
        t.tab->inflight++;
        run.push_back(id);
        if (t.own_pts) {
            SC_CUDA(serve_alloc(srv, (void**)&t.pts, (size_t)t.n_points * 3 * sizeof(double), ln.stream),
                    "serving points");
            SC_CUDA(cudaMemcpyAsync(t.pts, t.host_pts.data(), (size_t)t.n_points * 3 * sizeof(double),
                                    cudaMemcpyHostToDevice, ln.stream), "stage points");
        } else {
            t.pts = (double*)t.user_pts;
        }
        if (t.own_out) {
            const size_t ob = (size_t)t.n_omega * t.n_points * 3 * sizeof(float2);
            SC_CUDA(serve_alloc(srv, &t.E, ob, ln.stream), "serving outputs");
            SC_CUDA(serve_alloc(srv, &t.B, ob, ln.stream), "serving outputs");
        } else {
            t.E = t.E_user;
            t.B = t.B_user;
        }
        amp_off.push_back(amp_all.size());
        om_off.push_back(k_all.size());
        amp_all.insert(amp_all.end(), a.begin(), a.end());
        for (double w : t.omegas) k_all.push_back(2.0 * kPi * w);
    }
    ids.swap(run);
    if (ids.empty()) return SC_OK;
    sc_status st;
    if ((st = ensure(ctx, ln.amp, amp_all.size() * sizeof(double), ln.stream)) != SC_OK) return st;
    if ((st = ensure(ctx, ln.kval, k_all.size() * sizeof(double), ln.stream)) != SC_OK) return st;
    SC_CUDA(cudaMemcpyAsync(ln.amp.p, amp_all.data(), amp_all.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ln.stream), "upload amplitudes");
    SC_CUDA(cudaMemcpyAsync(ln.kval.p, k_all.data(), k_all.size() * sizeof(double),
                            cudaMemcpyHostToDevice, ln.stream), "upload wavenumbers");
    std::vector<Chunk> ch;
    for (size_t i = 0; i < ids.size(); ++i) {
        Ticket& t = srv->tickets[ids[i]];
        st = plan_request(ctx, ln, t.tab, t.omegas.data(), t.n_omega, t.dom, t.pts, t.n_points,
                          (const double*)ln.amp.p + amp_off[i], (const double*)ln.kval.p + om_off[i],
                          (float2*)t.E, (float2*)t.B, ch);
        if (st != SC_OK) return st;
        ctx->ctr.evals += (double)t.n_points * t.tab->n_surf * t.n_omega;
    }
    if (ln.max_launch_evals > 0.0) {
        // a long lane launches one bounded group now and the next when it
        // completes, so work admitted later is never queued behind the rest
        srv->pend[L].swap(ch);
        srv->pend_i[L] = 0;
        return launch_next_group(ctx, srv, L);
    }
    st = run_chunks(ctx, ln, ch);
    if (st != SC_OK) return st;
    SC_CUDA(cudaEventRecord(srv->done_ev[L], ln.stream), "completion event");
    return SC_OK;
}

// Launch the next bounded group of lane L's pending chunks (ctx->mu held);
// the lane's completion event follows it.
sc_status launch_next_group(sc_ctx* ctx, Server* srv, int L)
{
    Lane& ln = srv->lanes[L];
    const sc_status st = run_chunk_group(ctx, ln, srv->pend[L], srv->pend_i[L]);
    if (st != SC_OK) return st;
    if (srv->pend_i[L] >= srv->pend[L].size()) {
        srv->pend[L].clear();
        srv->pend_i[L] = 0;
    }
    SC_CUDA(cudaEventRecord(srv->done_ev[L], ln.stream), "completion event");
    return SC_OK;
}

// Fail every ticket of a batch whose launch failed on lane L.
void fail_batch(Server* srv, int L, const std::vector<uint64_t>& ids, sc_status st)
{
    cudaStreamSynchronize(srv->lanes[L].stream);
    for (uint64_t id : ids) {
        Ticket& t = srv->tickets[id];
        if (t.tab) t.tab->inflight--;
        t.tab = nullptr;
        t.state = 3;
        t.status = st;
        t.t_done = srv->now();
    }
    srv->pend[L].clear();
    srv->pend_i[L] = 0;
}

void serve(sc_ctx* ctx)
{
    Server* srv = ctx->server;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (!srv->stop) {
        bool changed = false;
        std::vector<int> next_group;  // long lanes whose group completed, with more to launch
        // completions
        for (int L = 0; L < Server::kLanes; ++L) {
            if (!srv->busy[L]) continue;
            const cudaError_t q = cudaEventQuery(srv->done_ev[L]);
            if (q == cudaErrorNotReady) continue;
            if (q == cudaSuccess && !srv->pend[L].empty()) {
                bool all_cancelled = true;
                for (uint64_t id : srv->batch[L]) all_cancelled = all_cancelled && srv->tickets[id].cancel;
                if (!all_cancelled) {
                    next_group.push_back(L);
                    continue;
                }
            }
            srv->pend[L].clear();  // done, failed, or all cancelled: drop what is left
            srv->pend_i[L] = 0;
            const double t = srv->now();
            for (uint64_t id : srv->batch[L]) {
                auto it = srv->tickets.find(id);
                if (it == srv->tickets.end()) continue;
                Ticket& tk = it->second;
                if (tk.tab) tk.tab->inflight--;
                tk.tab = nullptr;
                tk.t_done = t;
                if (q != cudaSuccess) {
                    tk.state = 3;
                    tk.status = SC_ERR_CUDA;
                } else {
                    tk.state = tk.cancel ? 4 : 2;
                }
            }
            if (q != cudaSuccess) cudaGetLastError();
            srv->batch[L].clear();
            srv->busy[L] = false;
            changed = true;
        }
        // admission and launch on free lanes: the short lanes first, then the
        // long lanes' next groups, then new long requests
        const int n_lanes = srv->priority ? Server::kLanes : 2;
        auto launch_groups = [&]() {
            for (int G : next_group) {
                const sc_status gst = launch_next_group(ctx, srv, G);
                if (gst != SC_OK) {
                    fail_batch(srv, G, srv->batch[G], gst);
                    srv->batch[G].clear();
                    srv->busy[G] = false;
                }
                changed = true;
            }
            next_group.clear();
        };
        for (int L = 0; L < n_lanes; ++L) {
            if (L == Server::kShortLanes) launch_groups();
            if (srv->busy[L] || srv->queue.empty()) continue;
            // workspace the lanes may still grow into (bounded by the cap)
            size_t reserve = size_t(16) << 20;
            for (int M = 0; M < n_lanes; ++M)
                if (srv->lanes[M].ws.n < ctx->ws_cap) reserve += ctx->ws_cap - srv->lanes[M].ws.n;
            const bool short_lane = L < Server::kShortLanes;
            std::vector<uint64_t> ids;
            double batch_evals = 0.0;
            for (auto it = srv->queue.begin(); it != srv->queue.end() && (int)ids.size() < srv->max_batch;) {
                Ticket& t = srv->tickets[*it];
                if (srv->priority && (t.evals > kLongEvals) == short_lane) {
                    ++it;  // a request for the other kind of lane
                    continue;
                }
                const size_t b = ticket_bytes(t);
                // admit only what fits next to every lane's full workspace; the
                // first request of an idle server is always admitted
                const bool idle = srv->held == 0 && ids.empty();
                if (ctx->budget && !idle && ctx->held + srv->held + b + reserve > ctx->budget) break;
                t.bytes = b;
                srv->held += b;
                ids.push_back(*it);
                it = srv->queue.erase(it);
                batch_evals += t.evals;
                // a long lane runs one request at a time; a short lane's batch
                // closes once it holds enough work to fill the GPU
                if (srv->priority && (!short_lane || batch_evals >= kShortBatchEvals)) break;
            }
            if (ids.empty()) continue;
            const sc_status st = launch_batch(ctx, srv, L, ids);
            if (st == SC_OK && ids.empty()) {
                changed = true;
                continue;
            }
            if (st != SC_OK) {
                fail_batch(srv, L, ids, st);
            } else {
                srv->batch[L] = ids;
                srv->busy[L] = true;
            }
            changed = true;
        }
        launch_groups();
        if (changed) srv->cv.notify_all();
        srv->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

sc_status start_server(sc_ctx* ctx)
{
    if (ctx->server) return SC_OK;
    Server* srv = new Server();
    srv->priority = ctx->serve_priority;
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    for (int L = 0; L < Server::kLanes; ++L) {
        Lane& ln = srv->lanes[L];
        const bool short_lane = srv->priority && L < Server::kShortLanes;
        const bool long_lane = srv->priority && L >= Server::kShortLanes;
        ln.prio = short_lane ? greatest : least;
        // captured launches are not relied on to keep the stream's priority
        ln.use_graphs = !short_lane;
        ln.max_launch_evals = long_lane ? kGroupEvals : 0.0;
        if (cudaStreamCreateWithPriority(&ln.stream, cudaStreamNonBlocking, ln.prio) != cudaSuccess ||
            cudaEventCreateWithFlags(&srv->done_ev[L], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            for (int M = 0; M <= L; ++M) {
                if (srv->lanes[M].stream) cudaStreamDestroy(srv->lanes[M].stream);
                if (srv->done_ev[M]) cudaEventDestroy(srv->done_ev[M]);
            }
            delete srv;
            return fail(ctx, SC_ERR_CUDA, "serving lane set-up failed");
        }
        ln.own_stream = true;
    }
    // The server's memory pool keeps what tickets free (no release threshold)
    // and is warmed with min(budget / 8, 1 GiB): growing device memory while
    // other lanes' kernels run can stall the server thread, which admits and
    // launches everything.  Without a pool of its own it uses the default one.
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = ctx->device;
    if (cudaMemPoolCreate(&srv->pool, &props) == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(srv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        size_t warm = size_t(1) << 30;
        if (ctx->budget) warm = std::min(warm, ctx->budget / 8);
        void* p = nullptr;
        cudaStream_t s0 = srv->lanes[0].stream;
        if (warm && cudaMallocFromPoolAsync(&p, warm, srv->pool, s0) == cudaSuccess) cudaFreeAsync(p, s0);
        cudaStreamSynchronize(s0);
        cudaGetLastError();
    } else {
        srv->pool = nullptr;
        cudaGetLastError();
    }
    ctx->server = srv;
    srv->th = std::thread(serve, ctx);
    return SC_OK;
}

void free_ticket_memory(Server* srv, Ticket& t)
{
    cudaStream_t s = t.lane >= 0 ? srv->lanes[t.lane].stream : nullptr;
    if (t.own_pts && t.pts) cudaFreeAsync(t.pts, s);
    if (t.own_out && t.E) cudaFreeAsync(t.E, s);
    if (t.own_out && t.B) cudaFreeAsync(t.B, s);
    t.pts = nullptr;
    t.E = t.B = nullptr;
    srv->held -= t.bytes;
    t.bytes = 0;
}

void stop_server(sc_ctx* ctx)
{
    Server* srv = ctx->server;
    if (!srv) return;
    {
        std::lock_guard<std::mutex> lock(ctx->mu);
        srv->stop = true;
    }
    srv->cv.notify_all();
    srv->th.join();
    cudaSetDevice(ctx->device);
    for (int L = 0; L < Server::kLanes; ++L) cudaStreamSynchronize(srv->lanes[L].stream);
    for (auto& kv : srv->tickets) {
        if (kv.second.tab) kv.second.tab->inflight--;
        free_ticket_memory(srv, kv.second);
    }
    for (int L = 0; L < Server::kLanes; ++L) {
        cudaStreamSynchronize(srv->lanes[L].stream);
        free_lane(srv->lanes[L]);
        if (srv->done_ev[L]) cudaEventDestroy(srv->done_ev[L]);
    }
    if (srv->pool) cudaMemPoolDestroy(srv->pool);  // its memory is all freed by now
    delete srv;
    ctx->server = nullptr;
}

}  // namespace sch
