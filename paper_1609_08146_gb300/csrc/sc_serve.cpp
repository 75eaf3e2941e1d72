// sc_serve.cpp -- serving (A9): the server thread that admits, batches and
// completes submitted requests on two lanes.
#include <algorithm>

#include "sc_host.h"

namespace sch {

// ------------------------------------------------------------------------
// Serving (A9): continuous batching of submitted requests.  A server thread
// admits queued requests in arrival order while their device memory (staged
// points and server-owned outputs) fits the context's HBM budget, batches up
// to max_batch of them and runs the batch on a free lane; with two lanes a
// new batch starts while the previous one is still on the GPU, so requests
// that arrive meanwhile overlap with it.  Completion is observed through an
// event per lane; memory returns to the budget when the caller releases the
// ticket.

size_t ticket_bytes(const Ticket& t)
{
    size_t b = 0;
    if (t.own_pts) b += (size_t)t.n_points * 3 * sizeof(double);
    if (t.own_out) b += (size_t)2 * t.n_omega * t.n_points * 3 * sizeof(float2);
    return b;
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
            SC_CUDA(cudaMallocAsync((void**)&t.pts, (size_t)t.n_points * 3 * sizeof(double), ln.stream),
                    "serving points");
            SC_CUDA(cudaMemcpyAsync(t.pts, t.host_pts.data(), (size_t)t.n_points * 3 * sizeof(double),
                                    cudaMemcpyHostToDevice, ln.stream), "stage points");
        } else {
            t.pts = (double*)t.user_pts;
        }
        if (t.own_out) {
            const size_t ob = (size_t)t.n_omega * t.n_points * 3 * sizeof(float2);
            SC_CUDA(cudaMallocAsync(&t.E, ob, ln.stream), "serving outputs");
            SC_CUDA(cudaMallocAsync(&t.B, ob, ln.stream), "serving outputs");
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
    st = run_chunks(ctx, ln, ch);
    if (st != SC_OK) return st;
    SC_CUDA(cudaEventRecord(srv->done_ev[L], ln.stream), "completion event");
    return SC_OK;
}

void serve(sc_ctx* ctx)
{
    Server* srv = ctx->server;
    cudaSetDevice(ctx->device);
    std::unique_lock<std::mutex> lk(ctx->mu);
    while (!srv->stop) {
        bool changed = false;
        // completions
        for (int L = 0; L < Server::kLanes; ++L) {
            if (!srv->busy[L]) continue;
            const cudaError_t q = cudaEventQuery(srv->done_ev[L]);
            if (q == cudaErrorNotReady) continue;
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
        // admission and launch on free lanes
        for (int L = 0; L < Server::kLanes && !srv->queue.empty(); ++L) {
            if (srv->busy[L]) continue;
            // workspace the lanes may still grow into (bounded by the cap)
            size_t reserve = size_t(16) << 20;
            for (int M = 0; M < Server::kLanes; ++M)
                if (srv->lanes[M].ws.n < ctx->ws_cap) reserve += ctx->ws_cap - srv->lanes[M].ws.n;
            std::vector<uint64_t> ids;
            while (!srv->queue.empty() && (int)ids.size() < srv->max_batch) {
                Ticket& t = srv->tickets[srv->queue.front()];
                const size_t b = ticket_bytes(t);
                // admit only what fits next to every lane's full workspace; the
                // first request of an idle server is always admitted
                const bool idle = srv->held == 0 && ids.empty();
                if (ctx->budget && !idle && ctx->held + srv->held + b + reserve > ctx->budget) break;
                t.bytes = b;
                srv->held += b;
                ids.push_back(srv->queue.front());
                srv->queue.pop_front();
            }
            if (ids.empty()) break;
            const sc_status st = launch_batch(ctx, srv, L, ids);
            if (st == SC_OK && ids.empty()) {
                changed = true;
                continue;
            }
            if (st != SC_OK) {
                cudaStreamSynchronize(srv->lanes[L].stream);
                for (uint64_t id : ids) {
                    Ticket& t = srv->tickets[id];
                    if (t.tab) t.tab->inflight--;
                    t.tab = nullptr;
                    t.state = 3;
                    t.status = st;
                    t.t_done = srv->now();
                }
            } else {
                srv->batch[L] = ids;
                srv->busy[L] = true;
            }
            changed = true;
        }
        if (changed) srv->cv.notify_all();
        srv->cv.wait_for(lk, std::chrono::microseconds(100));
    }
}

sc_status start_server(sc_ctx* ctx)
{
    if (ctx->server) return SC_OK;
    Server* srv = new Server();
    for (int L = 0; L < Server::kLanes; ++L) {
        if (cudaStreamCreateWithFlags(&srv->lanes[L].stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&srv->done_ev[L], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            delete srv;
            return fail(ctx, SC_ERR_CUDA, "serving lane set-up failed");
        }
        srv->lanes[L].own_stream = true;
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
    delete srv;
    ctx->server = nullptr;
}

}  // namespace sch
