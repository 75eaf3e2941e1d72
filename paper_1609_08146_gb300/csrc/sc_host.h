// sc_host.h -- host-side internals of libsc shared by its translation units:
// the handle structs behind the opaque types of sc.h, the node tables and
// execution lanes of a context, and the functions one unit calls in another.
//   sc_tables.cpp  quadrature, incident field and spectrum, mirror surfaces,
//                  the FP64 node-table builder and context helpers
//   sc_batch.cpp   batched FP32 execution: chunks, split autotuner, graphs
//   sc_serve.cpp   the serving loop (continuous batching of tickets)
//   sc_api.cpp     error and memory helpers and the C-ABI entry points
// Everything here is in namespace sch and hidden from the library's exports
// (only the extern "C" functions of sc.h are visible).
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <list>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "sc.h"
#include "sc_internal.h"

// --------------------------------------------------------------------------
// Handles
struct sc_mirror_t {
    uint64_t id;
    double f, r_min, r_max;
    sc_quadrature q;
    int surface = 0;        // 0 paraboloid, 2 ellipsoid (semi-axis c, focal half-distance e)
    double c = 0.0, e = 0.0;
};

struct sc_incident_t {
    uint64_t id;
    int profile, sg_order, pol;
    int order;                      // 0 collimated, 1 plus the O(eps) longitudinal terms
    int lg_p = 0, lg_l = 0;         // Laguerre-Gauss mode (profile 3)
    double z_waist = 0.0;
    sc_envelope_fn env = nullptr;   // caller's envelope (profile 4)
    void* env_user = nullptr;
    double om_lo = 0.0, om_hi = 0.0, fit_tol = 1e-8;  // band and tolerance of the k fit
    double dip[3] = {0.0, 0.0, 0.0};                  // dipole moment (profile 5)
    double w0, angle;
    std::vector<double> zern;
    int spec_kind;
    double fwhm_t, lambda_c, dlambda, energy;
    int sg_n;
    std::vector<double> s_omega, s_amp, phi;
};

namespace sch {

constexpr double kPi = 3.14159265358979323846;

struct DevBuf {
    void* p = nullptr;
    size_t n = 0;
};

// One node table of an incident.  Every part sums over the same nodes; its
// sums enter the result with a per-omega complex weight w_p(omega_n):
//   PART_ONE 1,  PART_INV_K -i/k_n (the 1/k longitudinal terms of order 1),
//   PART_CHEB_RE T_m(x_n),  PART_CHEB_IM i T_m(x_n)  (x_n = (k_n - kc) / kh,
//   the Chebyshev expansion in k of a k-dependent envelope),
//   PART_IK_POW (i k_n)^m (the terms of the dipole field).
enum { PART_ONE = 0, PART_INV_K = 1, PART_CHEB_RE = 2, PART_CHEB_IM = 3, PART_IK_POW = 4 };

struct TablePart {
    int kind = PART_ONE, m = 0;
    const float* d32 = nullptr;       // surface tiles, then this part's rim tiles
    int n_rim_tiles = 0;
    const sc::Node64* d64 = nullptr;  // surface records, then rim records
    int n_rim = 0;
};

struct Table {
    uint64_t mid = 0, iid = 0;
    float* d32 = nullptr;          // one allocation for every part's FP32 tiles
    int n_surf_tiles = 0, n_rim_tiles = 0;  // (rim: part 0's)
    sc::Node64* d64 = nullptr;     // and one for their FP64 records
    int n_surf = 0, n_rim = 0;
    std::vector<TablePart> parts;
    double kc = 0.0, kh = 1.0;     // Chebyshev band in k of the CHEB parts
    bool fp32_ok = true;           // the incident wavefront focuses on the origin, so the
                                   // compensated FP32 phase is exact (else FP64 only)
    size_t bytes = 0;
    uint64_t last_use = 0;
    int inflight = 0;              // serving batches on the GPU that read this table
};

struct GraphEntry {
    std::vector<unsigned char> sig;
    cudaGraphExec_t exec = nullptr;
    uint64_t last = 0;
};

// An execution lane of the FP32 path: a stream and the device buffers and
// graph cache that one batch in flight needs.  The context's own calls use
// lane `main` (on the caller's stream); the serving loop owns more lanes so
// that batches overlap on the GPU.
struct Lane {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int prio = 0;                   // stream priority of the lane (side streams take it too)
    bool use_graphs = true;         // capture its field launches (if the context does)
    double max_launch_evals = 0.0;  // > 0: bound the evaluations of one launch group
    DevBuf ws, desc, amp, kval;
    cudaStream_t cap_stream = nullptr;
    std::vector<GraphEntry> graphs;
    // one branch per kernel class of a batch: side streams forked from and
    // joined back into the lane's stream (graph branches when captured)
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join_ev;
    cudaEvent_t fork_ev = nullptr;
};

struct Server;

}  // namespace sch

struct sc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    size_t budget = 0;
    size_t held = 0;
    std::string err = "no error";
    std::list<sch::Table> tables;
    uint64_t tick = 0;
    sch::DevBuf pts, outE, outB, tkval, tvals, phasor, specE, specB, tE, tB;
    sch::DevBuf fpts, fspecE, fspecB, ftE, ftB;  // sc_eval_time_domain: points, chunk spectra, E(t), B(t)
    int* d_err = nullptr;
    int* h_err = nullptr;          // pinned
    sc_counters ctr{};
    bool time_field = false;
    long long nodes_per_split = 0;  // 0: choose splits for load balance
    long long flush_nodes = 2048;   // FP32 run length before each compensated fold
    size_t ws_cap = size_t(2) << 30;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pending;
    std::vector<cudaEvent_t> pool;
    // batched execution: lanes, graph counters, split autotuner, serving
    sch::Lane main;
    bool use_graphs = true;
    bool autotune = true;
    bool omega_chunks = true;       // plan omega chunk sizes (else 2048 per chunk)
    bool class_streams = true;      // a batch's kernel classes run as concurrent branches
    bool serve_priority = true;     // serving: short requests first, long ones preemptible
    int tile_layout = -1;           // -1 autotuned, 0 default, 1 alternative layout
    int shape_cls = -1, shape_splits = -1;  // tile shape of the last planned first chunk
    int fail_tile = -1;             // failure-path test: a node-tile copy left unissued
    int mfie_order = 0;             // 1: add the first MFIE correction (sc_eval)
    int mfie_rho = 64, mfie_phi = 128;  // its polar rule about each node
    sch::DevBuf mfie_geo, mfie_zern, mfie_gl, mfie_dJ;
    uint64_t graph_tick = 0;
    uint64_t graph_captures = 0, graph_replays = 0;
    std::map<std::tuple<int, int, int, int, int, int>, int> tuned;  // shape -> split count
    std::mutex mu;                                              // guards all of the above
    sch::Server* server = nullptr;
};

namespace sch {

// ---- errors and device memory (sc_api.cpp)
sc_status fail(sc_ctx* c, sc_status st, const char* fmt, ...);
sc_status cuda_fail(sc_ctx* c, cudaError_t e, const char* what);

#define SC_CUDA(call, what)                              \
    do {                                                 \
        cudaError_t e__ = (call);                        \
        if (e__ != cudaSuccess) return cuda_fail(ctx, e__, what); \
    } while (0)

// grow b to at least `bytes` (synchronizing sync_stream before freeing it)
sc_status ensure(sc_ctx* ctx, DevBuf& b, size_t bytes, cudaStream_t sync_stream);
sc_status ensure(sc_ctx* ctx, DevBuf& b, size_t bytes);
bool is_device_ptr(const void* p);

// ---- node tables, spectra and context helpers (sc_tables.cpp)
struct HostNode {
    double px, py, pz, pn, w, jx, jy, jz, rho;
};

// Host nodes of one table part (see TablePart).
struct HostPart {
    int kind = PART_ONE, m = 0;
    std::vector<HostNode> surf, rim;
};

sc_status spectrum_amps(sc_ctx* ctx, const sc_incident_t* in, const double* om, int n, std::vector<double>& amp);
bool focuses_on_origin(const sc_mirror_t* m, const sc_incident_t* in);
sc_status build_host_parts(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in, std::vector<HostPart>& hp,
                           double& kc, double& kh);
sc_status get_table(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in, Table** out, cudaStream_t stream);
void free_table(sc_ctx* ctx, Table& t);
sc_status request_amps(sc_ctx* ctx, const sc_incident_t* in, const Table* tab, const double* om, int n,
                       std::vector<double>& out);
sc_status check_device_error(sc_ctx* ctx);
cudaEvent_t take_event(sc_ctx* ctx);
void settle_events(sc_ctx* ctx);
sc_status check_points_host(sc_ctx* ctx, const sc_mirror_t* m, const double* pts, int n_pts);
bool uniform_grid(const double* om, int n, double& d);
void radial_rule(const sc_mirror_t* m, std::vector<double>& x, std::vector<double>& w);
void gauss_legendre(int n, double a, double b, std::vector<double>& x, std::vector<double>& w);
void noll_nm(int j, int& n, int& m);
struct SurfPt {
    double z, dzdr, pn, extra;
};
SurfPt surf_at(const sc_mirror_t* m, double r);

// ---- the first MFIE correction (sc_mfie_host.cpp)
// Why the pair cannot take it, or nullptr.
const char* mfie_unsupported(const sc_mirror_t* m, const sc_incident_t* in);
// Adds the field of the first MFIE correction of (m, in) to the outputs dE,
// dB (device, [n_omega][n_points][3], double2 if f64 else float2) on
// ctx->stream; d_amp, d_k: a_n and k_n on the device.
sc_status mfie_correction(sc_ctx* ctx, const sc_mirror_t* m, const sc_incident_t* in, int n_omega,
                          const double* d_pts, int n_points, const double* d_amp, const double* d_k, void* dE,
                          void* dB, bool f64);

// ---- batched FP32 execution (sc_batch.cpp)
struct Chunk {
    sc::FieldLaunch f;      // part 0; ws assigned at execution
    sc::ReduceLaunch rl;    // ws, off assigned at execution
    const Table* tab = nullptr;  // its parts share f's points, omegas and splits
    int n_parts = 1;
    int cls = 0, ppc = 1, pb = 1;
    size_t ws_elems = 0;    // float2 elements, every part (one section each)
};

sc_status plan_request(sc_ctx* ctx, Lane& ln, const Table* tab, const double* omegas, int n_omega, double dom,
                       const double* d_pts, int n_points, const double* d_amp, const double* d_k, float2* dE,
                       float2* dB, std::vector<Chunk>& out);
sc_status run_chunks(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch);
sc_status run_chunk_group(sc_ctx* ctx, Lane& ln, std::vector<Chunk>& ch, size_t& i);
void free_lane(Lane& ln);

// ---- serving (sc_serve.cpp)
struct Ticket {
    const sc_mirror_t* mirror = nullptr;
    const sc_incident_t* incident = nullptr;
    std::vector<double> omegas, host_pts;
    const double* user_pts = nullptr;   // caller's device points (or null)
    int n_points = 0, n_omega = 0;
    double dom = 0.0;
    void* E_user = nullptr;             // caller-owned device outputs (or null)
    void* B_user = nullptr;
    void* E = nullptr;                  // outputs in use
    void* B = nullptr;
    double* pts = nullptr;              // device points in use
    bool own_out = false, own_pts = false;
    size_t bytes = 0;                   // device bytes this ticket holds
    int state = 0;                      // 0 queued, 1 running, 2 done, 3 failed, 4 cancelled
    bool cancel = false;
    sc_status status = SC_OK;
    double t_submit = 0, t_start = 0, t_done = 0;
    int lane = -1;
    Table* tab = nullptr;
    double evals = 0.0;                 // points x surface nodes x omegas
};

struct Server {
    // lanes 0, 1: short requests, high stream priority; lanes 2, 3: long
    // requests, low priority, in launch groups of bounded size
    static constexpr int kLanes = 4;
    static constexpr int kShortLanes = 2;
    bool priority = true;               // sc_ctx::serve_priority when the server started
    // the server's own stream-ordered pool for ticket memory: it keeps what is
    // freed and is warmed at start, so that admitting a request rarely has to
    // grow device memory while other lanes' kernels run (nullptr: default pool)
    cudaMemPool_t pool = nullptr;
    std::thread th;
    bool stop = false;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::map<uint64_t, Ticket> tickets;
    Lane lanes[kLanes];
    cudaEvent_t done_ev[kLanes] = {};
    std::vector<uint64_t> batch[kLanes];
    bool busy[kLanes] = {};
    // a long lane's chunks not yet launched: one bounded group is in flight
    // at a time, the next is launched when it completes
    std::vector<Chunk> pend[kLanes];
    size_t pend_i[kLanes] = {};
    size_t held = 0;                    // bytes of admitted tickets not yet released
    uint64_t next_id = 1;
    int max_batch = 64;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now() const
    {
        return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
};

size_t ticket_bytes(const Ticket& t);
sc_status start_server(sc_ctx* ctx);
void free_ticket_memory(Server* srv, Ticket& t);
void stop_server(sc_ctx* ctx);

}  // namespace sch
