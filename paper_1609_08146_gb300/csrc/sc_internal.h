// Internal interface between the host side of libsc (handles, FP64 node
// tables, scheduling) and its CUDA kernels.  Not part of the C-ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace sc {

// Node tables are stored in tiles of kTile nodes; each tile holds kFields
// fields of kTile floats (structure of arrays inside the tile), so one tile is
// one contiguous 16-byte-aligned block that a single bulk copy stages into
// shared memory.
constexpr int kTile = 32;
constexpr int kFields = 10;
constexpr int kTileFloats = kTile * kFields;          // 320
constexpr int kTileBytes = kTileFloats * 4;           // 1280
enum NodeField {
    F_PX = 0, F_PY, F_PZ,  // node position P (focus at the origin)
    F_PN,                  // |P| = z + 2f on the paraboloid
    F_W,                   // optical path difference W at the node
    F_JX, F_JY, F_JZ,      // (N x B~) w / (2 pi): surface current times weight
    F_RHO,                 // (N . E~) w / (2 pi), or q / (2 pi) on a rim node
    F_PAD
};

// FP64 table for the plain FP64 path: one node per record.
struct Node64 {
    double px, py, pz, pn, w, jx, jy, jz, rho, pad;
};

// Error bits raised by kernels.
enum : int { ERR_TIMEOUT = 1, ERR_NEAR_SURFACE = 2, ERR_NONFINITE = 4 };

// Accumulator layout of one (point, omega) partial sum: E (re, im) x 3 then
// B (re, im) x 3.
constexpr int kAcc = 12;

struct FieldLaunch {
    const float* nodes;     // tiled table: surface tiles then rim tiles
    int n_surf_tiles;
    int n_rim_tiles;
    int tiles_per_split;    // surface tiles per split
    int n_splits;           // surface splits; split index n_splits = the rim
    int flush_tiles;        // tiles summed in FP32 before each compensated fold
    const double* pts;      // [n_pts][3] (this chunk)
    int n_pts;
    int n_omega;            // omegas in this chunk
    float om_hi0, om_lo0;   // first omega of the chunk as a float-float pair
    float dom_hi, dom_lo;   // grid step as a float-float pair
    float2* ws;             // compensated partials (hi, lo) [n_splits + 1][n_pts][n_omega][kAcc]
    int* err;               // device error word
};

// One request (or one chunk of a request) of a batched field-sum launch:
// work items are (point block, split) pairs, point blocks fastest, numbered
// from item0.
struct WorkReq {
    FieldLaunch f;
    int pb;                 // point blocks of f.n_pts
    int cls;                // kernel class (field_class)
    long long item0;        // first global item of this request
};

// A launch over many requests of one kernel class.  Queue mode: reqs is a
// device array sorted by item0 and CTAs take items from *queue (reset to 0
// before the launch).  Grid mode (reqs == nullptr): the single request `one`,
// item = blockIdx.x, grid = n_items.
//   abort      per-launch flag (reset to 0 before the launch, or null): a
//              CTA whose bounded wait runs out sets it, and every CTA stops
//              taking items once it is set, so a lost copy ends the launch
//              after one wait limit instead of one per item;
//   fail_tile  failure-path test (-1 off): the CTA that runs item 0 leaves
//              the bulk copy of that item's node tile fail_tile unissued, so
//              the wait for it runs out (no fault, no copy in flight).
struct BatchLaunch {
    const WorkReq* reqs;
    WorkReq one;
    int n_req;
    long long n_items;
    int* queue;
    int* err;
    int* abort;
    int fail_tile;
};

// Kernel class for a chunk of n_omega (<= 2048) omegas: 0..20 the direct
// kernel (1 to 32 threads per point, 1..8 omegas per thread, up to 256
// omegas), 21..23 the grouped kernel with 64, 128, 256 threads per point,
// 24..29 alternative direct layouts for the autotuner.
constexpr int kNumClasses = 30;
constexpr int kFirstGroupedClass = 21;  // grouped classes 21..23
constexpr int kFirstAltClass = 24;      // alternative direct layouts 24..29 (alt_field_class)
int field_class(int n_omega);
// The alternative direct layout the autotuner times against field_class(n)
// for n omegas, or -1 where there is none: 8 omegas on one thread of 8
// (against two of 4), 9..16 on four threads (against two), 33..64 on sixteen
// (against eight), 65..128 on 32 threads of 4 (against sixteen of 8).
int alt_field_class(int n_omega);
// Threads per point and omegas per thread of a class.
void class_layout(int cls, int* threads_per_point, int* omegas_per_thread);
inline bool is_direct_class(int cls) { return cls < kFirstGroupedClass || cls >= kFirstAltClass; }
// the direct kernel's classes (0 .. kFirstGroupedClass - 1), in sc_field_direct.cu
void direct_field_shape(int cls, int device, int* points_per_item, int* resident_ctas);
int launch_direct_field(int cls, const BatchLaunch& b, int grid, cudaStream_t s);
// Observation points per work item and resident CTAs on the device.
void field_shape(int cls, int device, int* points_per_item, int* resident_ctas);
// Launch one class; grid = CTAs (queue mode: resident slots; grid mode:
// n_items).  Returns kernels launched (1) or a negative cudaError_t.
int launch_field_batch(int cls, const BatchLaunch& b, int grid, cudaStream_t s);

// Single-request FP32 field sum in grid mode (no device descriptor, no
// queue).  Returns kernels launched or a negative cudaError_t.
int launch_field_f32(const FieldLaunch& p, cudaStream_t s);

// FP64 cross-split reduction and epilogue: E = a_n (S_E + (i/k_n) S_rim),
// B = a_n S_B, written as float2 into out[n_omega_total][n_pts_total][3]
// at (omega offset, point offset).
struct ReduceLaunch {
    const float2* ws;       // part 0's partials; part p's follow at p times
                            // (n_splits + 1) * n_pts * n_omega * kAcc
    int n_parts = 1;        // node tables summed, result = sum_p amp_p (S_p + (i/k) rim_p)
    long long amp_stride = 0;  // doubles from one part's amplitudes to the next
    int n_splits;           // surface splits (the rim slot follows)
    int n_pts, n_omega;
    const double* amp;      // [n_parts][..][2] of this chunk: a_n times the part's weight
    const double* kval;     // [n_omega] k_n of this chunk
    float2* E;              // output base (already offset to the chunk)
    float2* B;              // nullable
    long long out_pt_stride_omega;  // n_pts_total * 3
    long long off;          // prefix of n_pts * n_omega over a batch
};
int launch_reduce_f32(const ReduceLaunch& p, cudaStream_t s);
// Reduction of many requests in one launch: reqs is a device array sorted
// by off, total = sum of n_pts * n_omega.
int launch_reduce_batch(const ReduceLaunch* reqs, int n_req, long long total, cudaStream_t s);

// Plain FP64 path: direct sincos per (point, node, omega).
struct Field64Launch {
    const Node64* surf; int n_surf;
    const Node64* rim;  int n_rim;
    int accumulate = 0;                  // add to E, B instead of storing (later parts)
    const double* pts;  int n_pts;
    const double* kval; int n_omega;     // k_n per omega
    const double* amp;                   // [n_omega][2]: a_n times the part's weight
    double2* E; double2* B;              // [n_omega][n_pts][3]
};
int launch_field_f64(const Field64Launch& p, cudaStream_t s);

// Inverse transform: out[t][v] = 2 dk Re sum_n F[n][v] e^{-i k_n t_m}.
struct IdftLaunch {
    const void* F;          // [n_omega][n_vals] complex (float2 or double2)
    int f64;                // element type of F
    int n_omega;
    long long n_vals;
    const double* kval;     // [n_omega]
    const double* t;        // [n_t]
    int n_t;
    double dk;
    float* out;             // [n_t][n_vals]
    float2* phasor;         // scratch [n_omega][n_t]
    int accumulate = 0;     // add to out (a later chunk of omegas) instead of storing
};
int launch_idft(const IdftLaunch& p, cudaStream_t s);

// First correction beyond physical optics (sc_mfie.cu): the current dJ of the
// MFIE's Liouville-Neumann series at every surface node, by a polar rule about
// each node, and the field of dJ at the observation points.  FP64.
struct MfieZern {           // c_j Z_j = P(u^2 + v^2) {1, Re, Im}((u + iv)^m)
    int m;                  // |m|
    int kind;               // 0: m = 0, 1: cos (Re), 2: sin (Im)
    int deg;                // degree of P in u^2 + v^2
    double p[6];            // coefficients of P, constant first (times c_j N_j)
};
struct MfieLaunch {
    int surface;            // 0 paraboloid (f), 2 ellipsoid (c_ell, e_ell)
    double f, c_ell, e_ell;
    double zref;            // incident phase reference e^{-ik(z + zref)}
    double r_max;           // rim of the disk
    int profile, sg_order, pol;
    double w0, cos_a, sin_a;
    const MfieZern* zern;   // [n_zern], optical path in units of lambda0
    int n_zern;
    double r_norm;          // radius of the Zernike unit disk
    const double* gx;       // Gauss-Legendre nodes and weights on [0, 1] [n_rho]
    const double* gw;
    int n_rho, n_phi;
    const double4* geo;     // surface nodes (x, y, z, dS) [n_surf]
    int n_surf;
    const double* kval;     // [n_omega]
    int n_omega;
    double2* dJ;            // out [n_omega][n_surf][3]
};
struct MfieFieldLaunch {
    const double4* geo;     // (x, y, z, dS) [n_surf]
    int n_surf;
    const double2* dJ;      // [n_omega][n_surf][3]
    const double* pts;      // [n_pts][3]
    int n_pts;
    const double* kval;     // [n_omega]
    int n_omega;
    const double* amp;      // a_n [n_omega][2]
    void* E;                // added to: [n_omega][n_pts][3] float2 or double2
    void* B;                // nullable
    int f64;
    long long out_stride_omega;  // n_pts * 3
};
int launch_mfie_current(const MfieLaunch& p, cudaStream_t s);
int launch_mfie_field(const MfieFieldLaunch& p, cudaStream_t s);

// Failure-path self-test: one bounded mbarrier wait that nothing completes.
int launch_wait_selftest(int* err, cudaStream_t s);

// Arithmetic-pipe probes (sc_peaks.cu): kind 0 FP32 FMA, 1 packed FFMA2, 2
// MUFU rsqrt; each thread performs alu_probe_ops_per_thread(iters) of them
// (an FFMA2 counts as two lane-ops).  sink is never written.
int launch_alu_probe(int kind, int iters, float* sink, int grid, int block, cudaStream_t s);
long long alu_probe_ops_per_thread(int iters);
int alu_probe_grid(int kind, int device);  // resident 512-thread blocks on all SMs

// Fixed device scratch of the allocation-free entry point: 64 MiB of static
// device memory per GPU.  static_scratch() returns its device address on
// `device` (looked up once per device with that device current).
constexpr size_t kStaticScratchBytes = size_t(64) << 20;
cudaError_t static_scratch(int device, void** ptr);
// writes k_n = 2 pi (omega0 + n domega), n < count, into device memory k
int launch_kgrid(double* k, double omega0, double domega, int count, cudaStream_t s);

}  // namespace sc
