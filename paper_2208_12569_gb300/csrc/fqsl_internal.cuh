// Internal types shared by the fqsl CUDA translation units (not part of the
// public C ABI in include/fqsl.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "fqsl.h"

namespace fqsl {

// ---------------------------------------------------------------------------
// Packed node records (one gather fetches B and curl B of a node).
//   FP32: 32 B  = float4 {Bx, By, Bz, Jx}, float4 {Jy, Jz, 0, 0}
//   FP64: 64 B  = double2 {Bx, By}, {Bz, Jx}, {Jy, Jz}, {0, 0}
// Node (i,j,k) is record (k*ny + j)*nx + i.
// ---------------------------------------------------------------------------
template <typename T>
struct RecTraits;
template <>
struct RecTraits<float> {
    static constexpr int kVec = 2;  // float4 per record
};
template <>
struct RecTraits<double> {
    static constexpr int kVec = 4;  // double2 per record
};

struct FieldView {
    const void *rec;  // float4* (FP32) or double2* (FP64)
    int nx, ny, nz;
    double o[3];  // origin
    double d[3];  // spacing
    float cmax[3];            // largest cell index per axis, n - 2, as float
    float rd[3];              // 1 / spacing, as float
    int unit;                 // spacing (1, 1, 1): FP64 divisions by it are skipped (exact either way)
    unsigned sy32, sz32;      // FP32 record byte strides along y and z
    const void *grad;         // grad(B/|B|) node records (Method II way 1) or NULL:
                              // FP32 48 B {g0..g8, 0, 0, 0}, FP64 80 B {g0..g8, 0}
    long long nodes;          // nx * ny * nz
    unsigned long long *err;  // adjoint kernels: [0] first failed index check
                              // (code << 56 | value), [1] failed checks; NULL elsewhere
    // Stretched (rectilinear) grid, rect = 1: node coordinates per axis. o is
    // then the first node and d = 1, so FP32 state coordinates (r - o)/d are
    // physical coordinates relative to the first node; the FP64 state is the
    // physical position itself.
    // Cell search: bucket b covers [x_0 + b/bsc, x_0 + (b+1)/bsc) and is no
    // wider than the narrowest cell (unless that would exceed 16 buckets per
    // cell), so it holds at most one node.
    int rect;
    const double *x64[3];    // node coordinates
    const double *dco[3];    // per node, the three coefficients of its d/dx_a stencil (curl B)
    const double2 *cell64[3];  // per cell {x_i, x_{i+1}}
    const int *bkt[3];       // per bucket: the cell of its lower end
    const float4 *cell32[3];   // per cell, relative to x_0 in float: {x_i, x_{i+1}, 1/(x_{i+1} - x_i), 0}
    // per bucket (float), 32 B: {bits of c (the cell of its lower end), x_c, x_{c+1}, 1/w_c},
    // {x_{c+1} or inf when c = n-2, x_{c+2}, 1/w_{c+1}, 0}
    const float4 *bk32[3];
    int nbkt[3];
    double bsc64[3];         // buckets per unit length
    float bsc32[3];
    double lo64[3], hi64[3];  // first and last node coordinate
    float hi32[3];            // x_{n-1} - x_0 in float
};

struct DevParams {
    double tol, h0, hmin, hmax, rot, texp, graze, eps2;
    long long max_steps;
    int method, way;
    int refill;     // minimum idle lanes before a warp takes new seeds
    int sync_dirs;  // lanes wait for each other before their second direction
    int chunk;      // work items per grab of the counter (a multiple of 32)
    int scheme;     // 0 = RKF45, 1 = fixed-step 3/8 rule
    double step, step_min;  // fixed-step scheme: step_perp and Eq. step's floor (cells)
};

// Cell-centred lattice seed(i,j,k) = o + (i+1/2) a1 + (j+1/2) a2 + (k+1/2) a3.
// Work items walk it in tiles of kTileU x kTileV seeds per layer so that a
// warp traces neighbouring seeds together.
constexpr int kTileU = 8;
constexpr int kTileV = 4;

struct Lattice {
    double o[3], a1[3], a2[3], a3[3];
    // the same lattice in index coordinates: (o - origin)/d and a/d
    double xo[3], xa1[3], xa2[3], xa3[3];
    double n0[3];      // unit(a1 x a2)
    long long n1, n2, n3;
    long long tiles_u, tiles_v;
    double du, dv, drot;
    // spacing over lattice step, per axis: d_a/du, d_a/dv, d_a/drot (the FP32
    // assembly scales index-space footpoint differences by these)
    double sdu[3], sdv[3], sdr[3];
    int normal_axis;   // axis of n0 if it is a coordinate axis, else -1
    int allow_rot;     // Method I and some layer may be interior
};

// Per-line results in structure-of-arrays form (library scratch). The FP64
// tracer writes physical footpoints, Bn and the length/Tw totals; the FP32
// tracer writes index-space footpoints and compensated partial sums, which the
// FP32 assembly turns into the same quantities in FP64.
struct LineRecs {
    double *r1, *r2;    // FP64: physical footpoints, 3 per line
    double *bn1, *bn2;  // FP64: B . n at each end
    double *bn0;        // B0 . n0 (or |B0| when S0 is perpendicular to B)
    double *tw, *len;   // FP64: totals
    float *xi1, *xi2;   // FP32: index-space footpoints, 3 per line
    float4 *kacc;       // FP32: per direction {length sum, its carry, Tw sum, its carry}, 2 per line
    double *dev64;      // Method II, FP64: U1, V1, U2, V2 (12 per line)
    double *be64;       // Method II, FP64: B at end 1 and end 2 (6 per line)
    float *dev32;       // Method II, FP32: U1, V1, U2, V2 (12 per line)
    int8_t *f1, *f2;
    uint8_t *st;
    int32_t *steps;
};

// FP32 seed pre-pass output: index-space seed and tol^2, and flags.
constexpr uint8_t kSeedNegS0 = 1;   // end 1 is traced along +B (B0 . n0 < 0)
constexpr uint8_t kSeedDone = 2;    // the line's record is final (outside / null seed)
constexpr uint8_t kSeedRotated = 4; // S0 rotated (Sec. 4)
struct SeedPrep {
    float4 *seed;     // {xi_x, xi_y, xi_z, tol^2}
    uint8_t *flags;
    float4 *fu, *fv;  // Method II: initial deviation vectors U0, V0
};

struct Queue {
    unsigned long long *head;  // work counter of the launch
    unsigned int *rot_count;   // number of rotated seeds
    int32_t *rot_seed;         // rotated slot -> lattice index
    int32_t *rot_slot;         // lattice index -> slot + 1 (0 = not rotated)
};

enum Source { kSrcLattice = 0, kSrcExtra = 1, kSrcList = 2 };

// Step tape of the adjoint's forward pass (lattice lines). Each direction of
// a line (half-line 2 line + end) stores its accepted step sizes in chunks of
// k steps taken from a pool by a device counter; a chunk holds the state at
// its first step (the checkpoint the reverse sweep recomputes from) and the
// index of the previous chunk of the same half-line. The head of a half-line
// names its last chunk, the steps used in it, how the direction ended and its
// orientation; the end record holds the footpoint and, for a chord end, the
// size of the exiting step. A pool that runs out leaves the counter above cap
// (the host re-runs with a larger pool).
constexpr int kTapeExit = 16;         // + face: exit step onto that face
constexpr int kTapeExitClamped = 40;  // + face: the same, other coordinates clamped into the box
constexpr int kTapeChord = 48;        // + face: chord fallback after an exiting step of size hx
struct Tape {
    int k;                      // steps per chunk
    long long cap;              // chunks in the pool
    unsigned long long *next;   // chunks handed out
    int32_t *prev;              // [cap] previous chunk of the half-line, -1 for its first
    void *xi;                   // [cap] T[4]: state at the chunk's first step {x, y, z, 0}
    void *h;                    // [cap * k] T: accepted step sizes
    int4 *head;                 // [halves] {last chunk, steps in it, end code, orientation sign}
    void *xe;                   // [halves] T[4]: {footpoint x, y, z, exiting step of a chord end}
    int32_t *owner;             // [cap] half-line of each chunk
    long long hl_base;          // half-line of a launch's line 0: 0 for lattice lines,
                                // 2 n for the extra lines of rotated seeds (item = 4 slot + q)
    // Optional (NULL = not kept): the states and stage derivatives of every
    // accepted step as the forward computed them, in the reverse sweep's
    // layout, so that it need not recompute them from the checkpoints:
    //   wx [cap][k + 1][kStateStride] T: state {x, y, z, 0} at each step of a
    //      chunk and after its last
    //   wk [cap][k][kStageStride] T: position derivatives of stages 0..4 of
    //      each step (stage s at 3 s, zero padding at 15)
    // (padded so that each state and each step's record is written and read
    // with 16-byte vector accesses). They hold chunks [0, wcap) only; a map
    // that takes more chunks is recomputed from its checkpoints instead.
    void *wx, *wk;
    long long wcap;
};

constexpr int kStateStride = 4;
constexpr int kStageStride = 16;

struct TraceArgs {
    FieldView f;
    DevParams p;
    Lattice lat;
    const double *seeds;  // kSrcList: 3 per seed
    long long nitems;     // work items (kSrcExtra: read from rot_count)
    LineRecs rec;         // primary lines (lattice or list)
    LineRecs ext;         // rotated extra lines, 4 per slot
    Queue q;
    SeedPrep prep;        // FP32 lattice: filled by the seed pre-pass
    Tape tape;            // adjoint forward pass (lattice lines): the step tape
};

// A batch: many (field, lattice) entries traced by one launch. Work items are
// numbered across entries; ibase[b] is the first item of entry b (a multiple
// of 32, so a 32-item chunk never spans two entries), ibase[nent] the total.
struct BatchArgs {
    const TraceArgs *desc;  // per entry (device memory)
    const long long *ibase;
    int nent;
};

struct AssembleArgs {
    FieldView f;          // FP32 records (FP32 assembly: Bn at the footpoints)
    Lattice lat;
    LineRecs rec, ext;
    const int32_t *rot_slot;  // may be NULL
    fqsl_out out;
    long long n;
    int want_q;
    int qperp;  // Method II: Q_perp (end planes perpendicular to B)
};

constexpr unsigned kBad = FQSL_LINE_MAXSTEPS | FQSL_LINE_NULL_B | FQSL_LINE_OUTSIDE;

// Reverse mode of a taped plane map (adjoint.cu).
struct AdjArgs {
    FieldView f;       // records of the traced precision
    DevParams p;
    Lattice lat;
    LineRecs rec;      // the forward pass's line records
    SeedPrep prep;     // FP32: seed positions
    Tape tape;
    const double *dQ, *dTw;    // per-seed weights (NULL = 0)
    double *xbar;              // [2 n][3] adjoint of each footpoint (index coordinates)
    void *acc;                 // [nodes][8] {dB (3), dJ (3), 0, 0}, float or double
    long long n;
    LineRecs ext;              // extra lines of rotated seeds (4 per slot)
    const int32_t *rot_slot;   // lattice index -> rotated slot + 1 (0: not rotated); NULL if none
    const int32_t *rot_seed;   // rotated slot -> lattice index
    const unsigned *rot_count; // rotated seeds of the taped map
    double *xseed;             // [8 n][3] adjoint of each extra half-line's seed (index coordinates)
    // per-step work arrays of the reverse sweep, for chunks 0..chunks-1 (T):
    //   wx [chunk][k + 1][kStateStride] states, wj [chunk][k][12] step
    //   Jacobian J^T (9) and Tw gradient (3), wk [chunk][k][kStageStride]
    //   stage derivatives (the layouts of Tape::wx, wk), wb [chunk][k][3]
    //   adjoint of each step's end state
    long long chunks;
    void *wx, *wj, *wk, *wb;
    int stored;                // wx, wk hold the forward's values (pass A1 only lists the steps)
    int4 *cinfo;               // [chunks] {steps, orientation, half-line, live} (pass A1)
    int32_t *steps;            // [chunks * k] live steps c k + i, compacted (pass A1)
    unsigned long long *nsteps;  // number of entries in steps
};
// mode: 0 = FP32 state and float grid, 1 = FP32 state and double grid, 2 = FP64;
// tape_f64: the tape was written by the FP64 tracer
cudaError_t launch_q_vjp(const AdjArgs &a, int mode, bool tape_f64, cudaStream_t s);
cudaError_t launch_reverse(const AdjArgs &a, int mode, bool tape_f64, cudaStream_t s);
// passes A1, A2, B, C for a map traced with the fixed-step scheme (adjoint_rk38.cu)
cudaError_t launch_reverse_rk38(const AdjArgs &a, int mode, bool tape_f64, cudaStream_t s);
// passes A1, A2, B, C for a map on a stretched grid, either scheme
// (adjoint_rect.cu; the tape is in the sweep's state precision)
cudaError_t launch_reverse_rect(const AdjArgs &a, int mode, cudaStream_t s);
cudaError_t launch_curl_adjoint(const void *acc, bool acc64, const FieldView &g, void *dB, fqsl_dtype dt,
                                cudaStream_t s);
cudaError_t launch_tape_export(const Tape &tp, bool f64, const uint8_t *st, long long halves, int cap, int32_t *ns,
                               int32_t *code, double *hx, double *h, cudaStream_t s);
cudaError_t launch_loss(long long n, const double *Q, const double *Tw, const double *Qt, const double *Twt,
                        const uint8_t *st, double wtw, double *sums, double *loss, double *dQ, double *dTw,
                        cudaStream_t s);

// launch helpers implemented in the .cu files
cudaError_t launch_curl_pack(const void *B, fqsl_dtype bt, const FieldView &g, void *rec32, void *rec64,
                             cudaStream_t s);
cudaError_t launch_trace_f32(const TraceArgs &a, int src, int grid, int block, cudaStream_t s, bool acc64);
cudaError_t launch_trace_f64(const TraceArgs &a, int src, int grid, int block, cudaStream_t s);
// tracers that also write the step tape (a.tape; lattice or extra lines)
cudaError_t launch_trace_tape_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64);
cudaError_t launch_trace_tape_f64(const TraceArgs &a, int src, int grid, cudaStream_t s);
// the same on a stretched grid (RKF45; trace_rect_f32.cu, trace_rect_f64.cu)
cudaError_t launch_trace_tape_rect_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64);
cudaError_t launch_trace_tape_rect_f64(const TraceArgs &a, int src, int grid, cudaStream_t s);
int trace_tape_rect_blocks_per_sm_f32(int src, bool acc64);
int trace_tape_rect_blocks_per_sm_f64(int src);
cudaError_t launch_trace_tape_rect_rk38_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64);
cudaError_t launch_trace_tape_rect_rk38_f64(const TraceArgs &a, int src, int grid, cudaStream_t s);
int trace_tape_rect_rk38_blocks_per_sm_f32(int src, bool acc64);
int trace_tape_rect_rk38_blocks_per_sm_f64(int src);
int trace_tape_blocks_per_sm_f32(int src, bool acc64);
int trace_tape_blocks_per_sm_f64(int src);
// the same with the fixed-step scheme (trace_rk38_f32.cu, trace_rk38_f64.cu)
cudaError_t launch_trace_tape_rk38_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64);
cudaError_t launch_trace_tape_rk38_f64(const TraceArgs &a, int src, int grid, cudaStream_t s);
int trace_tape_rk38_blocks_per_sm_f32(int src, bool acc64);
int trace_tape_rk38_blocks_per_sm_f64(int src);
int trace_blocks_per_sm_f32(int src, bool acc64);
int trace_blocks_per_sm_f64(int src);
// the same on a stretched grid (FieldView::rect)
cudaError_t launch_trace_rect_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64);
cudaError_t launch_trace_rect_f64(const TraceArgs &a, int src, int grid, cudaStream_t s);
int trace_rect_blocks_per_sm_f32(int src, bool acc64);
int trace_rect_blocks_per_sm_f64(int src);
cudaError_t launch_seed_prep_rect_f32(const TraceArgs &a, long long n, unsigned grid, cudaStream_t s);
cudaError_t launch_trace_dev_rect_f32(const TraceArgs &a, int way, int grid, cudaStream_t s);
cudaError_t launch_trace_dev_rect_f64(const TraceArgs &a, int way, int grid, cudaStream_t s);
int trace_dev_rect_blocks_per_sm_f32(int way);
int trace_dev_rect_blocks_per_sm_f64(int way);
// the fixed-step 3/8-rule instantiations (uniform grids; Method I sources and Method II ways)
cudaError_t launch_trace_rk38_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64);
cudaError_t launch_trace_rk38_f64(const TraceArgs &a, int src, int grid, cudaStream_t s);
cudaError_t launch_trace_dev_rk38_f32(const TraceArgs &a, int way, int grid, cudaStream_t s);
cudaError_t launch_trace_dev_rk38_f64(const TraceArgs &a, int way, int grid, cudaStream_t s);
int trace_rk38_blocks_per_sm_f32(int src, bool acc64);
int trace_rk38_blocks_per_sm_f64(int src);
int trace_dev_rk38_blocks_per_sm_f32(int way);
int trace_dev_rk38_blocks_per_sm_f64(int way);
// the fixed-step scheme on a stretched grid
cudaError_t launch_trace_rect_rk38_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64);
cudaError_t launch_trace_rect_rk38_f64(const TraceArgs &a, int src, int grid, cudaStream_t s);
cudaError_t launch_trace_dev_rect_rk38_f32(const TraceArgs &a, int way, int grid, cudaStream_t s);
cudaError_t launch_trace_dev_rect_rk38_f64(const TraceArgs &a, int way, int grid, cudaStream_t s);
int trace_rect_rk38_blocks_per_sm_f32(int src, bool acc64);
int trace_rect_rk38_blocks_per_sm_f64(int src);
int trace_dev_rect_rk38_blocks_per_sm_f32(int way);
int trace_dev_rect_rk38_blocks_per_sm_f64(int way);
// Method II tracers (deviation vectors; way 1 = gradient grid, 2 = +-eps)
cudaError_t launch_trace_dev_f32(const TraceArgs &a, int way, int grid, int block, cudaStream_t s);
cudaError_t launch_trace_dev_f64(const TraceArgs &a, int way, int grid, int block, cudaStream_t s);
int trace_dev_blocks_per_sm_f32(int way);
int trace_dev_blocks_per_sm_f64(int way);
cudaError_t launch_gradb_pack(const void *B, fqsl_dtype bt, const FieldView &g, void *grad32, void *grad64,
                              cudaStream_t s);
cudaError_t launch_assemble_m2_f64(const AssembleArgs &a, cudaStream_t s);
cudaError_t launch_assemble_m2_f32(const AssembleArgs &a, cudaStream_t s);
constexpr int kTraceBlock = 128;
cudaError_t launch_assemble(const AssembleArgs &a, cudaStream_t s);
cudaError_t launch_assemble_f32(const AssembleArgs &a, cudaStream_t s);
cudaError_t launch_seed_prep_f32(const TraceArgs &a, long long n, cudaStream_t s);

// batches
cudaError_t launch_batch_seed_prep_f32(const TraceArgs *desc, const long long *nbase, int nent, long long total,
                                       cudaStream_t s);
cudaError_t launch_batch_extra_prefix(const unsigned *rot_counts, int nent, long long *xbase, cudaStream_t s);
cudaError_t launch_batch_trace_f32(const TraceArgs &a0, const BatchArgs &b, int src, bool acc64, int grid,
                                   cudaStream_t s);
cudaError_t launch_batch_trace_f64(const TraceArgs &a0, const BatchArgs &b, int src, int grid, cudaStream_t s);
int batch_trace_blocks_per_sm_f32(bool acc64, int scheme);
int batch_trace_blocks_per_sm_f64(int scheme);
// the same with the fixed-step scheme (trace_rk38_f32.cu, trace_rk38_f64.cu)
cudaError_t launch_batch_trace_rk38_f32(const TraceArgs &a0, const BatchArgs &b, int src, bool acc64, int grid,
                                        cudaStream_t s);
cudaError_t launch_batch_trace_rk38_f64(const TraceArgs &a0, const BatchArgs &b, int src, int grid, cudaStream_t s);
int batch_trace_rk38_blocks_per_sm_f32(bool acc64);
int batch_trace_rk38_blocks_per_sm_f64();
cudaError_t launch_batch_assemble_f32(const AssembleArgs *desc, const long long *nbase, int nent, long long total,
                                      cudaStream_t s);
cudaError_t launch_batch_assemble_f64(const AssembleArgs *desc, const long long *nbase, int nent, long long total,
                                      cudaStream_t s);

}  // namespace fqsl
