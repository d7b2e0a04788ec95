/*
 * fqsl -- squashing factor Q and twist number Tw of magnetic field lines
 * traced through a gridded 3D field on one NVIDIA GB300 (sm_103a).
 *
 * The operations follow Zhang, Chen, Liu & Wang (2022), "FastQSL: A Fast
 * Computation Method for Quasi-separatrix Layers" (ApJL; arXiv:2208.12569):
 *   - field lines dr/ds = B/|B| (Sec. 2.1, Eq. rb), traced from every seed of
 *     a plane or a volume lattice in both directions until they leave the box,
 *     with trilinear interpolation (Sec. 2.2, Eqs. interp, w0, w1) and the
 *     step-adaptive RKF45 scheme whose tolerance is in grid cells (Sec. 2.3);
 *   - Q = (a^2+b^2+c^2+d^2)/|det D| with |det D| -> |Bn1/Bn2| (Sec. 1, Eqs.
 *     D+-, Q+-, Bn1), D from neighbouring footpoints on an auxiliary plane S0
 *     (Method I, Sec. 2.1, Eqs. D+-2, D+-3; obliquity-scaled tolerance and
 *     local rotation of S0, Sec. 4, Eq. tol) or from deviation vectors
 *     (Method II, Sec. 2.1, Eqs. rb2, q_scott);
 *   - Tw = int (curl B . B)/(4 pi B^2) dl (Sec. 1, Eq. tw) from a curl grid,
 *     and the field-line length (Sec. 2.4).
 *
 * Conventions shared by every entry point
 *   - Every call is asynchronous on the CUDA stream it is given (a
 *     cudaStream_t passed as void*, NULL = the legacy default stream) and
 *     returns a status; no exception crosses this boundary. Argument errors are
 *     detected on the host before anything is launched. A thread-local message
 *     for the last error is available from fqsl_last_error().
 *   - Pointers named *_dev are device pointers. Caller-owned buffers must be
 *     contiguous, 16-byte aligned and stay valid until the stream has run the
 *     call. The library never frees caller memory.
 *   - B layout: nx*ny*nz nodes, x fastest then y then z, three components per
 *     node innermost: B[((k*ny + j)*nx + i)*3 + c], node (i,j,k) at physical
 *     origin + (i*dx, j*dy, k*dz).
 *   - Per-line problems are not errors: they are reported in status[] (the
 *     FQSL_LINE_* bits) and give NaN in Q (and Tw) as documented below.
 *   - Index coordinates xi = (r - origin)/spacing are used internally; step
 *     sizes and tolerances are in cells.
 */
#ifndef FQSL_H
#define FQSL_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* symbols exported from libfqsl.so */
#if defined(__GNUC__)
#define FQSL_API __attribute__((visibility("default")))
#else
#define FQSL_API
#endif

typedef struct fqsl_field_s *fqsl_field;

/* A taped map: the step sequence, checkpoints and line records of one plane or
 * volume map traced with params->tape = 1, which fqsl_backward differentiates.
 * Library-owned; made by the taped call, released by fqsl_tape_destroy. */
typedef struct fqsl_tape_s *fqsl_tape;

typedef enum {
    FQSL_OK = 0,
    FQSL_ERR_ARG = 1,         /* invalid argument; nothing was launched */
    FQSL_ERR_CUDA = 2,        /* a CUDA runtime call failed (message has the CUDA error) */
    FQSL_ERR_OOM = 3,         /* device memory could not be allocated */
    FQSL_ERR_TIMEOUT = 4,     /* reserved: no kernel of this library waits on anything; every device loop
                                 is bounded (a line that uses max_steps ends with FQSL_LINE_MAXSTEPS) */
    FQSL_ERR_UNSUPPORTED = 5  /* valid request the library does not implement */
} fqsl_status;

/* Element types of B, and tracing precisions (fqsl_params.precision):
 *   FQSL_F32        FP32 cube and stepping; error norm in FP32; length and Tw
 *                   as compensated FP32 sums formed in FP64 per direction;
 *                   tolerance, footpoints, Bn and Q assembly in FP64
 *   FQSL_F64        FP64 throughout; reproduces a plain FP64 evaluation of the
 *                   method bit for bit
 *   FQSL_F32_ACC64  as FQSL_F32 but the error norm and the length/Tw sums are
 *                   accumulated in FP64 at every step (precision only) */
typedef enum { FQSL_F32 = 0, FQSL_F64 = 1, FQSL_F32_ACC64 = 2 } fqsl_dtype;

/* fqsl_field_create flags: which packed node records to build. */
#define FQSL_PACK_F32 1u   /* 32-byte records {Bx,By,Bz,Jx | Jy,Jz,0,0} in float */
#define FQSL_PACK_F64 2u   /* 64-byte records {Bx,By | Bz,Jx | Jy,Jz | 0,0} in double */
#define FQSL_PACK_GRADB 4u /* also the grad(B/|B|) node grid for Method II way 1 (Sec. 4, Eq. grad_B):
                              48-byte FP32 and/or 80-byte FP64 records, for the precisions packed */

/* per-line status bits (status[] output) */
#define FQSL_LINE_MAXSTEPS 1u  /* max_steps trial steps used before both ends were found */
#define FQSL_LINE_NULL_B   2u  /* |B| = 0 (or not finite) at an evaluation */
#define FQSL_LINE_STALL    4u  /* a step was accepted at h_min above tolerance */
#define FQSL_LINE_MIXED    8u  /* Method I: no valid difference along one lattice axis at one end */
#define FQSL_LINE_OUTSIDE 16u  /* seed outside the box */
#define FQSL_LINE_ROTATED 32u  /* Method I: S0 rotated perpendicular to B at this seed */
#define FQSL_LINE_CHORD   64u  /* an end was placed on the chord after grazing the face */

/* Tracing and Q parameters. fqsl_params_default() fills the documented
 * defaults; all lengths are in cells. */
typedef struct {
    int method;           /* 1 = neighbour differences (Method I), 2 = deviation vectors (Method II) */
    int gradb_way;        /* Method II gradient of B/|B|: 1 = node grid (Eq. grad_B), 2 = +-eps differences */
    int precision;        /* FQSL_F32 (default), FQSL_F64 or FQSL_F32_ACC64 (see fqsl_dtype) */
    int refill_lanes;     /* scheduling: a warp takes new seeds once this many of its 32 lanes are idle
                             (1..32; 0 = library default). Results do not depend on it. */
    double tol;           /* tol_perp (Method I; scaled per line by |Bn0/B|^tol_exp) or tol (Method II, twist); default 10^-3.2 */
    double h0;            /* initial step, default 0.5 */
    double h_min;         /* smallest step, default 1e-6 */
    double h_max;         /* largest step, default 4 */
    long long max_steps;  /* trial steps per line over both directions, default 100000 (< 2^31) */
    double rot_thresh;    /* rotate S0 below this |Bn0/B| (interior planes), default 0.05 */
    double tol_exp;       /* obliquity exponent of Eq. tol, default 1.5 */
    double graze;         /* smallest outward face-normal velocity of the exit step, default 1e-3 */
    double eps_way2;      /* Method II way-2 offset, default 1e-3 */
    int sync_dirs;        /* scheduling: 1 = the lanes of a warp start their second directions together,
                             0 = each lane at once, -1 = library default. Results do not depend on it. */
    int chunk_tiles;      /* scheduling: 8x4-seed tiles a warp takes per grab of the work counter
                             (1..64; 0 = default 1; batches always take 1). Results do not depend on it. */
    int blocks_per_sm;    /* scheduling: resident 128-thread blocks per SM of the persistent tracer
                             (0 = as many as fit). Results do not depend on it. */
    int tape;             /* 1: fqsl_qmap_plane / fqsl_qmap_volume (Method I) also record the step tape
                             that fqsl_backward differentiates, into the call's tape_or_null (0 = default).
                             Results do not depend on it. */
    int tape_chunk;       /* steps per tape chunk, i.e. the checkpoint interval k of the reverse sweep
                             (1..32; 0 = default 16) */
    int reverse_precision; /* precision of fqsl_backward's reverse sweep for this taped map: -1 (default)
                             = precision; FQSL_F32, FQSL_F32_ACC64 (float state, double node grid) or
                             FQSL_F64; the field must be packed in it */
    int qperp;            /* Method II: 1 = Q_perp, with S1 and S2 turned perpendicular to the line at its
                             ends (Sec. 2.1, after Titov 2007): in Eq. q_scott n = B/|B| at each end, so
                             U~ = U - (U.B)/(B.B) B and B_n,e = |B_e|; 0 (default) = Q on the exit faces.
                             Method I returns FQSL_ERR_UNSUPPORTED for 1 */
    int scheme;           /* 0 = RKF45 (default); 1 = fixed-step 3/8-rule RK4 (Sec. 2.3): every trial is one
                             Kutta 3/8 step of the line's fixed size, always accepted (tol, h0, h_max unused).
                             A Method I lattice seed steps max(step |Bn0/B|, step_min) (Sec. 4 Eq. step);
                             rotated seeds, their extra lines, Method II lines and seed lists step `step`.
                             A grazing exit halves the step for the rest of the direction (down to h_min).
                             On a stretched grid the step is in cells of each trial's start cell.
                             Batches take it (all entries step with it). With tape = 1 (uniform grids) the tape
                             holds every step taken, grazing halvings included, and fqsl_backward
                             reverses the 3/8 rule's four stages */
    double step;          /* scheme 1: step_perp in cells, default 3.0 (Method I in the paper's Table 1) */
    double step_min;      /* scheme 1: lower bound of Eq. step in cells, default 0.15 = 3.0 x rot_thresh (the
                             paper gives no value) */
} fqsl_params;

/* Output buffers of one call (caller-owned device memory, n = number of
 * seeds; any pointer may be NULL to skip that output).
 *   Q        double[n]   squashing factor (NaN if status has MAXSTEPS, NULL_B,
 *                        OUTSIDE or MIXED)
 *   Tw       double[n]   twist number over the whole line (NaN if MAXSTEPS,
 *                        NULL_B or OUTSIDE)
 *   length   double[n]   physical field-line length (same NaN rule as Tw)
 *   r1, r2   double[3n]  physical footpoints. End 1 is the footpoint on the
 *                        side of S0 opposite to its normal n0 = unit(u x v)
 *                        (for a seed list: the backward end); end 2 the other.
 *   face1, face2 int8[n] exit face of each end: 0 x-min, 1 x-max, 2 y-min,
 *                        3 y-max, 4 z-min, 5 z-max, -1 none
 *   status   uint8[n]    FQSL_LINE_* bits
 *   steps    int32[n]    RKF45 trial steps (accepted, rejected and exit steps) */
typedef struct {
    double *Q, *Tw, *length, *r1, *r2;
    int8_t *face1, *face2;
    uint8_t *status;
    int32_t *steps;
} fqsl_out;

/* Fill *p with the defaults documented in fqsl_params. */
FQSL_API void fqsl_params_default(fqsl_params *p);

/* Library version string. */
FQSL_API const char *fqsl_version(void);

/* Message of the last failing call on this host thread ("" if none). */
FQSL_API const char *fqsl_last_error(void);

/* Build a field handle from a B cube (Sec. 2.2: B known at every node of a
 * uniform Cartesian grid). B_dev: device array in the layout above, of
 * b_dtype (FQSL_F32 or FQSL_F64); nx, ny, nz >= 2; spacing > 0. The library
 * computes curl B at the nodes (2nd-order central differences inside,
 * 2nd-order one-sided on the faces, first order on a 2-node axis: the curl grid
 * of Eq. tw) and packs B with it into node records of the precisions asked for
 * in flags (FQSL_PACK_F32 and/or FQSL_PACK_F64; FQSL_PACK_GRADB adds the
 * gradient grid of B/|B| for Method II way 1). The handle owns those
 * records and its scratch memory; the caller may free B_dev once the stream has
 * run the call. Errors: FQSL_ERR_ARG (null pointers, sizes, flags),
 * FQSL_ERR_OOM, FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_field_create(const void *B_dev, fqsl_dtype b_dtype, long long nx, long long ny,
                              long long nz, const double origin[3], const double spacing[3],
                              unsigned flags, void *cuda_stream, fqsl_field *out);

/* Build a field handle on a stretched (rectilinear) grid (Sec. 2.2: nodes
 * [x_i, y_j, z_k] from three increasing coordinate arrays; Sec. 2.3: step and
 * tolerance scaled per cell). x, y, z: HOST arrays of nx, ny, nz strictly
 * increasing finite coordinates (copied; the caller keeps ownership). B_dev,
 * b_dtype, nx, ny, nz, flags and cuda_stream as in fqsl_field_create
 * (FQSL_PACK_GRADB builds the gradient grid with the stencils below).
 * Interpolation finds a point's cell (the largest i with x_i <= x, clamped to
 * [0, n-2]; the paper uses a binary search, the library a bucket table that
 * gives the same cell) and weights it by Eqs. w0, w1. Curl B and grad(B/|B|)
 * take the 2nd-order three-point differences of a non-uniform axis
 * (one-sided on the faces). Each trial step is scaled by the widths w of the
 * cell it starts in: d r/d tau = B/|bt| with bt_a = B_a/w_a, and the error is
 * measured in those cells, so step, h_min, h_max and tol stay in cells.
 * Handles made here serve fqsl_qmap_plane, fqsl_qmap_volume,
 * fqsl_qmap_plane_static and fqsl_twist with Method I and Method II (way 2
 * offsets +-eps_way2 cells of the trial's start cell) and both schemes, and
 * the step tape of either scheme (fqsl_backward differentiates the map with
 * each step's start-cell widths held fixed, and with the reverse sweep in the
 * taped map's state precision: FP64 with FP64, FP32 or FP32_ACC64 with FP32);
 * batches return FQSL_ERR_UNSUPPORTED. Errors:
 * FQSL_ERR_ARG (null pointers, sizes, flags, coordinates not strictly
 * increasing or not finite, coordinates that collapse in float when
 * FQSL_PACK_F32 is asked for), FQSL_ERR_OOM, FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_field_create_rect(const void *B_dev, fqsl_dtype b_dtype, long long nx, long long ny,
                                            long long nz, const double *x, const double *y, const double *z,
                                            unsigned flags, void *cuda_stream, fqsl_field *out);

/* Replace the field's B by a new cube of the same shape and spacing (for a
 * time series of snapshots): recomputes curl B and repacks every record
 * precision the handle holds, asynchronously on cuda_stream, without
 * allocating. Errors: FQSL_ERR_ARG, FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_field_update(fqsl_field field, const void *B_dev, fqsl_dtype b_dtype, void *cuda_stream);

/* Release a field handle and everything it owns (synchronises the device). */
FQSL_API fqsl_status fqsl_field_destroy(fqsl_field field);

/* Q, Tw, length and footpoints on the cell-centred plane lattice
 *   seed(i,j) = origin + (i + 1/2) u + (j + 1/2) v,  0 <= i < nu, 0 <= j < nv,
 * output index i + nu*j. S0 is the plane spanned by u and v (u . v = 0
 * required), with normal n0 = unit(u x v); the refined lattice spacing delta
 * of Method I is |u| along u and |v| along v (Sec. 2.1). On a plane that lies
 * on a box face no rotation of S0 is done; elsewhere seeds with |Bn0/B| <
 * rot_thresh use S0 perpendicular to B and four extra lines at +-delta along
 * its axes, delta = min(|u|,|v|) (Sec. 4). With params->method = 2 every line
 * carries the deviation vectors U, V of the frame perpendicular to B at its
 * seed (Sec. 2.1, Eq. rb2) and Q follows Eq. q_scott; gradb_way 1 needs a
 * field packed with FQSL_PACK_GRADB. The field must have been packed in
 * params->precision.
 * tape_or_null: used only with params->tape = 1 (Method I), and then required.
 * If *tape_or_null is NULL the call makes a new tape and stores it there;
 * otherwise it records this map into the given tape, replacing what that tape
 * held (its buffers are reused and grown as needed). A tape records one map of
 * one field; several tapes may hold maps of the same field at once (for example
 * Q on two planes in one loss), each differentiated by its own fqsl_backward.
 * Calls that use the same tape must not overlap. If a call that made a new
 * tape fails, the tape is released and *tape_or_null is NULL again.
 * Errors: FQSL_ERR_ARG (including params->tape = 1 with tape_or_null NULL),
 * FQSL_ERR_UNSUPPORTED (precision or gradient grid not packed; the tape with
 * Method II or on a stretched grid), FQSL_ERR_OOM, FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_qmap_plane(fqsl_field field, const double origin[3], const double u[3],
                            const double v[3], long long nu, long long nv,
                            const fqsl_params *params, const fqsl_out *out, fqsl_tape *tape_or_null,
                            void *cuda_stream);

/* The same on the 3D lattice seed(i,j,k) = origin + ((i+1/2) sx, (j+1/2) sy,
 * (k+1/2) sz), output index i + nx*(j + ny*k); every z-layer is its own
 * horizontal S0 (Q extended to 3D by being constant along a line, Eq. qline).
 * tape_or_null as in fqsl_qmap_plane. */
FQSL_API fqsl_status fqsl_qmap_volume(fqsl_field field, const double origin[3], const double step[3],
                             long long nx, long long ny, long long nz, const fqsl_params *params,
                             const fqsl_out *out, fqsl_tape *tape_or_null, void *cuda_stream);

/* Tw, length, footpoints, faces, status and steps (no Q; out->Q ignored) for
 * an explicit list of physical seeds seeds_dev[3*n] (double), traced with
 * tol = params->tol (Sec. 2.4: Tw needs little or no refinement). */
FQSL_API fqsl_status fqsl_twist(fqsl_field field, const double *seeds_dev, long long n,
                       const fqsl_params *params, const fqsl_out *out, void *cuda_stream);

/* Per-kernel timing. With timing enabled, every later call on this field
 * records CUDA events on its own stream around its kernels; fqsl_field_times
 * waits for the events of the last call and returns their durations in
 * milliseconds: ms[0] line tracer (lattice or seed list; the FP32 seed
 * pre-pass runs just before it and is not included), ms[1] tracer of the
 * rotated-S0 extra lines (0 if not launched), ms[2] Q assembly. Errors:
 * FQSL_ERR_ARG (NULL, or no timed call yet), FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_field_set_timing(fqsl_field field, int enable);
FQSL_API fqsl_status fqsl_field_times(fqsl_field field, float ms[3]);

/* One seed plane of a batch: seed(i,j) = origin + (i+1/2) u + (j+1/2) v as in
 * fqsl_qmap_plane. */
typedef struct {
    double origin[3], u[3], v[3];
    long long nu, nv;
} fqsl_plane;

typedef struct fqsl_batch_s *fqsl_batch;

/* A batch plan: n (field, plane, outputs) entries of uneven sizes mapped
 * together (Method I; the paper has no counterpart, it maps one plane at a
 * time). Every entry computes exactly what fqsl_qmap_plane computes for it.
 * Creation validates the entries like fqsl_qmap_plane, allocates the scratch
 * of all entries and uploads the entry descriptors (it synchronises the
 * device). fields must share the current device and be packed in
 * params->precision; outs[k] receives entry k's nu*nv results and must stay
 * valid for the plan's lifetime. Errors: FQSL_ERR_ARG, FQSL_ERR_UNSUPPORTED,
 * FQSL_ERR_OOM, FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_batch_create(const fqsl_field *fields, const fqsl_plane *planes, const fqsl_out *outs,
                                       int n, const fqsl_params *params, fqsl_batch *out);

/* Run a batch plan on cuda_stream: one seed pre-pass (FP32), one persistent
 * tracer launch over the work items of all entries (a device counter hands
 * out 8x4-seed tiles of any entry), one launch for the rotated-S0 extra lines
 * of all entries (if any plane is interior) and one assembly launch. No
 * allocation and no host synchronisation happen here. */
FQSL_API fqsl_status fqsl_batch_run(fqsl_batch batch, void *cuda_stream);

/* Release a batch plan (synchronises the device; the fields stay). */
FQSL_API fqsl_status fqsl_batch_destroy(fqsl_batch batch);

/* Largest nu*nv accepted by fqsl_qmap_plane_static. */
#define FQSL_STATIC_MAX_SEEDS 65536

/* fqsl_qmap_plane without any memory allocation (the paper has no counterpart;
 * this is a deployment variant). Some callers cannot call cudaMalloc: for
 * example an application whose device memory is owned entirely by its own
 * fixed arena or pool allocator, or a latency-critical loop that cannot afford
 * the device-wide synchronisation that growing library scratch (cudaFree +
 * cudaMalloc) implies. This entry point computes exactly what fqsl_qmap_plane
 * computes, with the same arguments, outputs and errors, but keeps its
 * per-line scratch (line records, work counters, rotated-S0 buffers) in one
 * static device array of about 22 MiB that is part of the library: every GPU
 * that loads the library holds that array until the process exits, and this
 * call allocates nothing. Limits and rules:
 *   - nu*nv <= FQSL_STATIC_MAX_SEEDS, else FQSL_ERR_ARG with a message;
 *   - the first call on a device (with that device current) looks up the
 *     array's device address once. Under CUDA's lazy module loading (the
 *     default) that lookup is also what loads the part of the library holding
 *     the array, so the array's device memory is reserved then: the first call
 *     can fail with FQSL_ERR_OOM (or FQSL_ERR_CUDA) if the device is full.
 *     Make that first call at start-up, before the caller's arena takes the
 *     device memory and before any stream capture;
 *   - all calls share the one array: the call clears what must start at zero,
 *     and calls whose work overlaps on the GPU (other streams, other host
 *     threads) race on it, so serialise them;
 *   - the field handle (created beforehand by fqsl_field_create or
 *     fqsl_field_create_rect) is only read, apart from the timing events of
 *     fqsl_field_set_timing, which this call records like fqsl_qmap_plane;
 *   - Method I only (params->method = 2 gives FQSL_ERR_UNSUPPORTED), with
 *     either scheme, on uniform and stretched grids.
 */
FQSL_API fqsl_status fqsl_qmap_plane_static(fqsl_field field, const double origin[3], const double u[3],
                                            const double v[3], long long nu, long long nv,
                                            const fqsl_params *params, const fqsl_out *out, void *cuda_stream);

/* Reverse mode (the paper has no derivative; this is the discrete adjoint of
 * the computation it defines). For the plane or volume map recorded in tape
 * (by fqsl_qmap_plane or fqsl_qmap_volume on this field with params->tape = 1,
 * Method I), accumulate
 *   dB += d/dB ( sum_s dQ[s] Q[s] + dTw[s] Tw[s] )
 * where the derivative is that of the traced computation with each line's
 * accepted step sizes, exit faces and exit kinds (exit step onto a face, the
 * same with the point clamped into the box, chord after an exiting step)
 * frozen at their traced values -- so rejected trials contribute nothing --
 * while every position, stage value (Sec. 2.3), trilinear weight (Sec. 2.2,
 * Eq. interp), exit-step length, chord parameter, Bn at the seed and at both
 * ends (Eq. Bn1), the Method I difference stencils' values (Eqs. D+-2, D+-3)
 * and the curl grid (Eq. tw) vary with B.
 *   dQ_dev, dTw_dev  double[seeds] per-seed weights in the map's output order
 *                    (either may be NULL = 0). Seeds whose Q is NaN (status
 *                    MAXSTEPS, NULL_B, OUTSIDE or MIXED) contribute nothing
 *                    through Q. A seed whose S0 was rotated (ROTATED, plane
 *                    maps) takes Q from its four taped extra lines; its
 *                    derivative also carries the rotated frame's dependence
 *                    on B at the seed. NaN or infinite weights count as 0.
 *   dB_dev           B-shaped array (layout of fqsl_field_create) of db_dtype
 *                    (FQSL_F32 or FQSL_F64), accumulated into, not cleared.
 * The reverse sweep runs in the taped call's params->reverse_precision
 * (default: its precision). When that is the tape's precision class, the
 * taped call kept every accepted step's state and stage derivatives for as
 * many chunks as the tape's previous backward call needed (two per direction
 * at first; at most 4 GiB); otherwise, or when the map took more chunks, they
 * are recomputed from the checkpoints taken every params->tape_chunk accepted
 * steps. The node
 * adjoints accumulate in float (FQSL_F32) or double
  * (FQSL_F32_ACC64, FQSL_F64). The field must not be updated between the
 * taped call and this one; other maps of the field (taped into other tapes or
 * not) may run in between. The call waits on the host until the taped
 * call's tracers have finished (not for later work on the stream), to read
 * how many chunks of the tape's pool they used; if the pool did not suffice, it
 * traces the map again into the same tape with a larger pool. It therefore
 * cannot be captured in a CUDA graph. The tape keeps its map: fqsl_backward may run on it again with other
 * weights. With timing enabled, fqsl_field_times reports ms[0] = reverse
 * sweep, ms[1] = 0, ms[2] = curl transpose. Errors: FQSL_ERR_ARG (NULL field
 * or tape, a tape of another field or without a complete map, the field
 * updated since, NULL or misaligned pointers, db_dtype), FQSL_ERR_OOM,
 * FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_backward(fqsl_field field, fqsl_tape tape, const double *dQ_dev, const double *dTw_dev,
                                   void *dB_dev, fqsl_dtype db_dtype, void *cuda_stream);

/* The step sequence of the map held by a tape (the paper has no
 * counterpart; for inspection and for replaying a map's exact steps
 * elsewhere). For half-line hl = 2 s + e (seed s, end e = 0 for end 1):
 * nsteps_dev[hl] accepted steps (0 with code -1 for a line with MAXSTEPS,
 * NULL_B or OUTSIDE), h_dev[hl * cap + i] their sizes in cells in order when
 * nsteps_dev[hl] <= cap (cap = 0: counts only), code_dev[hl] how the direction ended (16 + face: exit step
 * onto that face; 40 + face: the same with the other coordinates clamped into
 * the box; 48 + face: chord onto that face after an exiting step of size
 * hx_dev[hl], which is 0 otherwise). Device arrays of 2 x seeds elements
 * (h_dev: 2 x seeds x cap). The pool must have sufficed (run fqsl_backward first
 * if unsure). Errors: FQSL_ERR_ARG, FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_tape_export(fqsl_tape tape, int cap, int32_t *nsteps_dev, int32_t *code_dev,
                                      double *hx_dev, double *h_dev, void *cuda_stream);

/* Release a tape and its device memory (synchronises the device). A tape may
 * outlive its field, but is then only good for fqsl_tape_export and this
 * call. Errors: FQSL_ERR_ARG (NULL). */
FQSL_API fqsl_status fqsl_tape_destroy(fqsl_tape tape);

/* The log-Q / Tw misfit of two maps and its gradient (a loss for
 * fqsl_backward; the paper has no counterpart):
 *   loss = (1/m) sum over usable seeds of (log10 Q - log10 Q_t)^2 + w_tw (Tw - Tw_t)^2,
 * usable = Q, Q_t, Tw, Tw_t finite, Q > 0, Q_t > 0 and (status_dev given) no
 * MAXSTEPS, NULL_B, OUTSIDE, MIXED or ROTATED bit; m = their number (1 if
 * none). Writes *loss_dev and dQ_dev[s], dTw_dev[s] = d loss / d Q[s], Tw[s]
 * (0 for seeds not usable; loss_dev, dQ_dev, dTw_dev may be NULL). sums_dev:
 * double[2] scratch of the caller. All pointers are device pointers of n
 * elements (status_dev may be NULL). dQ_dev and dTw_dev may be Q_dev and
 * Tw_dev themselves (in place); other partial overlaps of outputs and inputs
 * are not allowed. Errors: FQSL_ERR_ARG, FQSL_ERR_CUDA. */
FQSL_API fqsl_status fqsl_loss_logq_tw(long long n, const double *Q_dev, const double *Tw_dev,
                                       const double *Qt_dev, const double *Twt_dev, const uint8_t *status_dev,
                                       double w_tw, double *sums_dev, double *loss_dev, double *dQ_dev,
                                       double *dTw_dev, void *cuda_stream);

/* Synchronise cuda_stream and report device-side failures recorded by earlier
 * calls on this field: the reverse sweep's kernels check every index they
 * form and record, instead of making the access, the first that is out of
 * range and the number of such checks (FQSL_ERR_CUDA, the message names the
 * first check and its value). The record is cleared. */
FQSL_API fqsl_status fqsl_field_check(fqsl_field field, void *cuda_stream);

/* Testing aid (the paper has no counterpart): every later device allocation
 * the library makes that is larger than `bytes` fails as if the device were
 * out of memory, so that callers' and the library's out-of-memory paths can
 * be exercised without exhausting the GPU. 0 removes the cap (the default).
 * Process-wide; allocations already made are kept. */
FQSL_API void fqsl_debug_alloc_cap(unsigned long long bytes);

#ifdef __cplusplus
}
#endif

#endif /* FQSL_H */
