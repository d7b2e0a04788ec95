/*
 * fqsl_probes -- measurement kernels that give the field-line tracer its
 * roofline ceilings on the GPU at hand (libfqsl_probes.so). The paper has no
 * counterpart: these kernels compute nothing of the method; they measure how
 * fast this GPU serves the two kinds of work the tracer is made of.
 *
 *   - Trilinear gathers of 32-byte FP32 node records {Bx,By,Bz,Jx | Jy,Jz,0,0}
 *     (the layout of fqsl_field_create's FP32 records, node (i,j,k) at record
 *     (k*ny + j)*nx + i): each lane interpolates the 8 corner records of a cell
 *     with one 256-bit read-only load per record and keeps a running sum of
 *     the six interpolated components. Bytes requested per gather: 8 x 32.
 *   - Chains of fused multiply-adds in FP32 or FP64: 8 independent chains per
 *     thread, 2 flops per FMA.
 *
 * Conventions: launches are asynchronous on the given CUDA stream (void* =
 * cudaStream_t, NULL = legacy default stream); time them with events on that
 * stream. Returns 0 on success, 1 for an invalid argument (nothing launched),
 * 2 if the launch failed. Pointers named *_dev are device pointers.
 */
#ifndef FQSL_PROBES_H
#define FQSL_PROBES_H

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define FQSL_PROBE_API __attribute__((visibility("default")))
#else
#define FQSL_PROBE_API
#endif

/* Access patterns of fqsl_probe_gather (per warp of 32 lanes). */
#define FQSL_PROBE_WALK 0   /* an 8x4 tile of points 0.25 cells apart (a warp's tile of neighbouring seeds)
                               that walks 0.4 cells per gather along a straight line drawn at random, and
                               restarts at a random point when it would leave the cube: the locality of a
                               warp tracing neighbouring field lines */
#define FQSL_PROBE_TILE 1   /* the same tile at a new random point for every gather (no reuse between gathers) */
#define FQSL_PROBE_RANDOM 2 /* every lane at its own random point for every gather */

/* Gathers: grid = sms x blocks_per_sm blocks of 128 threads; every lane does
 * `gathers` trilinear gathers. rec_dev: nx*ny*nz records of 32 bytes, 32-byte
 * aligned, finite floats; nx, ny, nz >= 4. sink_dev: float[grid x 128],
 * receives each lane's sum (so that no load is dead). Total bytes requested =
 * sms x blocks_per_sm x 128 x gathers x 256. */
FQSL_PROBE_API int fqsl_probe_gather(const void *rec_dev, int nx, int ny, int nz, int pattern, int gathers,
                                     int sms, int blocks_per_sm, float *sink_dev, void *cuda_stream);

/* FMA chains: grid = sms x blocks_per_sm blocks of 256 threads; every thread
 * runs 8 chains of `iters` FMAs in FP32 (fp64 = 0) or FP64 (fp64 = 1).
 * sink_dev: float[grid x 256] or double[grid x 256]. Total flops =
 * sms x blocks_per_sm x 256 x 8 x iters x 2. */
FQSL_PROBE_API int fqsl_probe_fma(int fp64, int iters, int sms, int blocks_per_sm, void *sink_dev,
                                  void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* FQSL_PROBES_H */
