// Roofline probes of the field-line tracer (include/fqsl_probes.h): how fast
// this GPU serves trilinear gathers of 32-byte node records with a tracer
// warp's locality, and FP32 / FP64 fused multiply-add chains. They compute
// nothing of the method; the benchmark divides the tracer's algorithmic gather
// bytes and flops by these measured rates.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fqsl_probes.h"

namespace {

// 32-bit integer hash (Wellons' "lowbias32" mixer), for cheap random positions
__device__ __forceinline__ unsigned mix32(unsigned h)
{
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    h *= 0x846ca68bu;
    h ^= h >> 16;
    return h;
}

__device__ __forceinline__ float unit01(unsigned h) { return (float)(h >> 8) * (1.0f / 16777216.0f); }

// One 32-byte record in a single 256-bit read-only load, as the tracer loads it.
#pragma nv_diag_suppress 550
__device__ __forceinline__ void load_rec(const char *p, float v[6])
{
    float pad0, pad1;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(pad0), "=f"(pad1)
        : "l"(p));
}
#pragma nv_diag_default 550

// A random point of the tile origins' box and (walk) a random unit direction.
struct Walker {
    unsigned st;
    float ox, oy, oz, dx, dy, dz;
    __device__ __forceinline__ void restart(float hx, float hy, float hz)
    {
        st = mix32(st + 0x632be5abu);
        ox = unit01(st) * hx;
        st = mix32(st);
        oy = unit01(st) * hy;
        st = mix32(st);
        oz = unit01(st) * hz;
        st = mix32(st);
        float a = 2.f * unit01(st) - 1.f;
        st = mix32(st);
        float b = 2.f * unit01(st) - 1.f;
        st = mix32(st);
        float c = 2.f * unit01(st) - 1.f + 1e-3f;
        const float r = rsqrtf(a * a + b * b + c * c);
        dx = a * r;
        dy = b * r;
        dz = c * r;
    }
};

template <int P>
__global__ void __launch_bounds__(128) k_probe_gather(const char *__restrict__ rec, int nx, int ny, int nz,
                                                      int gathers, float *__restrict__ sink)
{
    const int lane = threadIdx.x & 31;
    const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
    // tile offsets of the lanes (8 x 4 points, 0.25 cells apart), and the box
    // the tile origin stays in so that every point lies in the cube
    const float lx = P == FQSL_PROBE_RANDOM ? 0.f : 0.25f * (float)(lane & 7);
    const float ly = P == FQSL_PROBE_RANDOM ? 0.f : 0.25f * (float)(lane >> 3);
    const float hx = (float)(nx - 1) - 2.f, hy = (float)(ny - 1) - 1.f, hz = (float)(nz - 1) - 0.01f;
    const size_t sy = (size_t)nx * 32u, sz = (size_t)nx * (size_t)ny * 32u;
    Walker w;
    w.st = mix32((P == FQSL_PROBE_RANDOM ? gid : (gid >> 5)) * 0x9e3779b9u + 1u);
    w.restart(hx, hy, hz);
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 2
    for (int g = 0; g < gathers; g++) {
        if (P == FQSL_PROBE_WALK) {
            w.ox += 0.4f * w.dx;
            w.oy += 0.4f * w.dy;
            w.oz += 0.4f * w.dz;
            if (!(w.ox >= 0.f && w.ox <= hx && w.oy >= 0.f && w.oy <= hy && w.oz >= 0.f && w.oz <= hz))
                w.restart(hx, hy, hz);
        } else {
            w.restart(hx, hy, hz);
        }
        const float px = w.ox + lx, py = w.oy + ly, pz = w.oz;
        const int cx = min((int)px, nx - 2), cy = min((int)py, ny - 2), cz = min((int)pz, nz - 2);
        const float wx = px - (float)cx, wy = py - (float)cy, wz = pz - (float)cz;
        const float ux = 1.f - wx, uy = 1.f - wy, uz = 1.f - wz;
        const char *p = rec + (size_t)cz * sz + (size_t)cy * sy + (size_t)cx * 32u;
#pragma unroll
        for (int c = 0; c < 4; c++) {
            const char *q = p + ((c & 1) ? sy : 0) + ((c & 2) ? sz : 0);
            const float wyz = ((c & 1) ? wy : uy) * ((c & 2) ? wz : uz);
            float a[6], b[6];
            load_rec(q, a);
            load_rec(q + 32, b);
#pragma unroll
            for (int k = 0; k < 6; k++) acc[k] += wyz * (ux * a[k] + wx * b[k]);
        }
    }
    sink[gid] = acc[0] + acc[1] + acc[2] + acc[3] + acc[4] + acc[5];
}

template <typename T>
__global__ void __launch_bounds__(256) k_probe_fma(int iters, T *__restrict__ sink)
{
    const unsigned gid = blockIdx.x * blockDim.x + threadIdx.x;
    const T a = (T)0.9999999, b = (T)1e-7;
    T x[8];
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (T)(gid & 1023) * (T)1e-4 + (T)k;
#pragma unroll 4
    for (int i = 0; i < iters; i++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    sink[gid] = s;
}

}  // namespace

extern "C" int fqsl_probe_gather(const void *rec_dev, int nx, int ny, int nz, int pattern, int gathers, int sms,
                                 int blocks_per_sm, float *sink_dev, void *cuda_stream)
{
    if (!rec_dev || !sink_dev || ((uintptr_t)rec_dev) % 32) return 1;
    if (nx < 4 || ny < 4 || nz < 4 || (long long)nx * ny * nz >= (1LL << 31)) return 1;
    if (gathers < 1 || sms < 1 || sms > 4096 || blocks_per_sm < 1 || blocks_per_sm > 64) return 1;
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const char *rec = (const char *)rec_dev;
    if (pattern == FQSL_PROBE_WALK)
        k_probe_gather<FQSL_PROBE_WALK><<<grid, 128, 0, s>>>(rec, nx, ny, nz, gathers, sink_dev);
    else if (pattern == FQSL_PROBE_TILE)
        k_probe_gather<FQSL_PROBE_TILE><<<grid, 128, 0, s>>>(rec, nx, ny, nz, gathers, sink_dev);
    else if (pattern == FQSL_PROBE_RANDOM)
        k_probe_gather<FQSL_PROBE_RANDOM><<<grid, 128, 0, s>>>(rec, nx, ny, nz, gathers, sink_dev);
    else
        return 1;
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}

extern "C" int fqsl_probe_fma(int fp64, int iters, int sms, int blocks_per_sm, void *sink_dev, void *cuda_stream)
{
    if (!sink_dev || iters < 1 || sms < 1 || sms > 4096 || blocks_per_sm < 1 || blocks_per_sm > 64) return 1;
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (fp64)
        k_probe_fma<double><<<grid, 256, 0, s>>>(iters, (double *)sink_dev);
    else
        k_probe_fma<float><<<grid, 256, 0, s>>>(iters, (float *)sink_dev);
    return cudaGetLastError() == cudaSuccess ? 0 : 2;
}
