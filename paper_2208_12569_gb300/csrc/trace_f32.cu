// FP32 instantiations of the persistent tracer: the cube and the line state
// are in float. ACC = false (precision FQSL_F32): error norm in float, length
// and Tw as compensated float sums formed in double per direction. ACC = true
// (FQSL_F32_ACC64): error norm and length/Tw sums accumulated in double. The
// per-line tolerance, footpoints and Bn are double in both.
#include "trace.cuh"

// minimum resident blocks per SM requested from the register allocator
#ifndef FQSL_TRACE_F32_MINB
#define FQSL_TRACE_F32_MINB 4
#endif

namespace fqsl {
namespace {
constexpr int kBlock = 128;

template <int SRC, bool ACC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_trace_f32(const TraceArgs A)
{
    trace::trace_body<float, SRC, ACC>(A, BatchArgs{});
}
}  // namespace

namespace {
template <bool ACC>
void launch(const TraceArgs &a, int src, int grid, int block, cudaStream_t s)
{
    if (src == kSrcLattice) k_trace_f32<kSrcLattice, ACC><<<grid, block, 0, s>>>(a);
    else if (src == kSrcExtra) k_trace_f32<kSrcExtra, ACC><<<grid, block, 0, s>>>(a);
    else k_trace_f32<kSrcList, ACC><<<grid, block, 0, s>>>(a);
}

template <bool ACC>
int blocks(int src)
{
    int b = 0;
    if (src == kSrcLattice)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f32<kSrcLattice, ACC>, kBlock, 0);
    else if (src == kSrcExtra)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f32<kSrcExtra, ACC>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f32<kSrcList, ACC>, kBlock, 0);
    return b > 0 ? b : 1;
}
}  // namespace

cudaError_t launch_trace_f32(const TraceArgs &a, int src, int grid, int block, cudaStream_t s, bool acc64)
{
    if (block != kBlock) return cudaErrorInvalidValue;
    if (a.p.scheme == 1)
        return a.f.rect ? launch_trace_rect_rk38_f32(a, src, grid, s, acc64) : launch_trace_rk38_f32(a, src, grid, s, acc64);
    if (a.f.rect) return launch_trace_rect_f32(a, src, grid, s, acc64);
    if (acc64) launch<true>(a, src, grid, block, s);
    else launch<false>(a, src, grid, block, s);
    return cudaGetLastError();
}

int trace_blocks_per_sm_f32(int src, bool acc64) { return acc64 ? blocks<true>(src) : blocks<false>(src); }

}  // namespace fqsl

namespace fqsl {
namespace {
__global__ void __launch_bounds__(256) k_seed_prep_f32(const TraceArgs A, long long n)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x)
        trace::seed_prep_f32(A, idx);
}
}  // namespace

cudaError_t launch_seed_prep_f32(const TraceArgs &a, long long n, cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (n + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    if (a.f.rect) return launch_seed_prep_rect_f32(a, n, (unsigned)blocks, s);
    k_seed_prep_f32<<<(unsigned)blocks, 256, 0, s>>>(a, n);
    return cudaGetLastError();
}

}  // namespace fqsl

namespace fqsl {
namespace {
template <int WAY>
__global__ void __launch_bounds__(kBlock) k_trace_dev_f32(const TraceArgs A)
{
    trace::trace_body<float, kSrcLattice, false, WAY>(A, BatchArgs{});
}
}  // namespace

cudaError_t launch_trace_dev_f32(const TraceArgs &a, int way, int grid, int block, cudaStream_t s)
{
    if (block != kBlock) return cudaErrorInvalidValue;
    if (a.p.scheme == 1)
        return a.f.rect ? launch_trace_dev_rect_rk38_f32(a, way, grid, s) : launch_trace_dev_rk38_f32(a, way, grid, s);
    if (a.f.rect) return launch_trace_dev_rect_f32(a, way, grid, s);
    if (way == 1) k_trace_dev_f32<1><<<grid, block, 0, s>>>(a);
    else k_trace_dev_f32<2><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_dev_blocks_per_sm_f32(int way)
{
    int b = 0;
    if (way == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_f32<1>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_f32<2>, kBlock, 0);
    return b > 0 ? b : 1;
}
}  // namespace fqsl

// ---------------------------------------------------------------------------
// batches: many (field, plane) entries in one launch
// ---------------------------------------------------------------------------
namespace fqsl {
namespace {
template <int SRC, bool ACC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_batch_trace_f32(const TraceArgs A0, const BatchArgs B)
{
    trace::trace_body<float, SRC, ACC, 0, true>(A0, B);
}

__global__ void __launch_bounds__(256) k_batch_seed_prep_f32(const TraceArgs *__restrict__ desc,
                                                             const long long *__restrict__ nbase, int nent)
{
    const long long total = nbase[nent];
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < total;
         idx += (long long)gridDim.x * blockDim.x) {
        int lo = 0, hi = nent - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (nbase[mid] <= idx) lo = mid;
            else hi = mid - 1;
        }
        trace::seed_prep_f32(desc[lo], idx - nbase[lo]);
    }
}

// work-item prefix of the rotated extra lines: 4 per rotated seed, padded to
// whole 32-item chunks per entry
__global__ void k_batch_extra_prefix(const unsigned *__restrict__ rot_counts, int nent, long long *xbase)
{
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    long long acc = 0;
    for (int b = 0; b < nent; b++) {
        xbase[b] = acc;
        acc += (4LL * rot_counts[b] + 31) / 32 * 32;
    }
    xbase[nent] = acc;
}
}  // namespace

cudaError_t launch_batch_seed_prep_f32(const TraceArgs *desc, const long long *nbase, int nent, long long total,
                                       cudaStream_t s)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    long long blocks = (total + 255) / 256;
    if (blocks > (long long)sms * 8) blocks = (long long)sms * 8;
    if (blocks < 1) blocks = 1;
    k_batch_seed_prep_f32<<<(unsigned)blocks, 256, 0, s>>>(desc, nbase, nent);
    return cudaGetLastError();
}

cudaError_t launch_batch_extra_prefix(const unsigned *rot_counts, int nent, long long *xbase, cudaStream_t s)
{
    k_batch_extra_prefix<<<1, 32, 0, s>>>(rot_counts, nent, xbase);
    return cudaGetLastError();
}

cudaError_t launch_batch_trace_f32(const TraceArgs &a0, const BatchArgs &b, int src, bool acc64, int grid,
                                   cudaStream_t s)
{
    if (a0.p.scheme == 1) return launch_batch_trace_rk38_f32(a0, b, src, acc64, grid, s);
    if (src == kSrcLattice) {
        if (acc64) k_batch_trace_f32<kSrcLattice, true><<<grid, kBlock, 0, s>>>(a0, b);
        else k_batch_trace_f32<kSrcLattice, false><<<grid, kBlock, 0, s>>>(a0, b);
    } else {
        if (acc64) k_batch_trace_f32<kSrcExtra, true><<<grid, kBlock, 0, s>>>(a0, b);
        else k_batch_trace_f32<kSrcExtra, false><<<grid, kBlock, 0, s>>>(a0, b);
    }
    return cudaGetLastError();
}

int batch_trace_blocks_per_sm_f32(bool acc64, int scheme)
{
    if (scheme == 1) return batch_trace_rk38_blocks_per_sm_f32(acc64);
    int b = 0;
    if (acc64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_trace_f32<kSrcLattice, true>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_trace_f32<kSrcLattice, false>, kBlock, 0);
    return b > 0 ? b : 1;
}
}  // namespace fqsl

// ---------------------------------------------------------------------------
// adjoint forward pass: the lattice tracer that also writes the step tape
// ---------------------------------------------------------------------------
namespace fqsl {
namespace {
template <int SRC, bool ACC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_trace_tape_f32(const TraceArgs A)
{
    trace::trace_body<float, SRC, ACC, 0, false, true>(A, BatchArgs{});
}
}  // namespace

cudaError_t launch_trace_tape_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64)
{
    if (src == kSrcExtra) {
        if (acc64) k_trace_tape_f32<kSrcExtra, true><<<grid, kBlock, 0, s>>>(a);
        else k_trace_tape_f32<kSrcExtra, false><<<grid, kBlock, 0, s>>>(a);
    } else {
        if (acc64) k_trace_tape_f32<kSrcLattice, true><<<grid, kBlock, 0, s>>>(a);
        else k_trace_tape_f32<kSrcLattice, false><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int trace_tape_blocks_per_sm_f32(int src, bool acc64)
{
    int b = 0;
    if (src == kSrcExtra) {
        if (acc64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_f32<kSrcExtra, true>, kBlock, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_f32<kSrcExtra, false>, kBlock, 0);
    } else {
        if (acc64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_f32<kSrcLattice, true>, kBlock, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_f32<kSrcLattice, false>, kBlock, 0);
    }
    return b > 0 ? b : 1;
}
}  // namespace fqsl
