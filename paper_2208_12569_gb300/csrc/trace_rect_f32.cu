// FP32 tracer instantiations for fields on stretched (rectilinear) grids
// (Sec. 2.2 and 2.3): the same persistent kernel as trace_f32.cu with the
// cell search, physical positions relative to the first node and per-cell
// step and error scaling of trace_body's RECT form (Method I, seed lists and
// Method II's deviation vectors), plus the FP32 seed pre-pass on such a grid.
#include "trace.cuh"

#ifndef FQSL_TRACE_F32_MINB
#define FQSL_TRACE_F32_MINB 4
#endif

namespace fqsl {
namespace {
constexpr int kBlock = 128;

template <int SRC, bool ACC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_trace_rect_f32(const TraceArgs A)
{
    trace::trace_body<float, SRC, ACC, 0, false, false, true>(A, BatchArgs{});
}

// Method II (deviation vectors) on a stretched grid
template <int WAY>
__global__ void __launch_bounds__(kBlock) k_trace_dev_rect_f32(const TraceArgs A)
{
    trace::trace_body<float, kSrcLattice, false, WAY, false, false, true>(A, BatchArgs{});
}

template <bool ACC>
void launch(const TraceArgs &a, int src, int grid, cudaStream_t s)
{
    if (src == kSrcLattice) k_trace_rect_f32<kSrcLattice, ACC><<<grid, kBlock, 0, s>>>(a);
    else if (src == kSrcExtra) k_trace_rect_f32<kSrcExtra, ACC><<<grid, kBlock, 0, s>>>(a);
    else k_trace_rect_f32<kSrcList, ACC><<<grid, kBlock, 0, s>>>(a);
}

template <bool ACC>
int blocks(int src)
{
    int b = 0;
    if (src == kSrcLattice)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_f32<kSrcLattice, ACC>, kBlock, 0);
    else if (src == kSrcExtra)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_f32<kSrcExtra, ACC>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_f32<kSrcList, ACC>, kBlock, 0);
    return b > 0 ? b : 1;
}

// the adjoint's forward pass: lattice or extra lines writing the step tape
template <int SRC, bool ACC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_trace_tape_rect_f32(const TraceArgs A)
{
    trace::trace_body<float, SRC, ACC, 0, false, true, true>(A, BatchArgs{});
}

__global__ void __launch_bounds__(256) k_seed_prep_rect_f32(const TraceArgs A, long long n)
{
    for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < n;
         idx += (long long)gridDim.x * blockDim.x)
        trace::seed_prep_f32<true>(A, idx);
}
}  // namespace

cudaError_t launch_trace_rect_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64)
{
    if (acc64) launch<true>(a, src, grid, s);
    else launch<false>(a, src, grid, s);
    return cudaGetLastError();
}

int trace_rect_blocks_per_sm_f32(int src, bool acc64) { return acc64 ? blocks<true>(src) : blocks<false>(src); }

cudaError_t launch_trace_dev_rect_f32(const TraceArgs &a, int way, int grid, cudaStream_t s)
{
    if (way == 1) k_trace_dev_rect_f32<1><<<grid, kBlock, 0, s>>>(a);
    else k_trace_dev_rect_f32<2><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_dev_rect_blocks_per_sm_f32(int way)
{
    int b = 0;
    if (way == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_f32<1>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_f32<2>, kBlock, 0);
    return b > 0 ? b : 1;
}

cudaError_t launch_trace_tape_rect_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64)
{
    if (src == kSrcExtra) {
        if (acc64) k_trace_tape_rect_f32<kSrcExtra, true><<<grid, kBlock, 0, s>>>(a);
        else k_trace_tape_rect_f32<kSrcExtra, false><<<grid, kBlock, 0, s>>>(a);
    } else {
        if (acc64) k_trace_tape_rect_f32<kSrcLattice, true><<<grid, kBlock, 0, s>>>(a);
        else k_trace_tape_rect_f32<kSrcLattice, false><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int trace_tape_rect_blocks_per_sm_f32(int src, bool acc64)
{
    int b = 0;
    if (src == kSrcExtra) {
        if (acc64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_f32<kSrcExtra, true>, kBlock, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_f32<kSrcExtra, false>, kBlock, 0);
    } else {
        if (acc64) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_f32<kSrcLattice, true>, kBlock, 0);
        else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_f32<kSrcLattice, false>, kBlock, 0);
    }
    return b > 0 ? b : 1;
}

cudaError_t launch_seed_prep_rect_f32(const TraceArgs &a, long long n, unsigned grid, cudaStream_t s)
{
    k_seed_prep_rect_f32<<<grid, 256, 0, s>>>(a, n);
    return cudaGetLastError();
}

}  // namespace fqsl
