// FP32 instantiation of the persistent tracer: the cube and the line state are
// in float; the error norm, the per-line tolerance and the Tw / length sums
// are in double.
#include "trace.cuh"

// minimum resident blocks per SM requested from the register allocator
#ifndef FQSL_TRACE_F32_MINB
#define FQSL_TRACE_F32_MINB 4
#endif

namespace fqsl {
namespace {
constexpr int kBlock = 128;

template <int SRC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_trace_f32(const TraceArgs A)
{
    trace::trace_body<float, SRC>(A);
}
}  // namespace

cudaError_t launch_trace_f32(const TraceArgs &a, int src, int grid, int block, cudaStream_t s)
{
    if (block != kBlock) return cudaErrorInvalidValue;
    if (src == kSrcLattice) k_trace_f32<kSrcLattice><<<grid, block, 0, s>>>(a);
    else if (src == kSrcExtra) k_trace_f32<kSrcExtra><<<grid, block, 0, s>>>(a);
    else k_trace_f32<kSrcList><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_blocks_per_sm_f32(int src)
{
    int b = 0;
    if (src == kSrcLattice) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f32<kSrcLattice>, kBlock, 0);
    else if (src == kSrcExtra) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f32<kSrcExtra>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f32<kSrcList>, kBlock, 0);
    return b > 0 ? b : 1;
}

}  // namespace fqsl
