// FP64 tracer instantiations for fields on stretched (rectilinear) grids
// (Sec. 2.2 and 2.3): physical positions, the cell search, Eq. w0 weights as
// written and per-cell step and error scaling (trace_body's RECT form). Built
// without contraction like trace_f64.cu, so that it reproduces a plain
// evaluation of the method to the last bit.
#include "trace.cuh"

namespace fqsl {
namespace {
constexpr int kBlock = 128;

template <int SRC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F64_MINB) k_trace_rect_f64(const TraceArgs A)
{
    trace::trace_body<double, SRC, true, 0, false, false, true>(A, BatchArgs{});
}
// Method II (deviation vectors) on a stretched grid
template <int WAY>
__global__ void __launch_bounds__(kBlock) k_trace_dev_rect_f64(const TraceArgs A)
{
    trace::trace_body<double, kSrcLattice, true, WAY, false, false, true>(A, BatchArgs{});
}

// the adjoint's forward pass: lattice or extra lines writing the step tape
template <int SRC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F64_MINB) k_trace_tape_rect_f64(const TraceArgs A)
{
    trace::trace_body<double, SRC, true, 0, false, true, true>(A, BatchArgs{});
}
}  // namespace

cudaError_t launch_trace_tape_rect_f64(const TraceArgs &a, int src, int grid, cudaStream_t s)
{
    if (src == kSrcExtra) k_trace_tape_rect_f64<kSrcExtra><<<grid, kBlock, 0, s>>>(a);
    else k_trace_tape_rect_f64<kSrcLattice><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_tape_rect_blocks_per_sm_f64(int src)
{
    int b = 0;
    if (src == kSrcExtra) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_f64<kSrcExtra>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_f64<kSrcLattice>, kBlock, 0);
    return b > 0 ? b : 1;
}

cudaError_t launch_trace_dev_rect_f64(const TraceArgs &a, int way, int grid, cudaStream_t s)
{
    if (way == 1) k_trace_dev_rect_f64<1><<<grid, kBlock, 0, s>>>(a);
    else k_trace_dev_rect_f64<2><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_dev_rect_blocks_per_sm_f64(int way)
{
    int b = 0;
    if (way == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_f64<1>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_f64<2>, kBlock, 0);
    return b > 0 ? b : 1;
}

cudaError_t launch_trace_rect_f64(const TraceArgs &a, int src, int grid, cudaStream_t s)
{
    if (src == kSrcLattice) k_trace_rect_f64<kSrcLattice><<<grid, kBlock, 0, s>>>(a);
    else if (src == kSrcExtra) k_trace_rect_f64<kSrcExtra><<<grid, kBlock, 0, s>>>(a);
    else k_trace_rect_f64<kSrcList><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_rect_blocks_per_sm_f64(int src)
{
    int b = 0;
    if (src == kSrcLattice)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_f64<kSrcLattice>, kBlock, 0);
    else if (src == kSrcExtra)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_f64<kSrcExtra>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_f64<kSrcList>, kBlock, 0);
    return b > 0 ? b : 1;
}

}  // namespace fqsl
