// FP64 tracer instantiations for the fixed-step scheme (3/8-rule RK4, Sec.
// 2.3; Eq. step) on stretched grids (Sec. 2.2-2.3). Built without
// contraction like trace_f64.cu, so that it reproduces a plain evaluation of
// the method to the last bit.
#include "trace.cuh"

namespace fqsl {
namespace {
constexpr int kBlock = 128;

template <int SRC>
__global__ void __launch_bounds__(kBlock) k_trace_rect_rk38_f64(const TraceArgs A)
{
    trace::trace_body<double, SRC, true, 0, false, false, true, 1>(A, BatchArgs{});
}

template <int WAY>
__global__ void __launch_bounds__(kBlock) k_trace_dev_rect_rk38_f64(const TraceArgs A)
{
    trace::trace_body<double, kSrcLattice, true, WAY, false, false, true, 1>(A, BatchArgs{});
}

// the adjoint's forward pass: lattice or extra lines writing the step tape
template <int SRC>
__global__ void __launch_bounds__(kBlock) k_trace_tape_rect_rk38_f64(const TraceArgs A)
{
    trace::trace_body<double, SRC, true, 0, false, true, true, 1>(A, BatchArgs{});
}
}  // namespace

cudaError_t launch_trace_tape_rect_rk38_f64(const TraceArgs &a, int src, int grid, cudaStream_t s)
{
    if (src == kSrcExtra) k_trace_tape_rect_rk38_f64<kSrcExtra><<<grid, kBlock, 0, s>>>(a);
    else k_trace_tape_rect_rk38_f64<kSrcLattice><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_tape_rect_rk38_blocks_per_sm_f64(int src)
{
    int b = 0;
    if (src == kSrcExtra)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_rk38_f64<kSrcExtra>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_rk38_f64<kSrcLattice>, kBlock, 0);
    return b > 0 ? b : 1;
}

cudaError_t launch_trace_rect_rk38_f64(const TraceArgs &a, int src, int grid, cudaStream_t s)
{
    if (src == kSrcLattice) k_trace_rect_rk38_f64<kSrcLattice><<<grid, kBlock, 0, s>>>(a);
    else if (src == kSrcExtra) k_trace_rect_rk38_f64<kSrcExtra><<<grid, kBlock, 0, s>>>(a);
    else k_trace_rect_rk38_f64<kSrcList><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_rect_rk38_blocks_per_sm_f64(int src)
{
    int b = 0;
    if (src == kSrcLattice)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_rk38_f64<kSrcLattice>, kBlock, 0);
    else if (src == kSrcExtra)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_rk38_f64<kSrcExtra>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_rk38_f64<kSrcList>, kBlock, 0);
    return b > 0 ? b : 1;
}

cudaError_t launch_trace_dev_rect_rk38_f64(const TraceArgs &a, int way, int grid, cudaStream_t s)
{
    if (way == 1) k_trace_dev_rect_rk38_f64<1><<<grid, kBlock, 0, s>>>(a);
    else k_trace_dev_rect_rk38_f64<2><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_dev_rect_rk38_blocks_per_sm_f64(int way)
{
    int b = 0;
    if (way == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_rk38_f64<1>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_rk38_f64<2>, kBlock, 0);
    return b > 0 ? b : 1;
}

}  // namespace fqsl
