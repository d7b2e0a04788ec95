// FP32 tracer instantiations for the fixed-step scheme (3/8-rule RK4, Sec.
// 2.3; Eq. step) on stretched grids (Sec. 2.2-2.3): trace_body with both the
// RECT and the SCH forms. Method I sources and Method II's two ways.
#include "trace.cuh"

#ifndef FQSL_TRACE_F32_MINB
#define FQSL_TRACE_F32_MINB 4
#endif

namespace fqsl {
namespace {
constexpr int kBlock = 128;

template <int SRC, bool ACC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_trace_rect_rk38_f32(const TraceArgs A)
{
    trace::trace_body<float, SRC, ACC, 0, false, false, true, 1>(A, BatchArgs{});
}

template <int WAY>
__global__ void __launch_bounds__(kBlock) k_trace_dev_rect_rk38_f32(const TraceArgs A)
{
    trace::trace_body<float, kSrcLattice, false, WAY, false, false, true, 1>(A, BatchArgs{});
}

// the adjoint's forward pass: lattice or extra lines writing the step tape
template <int SRC, bool ACC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F32_MINB) k_trace_tape_rect_rk38_f32(const TraceArgs A)
{
    trace::trace_body<float, SRC, ACC, 0, false, true, true, 1>(A, BatchArgs{});
}

template <bool ACC>
void launch(const TraceArgs &a, int src, int grid, cudaStream_t s)
{
    if (src == kSrcLattice) k_trace_rect_rk38_f32<kSrcLattice, ACC><<<grid, kBlock, 0, s>>>(a);
    else if (src == kSrcExtra) k_trace_rect_rk38_f32<kSrcExtra, ACC><<<grid, kBlock, 0, s>>>(a);
    else k_trace_rect_rk38_f32<kSrcList, ACC><<<grid, kBlock, 0, s>>>(a);
}

template <bool ACC>
int blocks(int src)
{
    int b = 0;
    if (src == kSrcLattice)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_rk38_f32<kSrcLattice, ACC>, kBlock, 0);
    else if (src == kSrcExtra)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_rk38_f32<kSrcExtra, ACC>, kBlock, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_rect_rk38_f32<kSrcList, ACC>, kBlock, 0);
    return b > 0 ? b : 1;
}
}  // namespace

cudaError_t launch_trace_rect_rk38_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64)
{
    if (acc64) launch<true>(a, src, grid, s);
    else launch<false>(a, src, grid, s);
    return cudaGetLastError();
}

int trace_rect_rk38_blocks_per_sm_f32(int src, bool acc64) { return acc64 ? blocks<true>(src) : blocks<false>(src); }

cudaError_t launch_trace_tape_rect_rk38_f32(const TraceArgs &a, int src, int grid, cudaStream_t s, bool acc64)
{
    if (src == kSrcExtra) {
        if (acc64) k_trace_tape_rect_rk38_f32<kSrcExtra, true><<<grid, kBlock, 0, s>>>(a);
        else k_trace_tape_rect_rk38_f32<kSrcExtra, false><<<grid, kBlock, 0, s>>>(a);
    } else {
        if (acc64) k_trace_tape_rect_rk38_f32<kSrcLattice, true><<<grid, kBlock, 0, s>>>(a);
        else k_trace_tape_rect_rk38_f32<kSrcLattice, false><<<grid, kBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

int trace_tape_rect_rk38_blocks_per_sm_f32(int src, bool acc64)
{
    int b = 0;
    if (src == kSrcExtra) {
        if (acc64)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_rk38_f32<kSrcExtra, true>, kBlock, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_rk38_f32<kSrcExtra, false>, kBlock, 0);
    } else {
        if (acc64)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_rk38_f32<kSrcLattice, true>, kBlock, 0);
        else
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_rect_rk38_f32<kSrcLattice, false>, kBlock,
                                                          0);
    }
    return b > 0 ? b : 1;
}

cudaError_t launch_trace_dev_rect_rk38_f32(const TraceArgs &a, int way, int grid, cudaStream_t s)
{
    if (way == 1) k_trace_dev_rect_rk38_f32<1><<<grid, kBlock, 0, s>>>(a);
    else k_trace_dev_rect_rk38_f32<2><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_dev_rect_rk38_blocks_per_sm_f32(int way)
{
    int b = 0;
    if (way == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_rk38_f32<1>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_rect_rk38_f32<2>, kBlock, 0);
    return b > 0 ? b : 1;
}

}  // namespace fqsl
