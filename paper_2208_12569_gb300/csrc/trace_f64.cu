// FP64 instantiation of the persistent tracer: the cube, the line state and all
// arithmetic are in double (the parity reference of the float tracer).
#include "trace.cuh"

namespace fqsl {
namespace {
constexpr int kBlock = 128;

template <int SRC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F64_MINB) k_trace_f64(const TraceArgs A)
{
    trace::trace_body<double, SRC, true>(A, BatchArgs{});
}
}  // namespace

cudaError_t launch_trace_f64(const TraceArgs &a, int src, int grid, int block, cudaStream_t s)
{
    if (block != kBlock) return cudaErrorInvalidValue;
    if (a.p.scheme == 1)
        return a.f.rect ? launch_trace_rect_rk38_f64(a, src, grid, s) : launch_trace_rk38_f64(a, src, grid, s);
    if (a.f.rect) return launch_trace_rect_f64(a, src, grid, s);
    if (src == kSrcLattice) k_trace_f64<kSrcLattice><<<grid, block, 0, s>>>(a);
    else if (src == kSrcExtra) k_trace_f64<kSrcExtra><<<grid, block, 0, s>>>(a);
    else k_trace_f64<kSrcList><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_blocks_per_sm_f64(int src)
{
    int b = 0;
    if (src == kSrcLattice) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f64<kSrcLattice>, kBlock, 0);
    else if (src == kSrcExtra) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f64<kSrcExtra>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_f64<kSrcList>, kBlock, 0);
    return b > 0 ? b : 1;
}

}  // namespace fqsl

namespace fqsl {
namespace {
template <int WAY>
__global__ void __launch_bounds__(kBlock) k_trace_dev_f64(const TraceArgs A)
{
    trace::trace_body<double, kSrcLattice, true, WAY>(A, BatchArgs{});
}
}  // namespace

cudaError_t launch_trace_dev_f64(const TraceArgs &a, int way, int grid, int block, cudaStream_t s)
{
    if (block != kBlock) return cudaErrorInvalidValue;
    if (a.p.scheme == 1)
        return a.f.rect ? launch_trace_dev_rect_rk38_f64(a, way, grid, s) : launch_trace_dev_rk38_f64(a, way, grid, s);
    if (a.f.rect) return launch_trace_dev_rect_f64(a, way, grid, s);
    if (way == 1) k_trace_dev_f64<1><<<grid, block, 0, s>>>(a);
    else k_trace_dev_f64<2><<<grid, block, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_dev_blocks_per_sm_f64(int way)
{
    int b = 0;
    if (way == 1) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_f64<1>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_dev_f64<2>, kBlock, 0);
    return b > 0 ? b : 1;
}
}  // namespace fqsl

namespace fqsl {
namespace {
template <int SRC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F64_MINB) k_batch_trace_f64(const TraceArgs A0, const BatchArgs B)
{
    trace::trace_body<double, SRC, true, 0, true>(A0, B);
}
}  // namespace

cudaError_t launch_batch_trace_f64(const TraceArgs &a0, const BatchArgs &b, int src, int grid, cudaStream_t s)
{
    if (a0.p.scheme == 1) return launch_batch_trace_rk38_f64(a0, b, src, grid, s);
    if (src == kSrcLattice) k_batch_trace_f64<kSrcLattice><<<grid, kBlock, 0, s>>>(a0, b);
    else k_batch_trace_f64<kSrcExtra><<<grid, kBlock, 0, s>>>(a0, b);
    return cudaGetLastError();
}

int batch_trace_blocks_per_sm_f64(int scheme)
{
    if (scheme == 1) return batch_trace_rk38_blocks_per_sm_f64();
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_batch_trace_f64<kSrcLattice>, kBlock, 0);
    return b > 0 ? b : 1;
}
}  // namespace fqsl

namespace fqsl {
namespace {
// adjoint forward pass: the tracers that also write the step tape
template <int SRC>
__global__ void __launch_bounds__(kBlock, FQSL_TRACE_F64_MINB) k_trace_tape_f64(const TraceArgs A)
{
    trace::trace_body<double, SRC, true, 0, false, true>(A, BatchArgs{});
}
}  // namespace

cudaError_t launch_trace_tape_f64(const TraceArgs &a, int src, int grid, cudaStream_t s)
{
    if (src == kSrcExtra) k_trace_tape_f64<kSrcExtra><<<grid, kBlock, 0, s>>>(a);
    else k_trace_tape_f64<kSrcLattice><<<grid, kBlock, 0, s>>>(a);
    return cudaGetLastError();
}

int trace_tape_blocks_per_sm_f64(int src)
{
    int b = 0;
    if (src == kSrcExtra) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_f64<kSrcExtra>, kBlock, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_trace_tape_f64<kSrcLattice>, kBlock, 0);
    return b > 0 ? b : 1;
}
}  // namespace fqsl
