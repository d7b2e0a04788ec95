// Reverse sweep of a taped map traced with the fixed-step scheme (Sec. 2.3:
// Kutta's 3/8-rule RK4, the per-line step of Sec. 4 Eq. step): the passes of
// adjoint.cu with the four-stage step, in a translation unit of their own.
#include "adjoint.cuh"

namespace fqsl {
namespace {
template <typename TT>
void reverse_mode(const AdjArgs &a, int mode, cudaStream_t s)
{
    if (mode == 0) adj::reverse_passes<float, float, TT, 1>(a, s);
    else if (mode == 1) adj::reverse_passes<float, double, TT, 1>(a, s);
    else adj::reverse_passes<double, double, TT, 1>(a, s);
}
}  // namespace

cudaError_t launch_reverse_rk38(const AdjArgs &a, int mode, bool tape_f64, cudaStream_t s)
{
    if (tape_f64) reverse_mode<double>(a, mode, s);
    else reverse_mode<float>(a, mode, s);
    return cudaGetLastError();
}

}  // namespace fqsl
