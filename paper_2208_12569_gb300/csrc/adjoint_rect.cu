// Reverse sweep of a taped map on a stretched grid (Sec. 2.2-2.3: the
// cell search, Eq. w0 weights in physical coordinates, each step scaled by the
// widths of the cell it starts in): the passes of adjoint.cu in their RECT
// form, for RKF45 and the fixed-step 3/8 rule, in a translation unit of their
// own. The tape and the sweep share their
// state precision (FP64 physical positions, or FP32 positions relative to the
// first node).
#include "adjoint.cuh"

namespace fqsl {

namespace {
template <int SCH>
void rect_mode(const AdjArgs &a, int mode, cudaStream_t s)
{
    if (mode == 0) adj::reverse_passes<float, float, float, SCH, true>(a, s);
    else if (mode == 1) adj::reverse_passes<float, double, float, SCH, true>(a, s);
    else adj::reverse_passes<double, double, double, SCH, true>(a, s);
}
}  // namespace

cudaError_t launch_reverse_rect(const AdjArgs &a, int mode, cudaStream_t s)
{
    if (a.p.scheme == 1) rect_mode<1>(a, mode, s);
    else rect_mode<0>(a, mode, s);
    return cudaGetLastError();
}

}  // namespace fqsl
