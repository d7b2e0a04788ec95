// Reverse sweep of a taped RKF45 map on a stretched grid (Sec. 2.2-2.3: the
// cell search, Eq. w0 weights in physical coordinates, each step scaled by the
// widths of the cell it starts in): the passes of adjoint.cu in their RECT
// form, in a translation unit of their own. The tape and the sweep share their
// state precision (FP64 physical positions, or FP32 positions relative to the
// first node).
#include "adjoint.cuh"

namespace fqsl {

cudaError_t launch_reverse_rect(const AdjArgs &a, int mode, cudaStream_t s)
{
    if (mode == 0) adj::reverse_passes<float, float, float, 0, true>(a, s);
    else if (mode == 1) adj::reverse_passes<float, double, float, 0, true>(a, s);
    else adj::reverse_passes<double, double, double, 0, true>(a, s);
    return cudaGetLastError();
}

}  // namespace fqsl
