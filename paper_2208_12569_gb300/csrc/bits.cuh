// Exact float <-> double moves by bit manipulation on the integer pipe. On
// GB300 the conversion instructions between float and double run on the
// narrow FP64 pipe; these helpers give the same values without it.
#pragma once

#include <stdint.h>
#include <string.h>

namespace fqsl {
namespace bits {

// The float equal to d, for a double d that holds a float value (every float
// is exactly a double, e.g. one widened by the tracers' f2d): the sign, the
// exponent rebased from 1023 to 127, and the top 23 of the 52 mantissa bits
// (the other 29 are zero). Doubles below the smallest normal float hold a
// float subnormal, whose significand is shifted right instead. The result is
// meaningless for a double that is not a float value.
__host__ __device__ inline float narrow_exact(double d)
{
    uint64_t b;
#ifdef __CUDA_ARCH__
    b = (uint64_t)__double_as_longlong(d);
#else
    memcpy(&b, &d, sizeof b);
#endif
    const uint32_t sign = (uint32_t)(b >> 32) & 0x80000000u;
    const uint32_t e = (uint32_t)(b >> 52) & 0x7ffu;
    const uint32_t m = (uint32_t)(b >> 29) & 0x7fffffu;
    uint32_t f;
    if (e == 0x7ffu) f = sign | 0x7f800000u | m | (m == 0u && (b & 0xfffffffffffffull) ? 1u : 0u);  // inf, NaN
    else if (e >= 897u) f = sign | ((e - 896u) << 23) | m;  // normal float: 2^-126 <= |d|
    else if (e > 873u) f = sign | ((0x800000u | m) >> (897u - e));  // float subnormal: shift 1 .. 23
    else f = sign;  // zero
    float r;
#ifdef __CUDA_ARCH__
    r = __uint_as_float(f);
#else
    memcpy(&r, &f, sizeof r);
#endif
    return r;
}

}  // namespace bits
}  // namespace fqsl
