// binary32 <-> binary64 conversions and a binary64 reciprocal that keep work
// off the FP64 pipe (shared by the viscous/RK kernel and the diagnostics).
#pragma once

#include <cuda_runtime.h>

namespace nopcs {

// Conversions between binary32 and binary64 by integer operations on the
// IEEE 754 bit patterns, for the FP64 arithmetic of the mixed form, whose
// conversions would otherwise load the FP64 pipe (GB300 runs it at 1/64 of the
// FP32 rate).  Normal numbers only; zero, subnormals, infinities and NaN take
// the hardware conversion, which gives the same result.
//   widen: sign kept, exponent re-biased by 1023 - 127, the 23 fraction bits
//          moved to the top of the 52 (exact);
//   narrow: exponent re-biased by 127 - 1023 where the result is a normal
//          binary32, fraction cut to 23 bits and rounded to nearest, ties to
//          even, from the 29 bits cut off; a carry out of the fraction moves
//          into the exponent (up to infinity), as rounding does.
__device__ __forceinline__ double widen_f32(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e - 1u < 0xfeu) {
        const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u >> 3) & 0xfffffu);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    return (double)f;
}
__device__ __forceinline__ float narrow_f64(double d)
{
    const unsigned hi = (unsigned)__double2hiint(d), lo = (unsigned)__double2loint(d);
    const unsigned e = (hi >> 20) & 0x7ffu;
    if (e - 897u < 254u) {
        unsigned r = ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;
        r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
        return __uint_as_float(r | (hi & 0x80000000u));
    }
    return (float)d;
}


// Reciprocal of a binary64 value by the Newton-Raphson iteration for 1/a,
// y <- y + y (1 - a y), each step about doubling the correct bits: the seed is
// the approximate binary32 reciprocal of a rounded to binary32 (about 22
// correct bits), two steps in binary64 arithmetic reach its precision (within
// an ulp of 1/a, not always the correctly rounded value).  Four FMAs instead of
// a binary64 division.  Where a or its reciprocal is not a normal binary32
// (zero, tiny, huge, infinite, NaN) the division is used.
__device__ __forceinline__ double recip_newton(double a)
{
    const float af = narrow_f64(a);
    const unsigned e = (__float_as_uint(af) >> 23) & 0xffu;
    if (e - 2u >= 0xfcu) return 1.0 / a;
    double y = widen_f32(__fdividef(1.0f, af));
    y = __fma_rn(y, __fma_rn(-a, y, 1.0), y);
    y = __fma_rn(y, __fma_rn(-a, y, 1.0), y);
    return y;
}

}  // namespace nopcs
