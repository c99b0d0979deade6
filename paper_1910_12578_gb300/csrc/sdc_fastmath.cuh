// sdc_fastmath.cuh -- FP64 helpers that keep work off GB300's narrow FP64 pipe.
//
// GB300 issues FP64 arithmetic at 1/61 of its FP32 rate, so the hot kernels
// count FP64 instructions.  Two classical devices are used:
//  * reciprocal and reciprocal square root by Newton-Raphson iteration
//    (y <- y (2 - x y) and y <- y (3 - x y^2) / 2, quadratic convergence) from
//    the hardware approximations of PTX rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64
//    (a few correct bits, issued outside the FP64 FMA pipe); two steps give a
//    result within a few ulp of the correctly rounded value;
//  * exact operations on IEEE-754 bit patterns done on the integer pipe: |x|,
//    sign tests, x2 and x1/2 by exponent increment/decrement (exact for normal
//    numbers), and min of non-negative doubles (their bit patterns order like
//    the values).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace sdcd {

__device__ __forceinline__ double rcp_seed(double x) {
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

__device__ __forceinline__ double rsqrt_seed(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    return y;
}

// 1/x for finite, normal, nonzero x (Newton-Raphson, 2 steps)
__device__ __forceinline__ double rcp_nr(double x) {
    double y = rcp_seed(x);
    double e = fma(-x, y, 1.0);
    y = fma(y, e, y);
    e = fma(-x, y, 1.0);
    return fma(y, e, y);
}

// sqrt(x) for finite, positive, normal x: x * rsqrt(x) with rsqrt refined by
// two Newton-Raphson steps
__device__ __forceinline__ double sqrt_nr(double x) {
    double y = rsqrt_seed(x);
    double h = 0.5 * y;
    double e = fma(-x * y, y, 1.0);
    y = fma(h, e, y);
    h = 0.5 * y;
    e = fma(-x * y, y, 1.0);
    y = fma(h, e, y);
    return x * y;
}

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd(long long b) { return __longlong_as_double(b); }

constexpr long long SIGN_BIT = (long long)0x8000000000000000ull;
constexpr long long ABS_MASK = 0x7FFFFFFFFFFFFFFFll;
constexpr long long EXP_ONE = 1ll << 52;  // one unit of the exponent field

// MC-limited slope from three values with integer-pipe limiting:
//   dl = q0 - qm, dr = qp - q0; slope = 0 when dl*dr <= 0, else
//   sign(dl+dr) * min(2|dl|, 2|dr|, |dl+dr|/2).
// Returns half the slope (the offset from the zone average to a face).
// Matches the plain formula exactly for normal numbers (the scalings by two
// are exponent shifts); it differs only when dl*dr underflows to zero.
__device__ __forceinline__ double mc_half_slope(int limiter, double qm, double q0, double qp) {
    const double dl = q0 - qm, dr = qp - q0, s = dl + dr;
    if (!limiter) return 0.25 * s;
    const long long bl = dbits(dl), br = dbits(dr), bs = dbits(s);
    const long long al = bl & ABS_MASK, ar = br & ABS_MASK;
    if (((bl ^ br) < 0) || al == 0 || ar == 0) return 0.0;
    // both nonzero with one sign: s has that sign and |s| >= 2 min(|dl|, |dr|)
    const long long m2 = (al < ar ? al : ar) + EXP_ONE;   // 2 min(|dl|, |dr|)
    const long long hs = (bs & ABS_MASK) - EXP_ONE;        // |s| / 2
    long long lim = m2 < hs ? m2 : hs;
    lim -= EXP_ONE;                                       // half the limited slope
    return bitsd(lim | (bs & SIGN_BIT));
}

}  // namespace sdcd
