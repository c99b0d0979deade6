// sdc_fastmath.cuh -- FP64 helpers that keep work off GB300's narrow FP64 pipe.
//
// GB300 issues FP64 arithmetic at 1/61 of its FP32 rate, so the hot kernels
// count FP64 instructions.  Two classical devices are used:
//  * reciprocal and reciprocal square root refined from the hardware
//    approximations of PTX rcp.approx.ftz.f64 / rsqrt.approx.ftz.f64 (about 19
//    correct bits, issued outside the FP64 FMA pipe) by one step of a
//    third-order iteration (the series of 1/x and 1/sqrt(x) about the seed to
//    second order); the result is within a few ulp of the correctly rounded
//    value;
//  * exact operations on IEEE-754 bit patterns done on the integer pipe: |x|,
//    sign tests, x1/4 by an exponent decrement (exact while the result stays
//    normal; callers guard the range), and min of non-negative doubles (their
//    bit patterns order like the values).
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

// The hardware approximations are within 2^-19 relative (measured on GB300
// over 4M log-uniform arguments in 1e-30..1e30: |1 - x y| <= 2^-19.9 for the
// reciprocal, |1 - x y^2| <= 2^-19.0 for the reciprocal square root).  From a
// seed y with relative error e, one step of a higher-order iteration suffices:
//   1/x       = y (1 + e + e^2 + ...),              e = 1 - x y,
//   1/sqrt(x) = y (1 + e/2 + 3e^2/8 + ...),          e = 1 - x y^2,
// truncated after e^2: the next term is below 2^-56 relative, so the result is
// the correctly rounded value to within about an ulp, in 3 (reciprocal) and 5
// (reciprocal square root) FP64 operations instead of the 4 and 8 of two
// Newton-Raphson steps.

// 1/x for finite, normal, nonzero x
__device__ __forceinline__ double rcp_nr(double x) {
    const double y = rcp_seed(x);
    const double e = fma(-x, y, 1.0);
    return fma(y, fma(e, e, e), y);
}

// 1/sqrt(x) for finite, positive, normal x
__device__ __forceinline__ double rsqrt_nr(double x) {
    const double y = rsqrt_seed(x);
    const double e = fma(-x * y, y, 1.0);
    return fma(y * e, fma(e, 0.375, 0.5), y);
}

// sqrt(x) for finite, positive, normal x: x * rsqrt(x)
__device__ __forceinline__ double sqrt_nr(double x) { return x * rsqrt_nr(x); }

__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ double bitsd(long long b) { return __longlong_as_double(b); }

// Conversions between double and float on the integer pipe: GB300 issues the
// conversion instructions on its narrow FP64 pipe, where the FP32-Jacobian
// Newton spent a fifth of its FP64 issue slots on them.
// narrow: a double in the normal range of float to float, its mantissa
// truncated (the Jacobian's inputs, where the rounding does not matter);
// signed zeros exactly; anything else (tiny, huge, inf, nan) by the conversion
// instruction.
__device__ __forceinline__ float narrow(double x) {
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int e = (int)((hi >> 20) & 0x7ffu) - 896;  // exponent field of the float
    if (e <= 0 || e >= 255) {
        if (((hi << 1) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
        return (float)x;
    }
    return __uint_as_float((hi & 0x80000000u) | ((unsigned)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29));
}

// widen: a float to double, exactly (normal floats and zeros on the integer
// pipe; subnormals, inf and nan by the conversion instruction)
__device__ __forceinline__ double widen(float x) {
    const unsigned f = __float_as_uint(x);
    const unsigned ef = (f >> 23) & 0xffu;
    if (ef == 0u || ef == 255u) {
        if ((f << 1) == 0u) return __hiloint2double((int)(f & 0x80000000u), 0);
        return (double)x;
    }
    return __hiloint2double((int)((f & 0x80000000u) | ((ef + 896u) << 20) | ((f >> 3) & 0xfffffu)), (int)(f << 29));
}

// ---- float pairs ---------------------------------------------------------
// The FP32-pair Newton matrix is formed and eliminated on the FP32 pipe in
// double-float arithmetic: a value is the unevaluated sum hi + lo of two floats
// with |lo| below an ulp of hi (about 48 significant bits).  The operations are
// composed from the classical error-free transformations: Knuth's TwoSum
// (a + b = s + e exactly, six additions), Dekker's Fast2Sum (the same in three
// when |a| >= |b|) and the exact product through the fused multiply-add
// (a b = p + e with p = a b rounded and e = fma(a, b, -p)).  The explicitly
// rounded intrinsics keep the compiler from contracting or reassociating them.
// Every operation below is within a small multiple of 2^-46 of its operands'
// magnitude (relative, for products); the solve only forms Newton's step, whose
// residual and update stay in FP64, so the pair's rounding slows the iteration
// by about 2^-44 times the matrix's condition number and does not move the root.
struct f2 {
    float hi, lo;
    f2() = default;
    __device__ __forceinline__ constexpr f2(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ explicit f2(int v) : hi((float)v), lo(0.0f) {}  // small integers, exactly
};

// s + e = a + b exactly, given |a| >= |b| (or a = 0)
__device__ __forceinline__ f2 fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return f2(s, __fsub_rn(b, __fsub_rn(s, a)));
}

// s + e = a + b exactly, any order of magnitude
__device__ __forceinline__ f2 two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return f2(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

__device__ __forceinline__ f2 operator-(f2 x) { return f2(-x.hi, -x.lo); }

__device__ __forceinline__ f2 operator+(f2 x, f2 y) {
    const f2 s = two_sum(x.hi, y.hi);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ f2 operator-(f2 x, f2 y) { return x + (-y); }

// the product's leading part p and its correction e (x.lo y.lo, below 2^-46 of
// the product, is left out)
__device__ __forceinline__ void prod_parts(f2 x, f2 y, float& p, float& e) {
    p = __fmul_rn(x.hi, y.hi);
    e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
}

__device__ __forceinline__ f2 operator*(f2 x, f2 y) {
    float p, e;
    prod_parts(x, y, p, e);
    return fast_two_sum(p, e);
}

__device__ __forceinline__ bool operator!=(f2 x, f2 y) { return x.hi != y.hi || x.lo != y.lo; }

// a - x y with one normalisation
__device__ __forceinline__ f2 msub(f2 a, f2 x, f2 y) {
    float p, e;
    prod_parts(x, y, p, e);
    const f2 s = two_sum(a.hi, -p);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, __fsub_rn(a.lo, e)));
}
__device__ __forceinline__ double msub(double a, double x, double y) { return fma(-x, y, a); }
__device__ __forceinline__ float msub(float a, float x, float y) { return fmaf(-x, y, a); }

// 1/x from the hardware reciprocal y of x.hi (within an ulp: |r| <= 2^-22 for
// r = 1 - x y) and the series 1/x = y (1 + r + r^2 + ...), cut after r^2; x
// normal and nonzero
__device__ __forceinline__ f2 inv_mt(f2 x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x.hi));
    float r = __fmaf_rn(-x.hi, y, 1.0f);
    r = __fmaf_rn(-x.lo, y, r);
    return fast_two_sum(y, __fmul_rn(y, __fmaf_rn(r, r, r)));
}
__device__ __forceinline__ double inv_mt(double x) { return rcp_nr(x); }
__device__ __forceinline__ float inv_mt(float x) { return 1.0f / x; }

// x != 0 (a nan counts as nonzero, as in IEEE compares): for a double on the
// bit pattern (integer pipe), for float and float pairs on the FP32 pipe
__device__ __forceinline__ bool nonzero(double x) { return ((unsigned long long)dbits(x) << 1) != 0ull; }
__device__ __forceinline__ bool nonzero(float x) { return x != 0.0f; }
__device__ __forceinline__ bool nonzero(f2 x) { return x.hi != 0.0f || x.lo != 0.0f; }

// |x| ordered on the integer pipe: the leading float decides
__device__ __forceinline__ unsigned int mag2(f2 x) { return (unsigned int)__float_as_int(x.hi) << 1; }

// the working type MT of a Newton matrix: identity for double
template <typename MT> __device__ __forceinline__ MT to_mt(double x);
template <> __device__ __forceinline__ double to_mt<double>(double x) { return x; }
template <> __device__ __forceinline__ float to_mt<float>(double x) { return narrow(x); }
// a double as a float pair: hi its leading 24 bits (truncated), lo the leading
// 24 of the rest (x - hi is exact in FP64: the two share their exponent).  For
// x in float's normal range the rest is the 29 mantissa bits below hi's, so lo
// is formed from them on the integer pipe: their leading one gives lo's
// exponent, the next 23 bits (truncated) its mantissa, x its sign; a rest of
// zero gives +0, as x - hi does.  Elsewhere (and where lo would not be a normal
// float) the FP64 difference and narrow.
template <> __device__ __forceinline__ f2 to_mt<f2>(double x) {
    const float h = narrow(x);
    const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
    const int ef = (int)((hi >> 20) & 0x7ffu);
    const int e = ef - 896;  // exponent field of x as a float
    const unsigned r = lo & 0x1fffffffu;
    if (e > 0 && e < 255) {
        if (r == 0u) return f2(h, 0.0f);
        const int p = 31 - __clz((int)r);   // leading one of the rest, 0..28
        const int fe = ef - 948 + p;        // lo's exponent field: r 2^(ef - 1075) = 1.f 2^(ef - 1075 + p)
        if (fe > 0) {
            const unsigned m = (p <= 23 ? (r << (23 - p)) : (r >> (p - 23))) & 0x7fffffu;
            return f2(h, __uint_as_float((hi & 0x80000000u) | ((unsigned)fe << 23) | m));
        }
    }
    return f2(h, narrow(x - widen(h)));
}
__device__ __forceinline__ double from_mt(double x) { return x; }
__device__ __forceinline__ double from_mt(float x) { return widen(x); }
__device__ __forceinline__ double from_mt(f2 x) { return widen(x.hi) + widen(x.lo); }

// The type in which a solve's step is tested and applied: a float pair is
// summed into a double once; a float or double step is used as it is.
template <typename MT> struct StepType { using type = MT; };
template <> struct StepType<f2> { using type = double; };
__device__ __forceinline__ double step_value(f2 x) { return from_mt(x); }
__device__ __forceinline__ double step_value(double x) { return x; }
__device__ __forceinline__ float step_value(float x) { return x; }

constexpr long long SIGN_BIT = (long long)0x8000000000000000ull;
constexpr long long ABS_MASK = 0x7FFFFFFFFFFFFFFFll;
constexpr long long EXP_ONE = 1ll << 52;  // one unit of the exponent field

// |x| as an unsigned integer that orders like |x|: the bit pattern shifted
// left by one, which drops the sign (a mask of the sign bit would be compiled
// into an FP64 absolute value on the FP64 pipe; the shift stays on the integer
// pipe).  Zero for +-0.
__device__ __forceinline__ unsigned long long mag2(double x) { return (unsigned long long)dbits(x) << 1; }
__device__ __forceinline__ unsigned int mag2(float x) { return (unsigned int)__float_as_int(x) << 1; }

// MC-limited slope from three values with integer-pipe limiting:
//   dl = q0 - qm, dr = qp - q0; slope = 0 when dl*dr <= 0, else
//   sign(dl+dr) * min(2|dl|, 2|dr|, |dl+dr|/2).
// Returns half the slope (the offset from the zone average to a face), formed
// as sign(s) * min(|dl|, |dr|, |s|/4) with s = dl + dr: the minimum is taken on
// bit patterns (they order like the values for every non-negative double,
// subnormals included) and |s|/4 is an exponent decrement of two, exact while
// |s| >= 2^-1020.  Below that the offset is returned as zero; it then differs
// from the plain formula by less than 2^-1022 in absolute value.  The plain
// formula's dl*dr test also reads zero when the product underflows; here only
// the signs decide.  Everywhere else the two agree exactly.
// The same from the two one-sided differences dl = q0 - qm and dr = qp - q0
// (a pass that forms each difference once per face passes them in).
__device__ __forceinline__ double mc_half_slope_d(int limiter, double dl, double dr) {
    const double s = dl + dr;
    if (!limiter) return 0.25 * s;
    const long long bl = dbits(dl), br = dbits(dr), bs = dbits(s);
    // magnitudes as bit patterns shifted left by one (mag2)
    const unsigned long long al = mag2(dl), ar = mag2(dr), as = mag2(s);
    constexpr unsigned long long E2 = (unsigned long long)EXP_ONE << 1;
    if (((bl ^ br) < 0) || al == 0 || ar == 0 || as < 3 * E2) return 0.0;
    const unsigned long long q = as - 2 * E2;  // |s| / 4
    unsigned long long lim = al < ar ? al : ar;
    lim = lim < q ? lim : q;
    return bitsd((long long)(lim >> 1) | (bs & SIGN_BIT));
}

__device__ __forceinline__ double mc_half_slope(int limiter, double qm, double q0, double qp) {
    return mc_half_slope_d(limiter, q0 - qm, qp - q0);
}

}  // namespace sdcd
