// sdc_pow.cuh -- T^nu = 2^(nu log2 T) for the power-law rate factors of the
// reaction network, with a table-driven base-2 logarithm and exponential
// (P. T. P. Tang, ACM TOMS 15 (1989) 144-157 and 16 (1990) 378-400): per call
// about 13 FP64 instructions for log2 and 9 for exp2, against about 30 and 16
// for the library's log and exp, on a GPU whose FP64 pipe is the bottleneck.
// Tables and coefficients: sdc_pow_tables.h, written by gen_pow_tables.py.
//
// Accuracy: log2 x is rounded once from a sum accurate to about 5e-18 (so
// within 1.1e-16 |log2 x| + 5e-18), exp2 within about 2.6e-16 relative; T^nu
// = 2^y, y = nu log2 T, therefore within ln 2 (2.2e-16 |y| + 5e-18 nu) +
// 2.6e-16 relative (the rounding of the product nu log2 T dominates, as that of
// nu log T does in exp(nu log T)).  Arguments outside the tables' range (T not
// a positive normal number; |y| >= 512) take the library functions.
#pragma once
#include <cuda_runtime.h>

#include "sdc_fastmath.cuh"
#include "sdc_pow_tables.h"

namespace sdcd {

// log2 x (the library's log2 where x is not a positive normal number)
__device__ __forceinline__ double log2_tab(double x) {
    const long long b = dbits(x);
    const int ef = (int)((b >> 52) & 0x7ff);
    if (b <= 0 || ef == 0 || ef == 0x7ff) return log2(x);  // not positive, subnormal, inf or nan
    const int j = (int)((b >> 45) & 127);
    const double m = bitsd((b & 0x000fffffffffffffll) | 0x3ff0000000000000ll);  // [1, 2)
    const double r = fma(m, __ldg(POW_LOG_C + j), -1.0);                            // |r| <= 1/255
    double p = fma(r, POW_LOG_A6, POW_LOG_A5);
    p = fma(r, p, POW_LOG_A4);
    p = fma(r, p, POW_LOG_A3);
    p = fma(r, p, POW_LOG_A2);
    p = fma(r, p, POW_LOG_A1);
    p = r * p;
    // e + hi exactly as a pair (Fast2Sum: |e| >= hi when e != 0), then one rounding
    const double e = (double)(ef - 1023), hi = __ldg(POW_LOG_HI + j);
    const double s = e + hi;
    const double se = hi - (s - e);
    return s + ((p + __ldg(POW_LOG_LO + j)) + se);
}

// 2^y
__device__ __forceinline__ double exp2_tab(double y) {
    // |y| < 512 (and not nan) read from the exponent field, on the integer pipe;
    // beyond it the library (the scaling below keeps 2^y normal for |y| < 1021)
    if (((dbits(y) >> 52) & 0x7ff) >= 1023 + 9) return exp2(y);
    const double SHIFT = 0x1.8p52;           // 256 y + SHIFT rounds 256 y to an integer in the low bits
    const double t = fma(y, 256.0, SHIFT);
    const double nf = t - SHIFT;
    const double r = fma(nf, -0x1p-8, y);    // y - n/256 exactly, |r| <= 1/512
    const int n = (int)(dbits(t) & 0xffffffffll);
    const int i = n & 255, k = n >> 8;
    double p = fma(r, POW_EXP_B4, POW_EXP_B3);
    p = fma(r, p, POW_EXP_B2);
    p = fma(r, p, POW_EXP_B1);
    p = r * p;
    const double ti = __ldg(POW_EXP2_T + i);
    const double v = fma(ti, p, ti);         // 2^(i/256) 2^r, in [0.997, 2.003)
    return bitsd(dbits(v) + ((long long)k << 52));
}

}  // namespace sdcd
