// FP64 reciprocal and square root with fewer FP64 issue slots than the
// IEEE-rounded operations.  GB300 issues FP64 arithmetic at 2 lanes per
// clock per SM, and measured on it (throughput of dependent chains against
// a chain of FMAs): IEEE 1/x costs ~4.5 FP64 issue slots, the rounded
// square root ~7.4, rsqrt ~4.8, while the approximate reciprocal
// rcp.approx.ftz.f64 issues outside the FP64 pipe.
#pragma once

#include <cstdint>

namespace rich {

// 1/x for a normal x with |x| in [2^-1021, 2^1020): the hardware's
// approximate reciprocal y (about 20 correct bits, issued outside the FP64
// pipe) refined by the geometric series 1/x = y / (1 - e) ~ y (1 + e + e^2),
// e = 1 - x y: three FMAs, relative error O(e^3) plus rounding, so within
// one ulp of the correctly rounded quotient, where IEEE division costs
// about 4.5 FP64 issue slots.  Other arguments take the IEEE division.
static __device__ __forceinline__ double recip(double x)
{
    const unsigned ex = ((unsigned)__double2hiint(x) >> 20) & 0x7ffu;
    if (ex - 2u > 2040u) return 1.0 / x;
    double y;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    const double e = fma(-x, y, 1.0);
    return fma(fma(e, e, e), y, y);
}
static __device__ __forceinline__ float recip(float x) { return 1.0f / x; }

// sqrt(x) as x / sqrt(x) through one reciprocal square root (about 5.8
// FP64 issue slots against 7.4 for the rounded square root) for +0 and
// positive normal x; subnormal, infinite, negative and NaN arguments take
// the rounded square root.  Tests and selects on the bits.
static __device__ __forceinline__ double sqrt_nonneg(double x)
{
    const long long b = __double_as_longlong(x);
    if (b != 0 && (unsigned long long)(b - 0x0010000000000000ll) >= 0x7fe0000000000000ull) return sqrt(x);
    const double r = x * rsqrt(x);
    return b == 0 ? 0.0 : r;
}
static __device__ __forceinline__ float sqrt_nonneg(float x) { return sqrtf(x); }

}  // namespace rich
