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

// Conversions between FP64 and FP32 on the integer pipe (F2F conversions
// issue on the FP64 pipe on this part).  Both give the hardware's results
// bit for bit: d2f_rn rounds to nearest even, f2d widens exactly.  Normal
// results and zeros take the integer path; the rest (FP32 subnormals,
// overflow from beyond FLT_MAX, inf, NaN) the hardware conversion.
static __device__ __forceinline__ float d2f_rn(double v)
{
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
    const unsigned sign = hi & 0x80000000u;
    const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;  // the FP32 exponent field
    if (e >= 1 && e <= 254) {
        // the 23 FP32 mantissa bits (20 from hi, 3 from lo); the other 29 round
        const unsigned m = ((hi & 0xfffffu) << 3) | (lo >> 29);
        const unsigned rem = lo & 0x1fffffffu;
        const unsigned up = (rem > 0x10000000u || (rem == 0x10000000u && (m & 1u))) ? 1u : 0u;
        // a carry out of the mantissa moves into the exponent (255: inf)
        return __uint_as_float((sign | ((unsigned)e << 23) | m) + up);
    }
    if ((b << 1) == 0) return __uint_as_float(sign);
    return __double2float_rn(v);
}

static __device__ __forceinline__ double f2d(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned e = (u >> 23) & 0xffu;
    if (e - 1u < 254u) {
        const unsigned hi = (u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3);
        return __hiloint2double((int)hi, (int)(u << 29));
    }
    if ((u << 1) == 0) return __hiloint2double((int)(u & 0x80000000u), 0);
    return (double)f;
}

// FP64 value in the reconstruction precision R, and back to FP64
template <class R> __device__ __forceinline__ R to_R(double v);
template <> __device__ __forceinline__ double to_R<double>(double v) { return v; }
template <> __device__ __forceinline__ float to_R<float>(double v) { return d2f_rn(v); }
static __device__ __forceinline__ double to_d(double v) { return v; }
static __device__ __forceinline__ double to_d(float v) { return f2d(v); }

}  // namespace rich
