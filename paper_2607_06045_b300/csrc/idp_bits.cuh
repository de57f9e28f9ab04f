// idp_bits.cuh -- FP32/FP64 conversions and FP64 comparisons on the integer
// pipe.
//
// B300 executes FP64 arithmetic, FP64 compares and min/max, and conversions
// between FP32 and FP64 on its FP64 pipe, which runs at 1/64 of the FP32
// rate; a compare or a min costs as much as a fused multiply-add there. The
// element pass therefore moves values between its FP32 flux arithmetic and its
// FP64 limiter, and takes the limiter's comparisons, through the IEEE-754 bit
// patterns on the integer pipe:
//  - float -> double is exact (rebias the exponent, widen the fraction);
//    subnormal floats flush to a zero of the same sign;
//  - double -> float rounds to nearest with ties away from zero (error at
//    most half an ulp, as for the hardware conversion); magnitudes below the
//    normal float range flush to a signed zero, above it round to infinity,
//    NaN stays NaN;
//  - the order key of a double (its magnitude bits, negated for negative
//    numbers) is a 64-bit integer that orders all non-NaN doubles like their
//    values, with -0 == +0, so <, min and max become integer operations.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace idp {

__device__ __forceinline__ double f2d(float x) {
    const unsigned b = __float_as_uint(x), a = b & 0x7fffffffu, s = b & 0x80000000u;
    // exponent bias 127 -> 1023; Inf/NaN keep the all-ones exponent
    unsigned hi = s | ((a >> 3) + (a >= 0x7f800000u ? 0x70000000u : 0x38000000u));
    unsigned lo = b << 29;
    if (a < 0x00800000u) { hi = s; lo = 0u; }
    return __hiloint2double((int)hi, (int)lo);
}

__device__ __forceinline__ float d2f(double x) {
    unsigned long long bits = (unsigned long long)__double_as_longlong(x);
    const unsigned ohi = (unsigned)(bits >> 32);
    bits += 0x10000000ull;   // half an ulp of the 23-bit fraction
    const unsigned hi = (unsigned)(bits >> 32), lo = (unsigned)bits;
    const unsigned s = ohi & 0x80000000u, a = hi & 0x7fffffffu;
    // fraction: 20 bits from hi, 3 from lo; exponent bias 1023 -> 127
    unsigned m = __funnelshift_l(lo, a, 3) - (896u << 23);
    if (a < (897u << 20)) m = 0u;
    else if (a >= (1151u << 20)) m = (ohi & 0x7fffffffu) > 0x7ff00000u ? 0x7fc00000u : 0x7f800000u;
    return __uint_as_float(s | m);
}

__device__ __forceinline__ long long okey(double x) {
    const long long b = __double_as_longlong(x);
    const long long m = b & 0x7fffffffffffffffLL;
    return b < 0 ? -m : m;
}

// the double with order key k (-0 comes back as +0)
__device__ __forceinline__ double okey_value(long long k) {
    return __longlong_as_double(k < 0 ? (-k | (long long)0x8000000000000000ULL) : k);
}

__device__ __forceinline__ bool dlt(double a, double b) { return okey(a) < okey(b); }
__device__ __forceinline__ double dmin(double a, double b) { return okey(b) < okey(a) ? b : a; }
__device__ __forceinline__ double dmax(double a, double b) { return okey(b) > okey(a) ? b : a; }

// For operands known to be >= +0 (or -0) and not NaN the bits order directly.
__device__ __forceinline__ bool nn_lt(double a, double b) {
    return (__double_as_longlong(a) & 0x7fffffffffffffffLL) < (__double_as_longlong(b) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double nn_min(double a, double b) { return nn_lt(b, a) ? b : a; }

// x > 0 and finite (NaN fails)
__device__ __forceinline__ bool dpos(double x) {
    const long long b = __double_as_longlong(x);
    return b > 0 && b < 0x7ff0000000000000LL;
}
// x < 0 (-0 and NaN fail)
__device__ __forceinline__ bool dneg(double x) {
    const long long b = __double_as_longlong(x);
    return b < 0 && b != (long long)0x8000000000000000ULL && (b & 0x7fffffffffffffffLL) <= 0x7ff0000000000000LL;
}
__device__ __forceinline__ bool dfinite(double x) {
    return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}

}  // namespace idp
