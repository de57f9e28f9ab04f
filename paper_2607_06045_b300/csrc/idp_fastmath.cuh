// idp_fastmath.cuh -- FP64 reciprocal, square root and natural logarithm for
// the FP64 flux arithmetic, in fewer FP64-pipe instructions than the
// correctly rounded library routines (about 1 ulp instead of 0.5):
//  - reciprocal: Newton-Raphson iteration r <- r + r (1 - x r) from the PTX
//    approximation rcp.approx.ftz.f64 (two steps);
//  - square root: Goldschmidt's coupled iteration for s ~ sqrt(x) and
//    h ~ 1 / (2 sqrt(x)) from the PTX approximation rsqrt.approx.ftz.f64,
//    then one Newton correction s <- s + h (x - s^2);
//  - logarithm: P. T. P. Tang's table-driven method (ACM TOMS 16(4), 1990):
//    x = 2^k m, m = F (1 + r) with F = 1 + j/128 the nearest table point,
//    ln x = k ln 2 + ln F + ln(1 + r), |r| <= 2^-8, ln(1 + r) from its Taylor
//    series to r^7, ln F and ln 2 carried as a head and a tail.
// The inputs here are positive, finite and normal (densities, pressures,
// wave speeds, products of differences that are not zero); other inputs give
// unspecified results.
#pragma once

#include <cuda_runtime.h>

namespace idp {

constexpr int kLogTab = 128;

// Table of Tang's method, formed on the host (host_log_table in idp_host.cu):
// inv[j] = 1 / F_j rounded, hi[j] + lo[j] = ln F_j, F_j = 1 + j / 128; ln 2 as
// ln2_hi (42 significant bits, so k * ln2_hi is exact for |k| < 2^11) + ln2_lo.
struct LogTab {
    double inv[kLogTab], hi[kLogTab], lo[kLogTab];
    double ln2_hi, ln2_lo;
};

__device__ __forceinline__ double fast_rcp(double x) {
    double r;
    asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
    double e = fma(-x, r, 1.0);
    r = fma(r, e, r);
    e = fma(-x, r, 1.0);
    return fma(r, e, r);
}

__device__ __forceinline__ double fast_sqrt(double x) {
    double y;
    asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
    double s = __dmul_rn(x, y), h = 0.5 * y;
    double r = fma(-s, h, 0.5);
    s = fma(s, r, s);
    h = fma(h, r, h);
    double d = fma(-s, s, x);
    return fma(d, h, s);
}

__device__ __forceinline__ double fast_log(double x, const LogTab *__restrict__ T) {
    const int hi = __double2hiint(x), lo = __double2loint(x);
    int k = (hi >> 20) - 1023;
    const int mh = hi & 0x000fffff;
    int j = (mh + (1 << 12)) >> 13;            // nearest of 128 points in [1, 2]
    // m in [1, 2) with x = 2^k m; j = 128 rounds to 2: use m / 2 and F = 1
    int mhi = mh | 0x3ff00000;
    if (j == kLogTab) { j = 0; k += 1; mhi = mh | 0x3fe00000; }
    const double m = __hiloint2double(mhi, lo);
    const double F = __hiloint2double(0x3ff00000 | (j << 13), 0);
    const double f = m - F;                   // exact (m and F within a factor 2)
    const double r = f * __ldg(&T->inv[j]);
    const double r2 = r * r;
    double p = fma(r, 1.0 / 7.0, -1.0 / 6.0);
    p = fma(r, p, 1.0 / 5.0);
    p = fma(r, p, -1.0 / 4.0);
    p = fma(r, p, 1.0 / 3.0);
    p = fma(r, p, -0.5);
    const double kd = (double)k;
    const double head = fma(kd, T->ln2_hi, __ldg(&T->hi[j]));
    const double tail = fma(kd, T->ln2_lo, __ldg(&T->lo[j]));
    return head + (r + fma(r2, p, tail));
}

}  // namespace idp
