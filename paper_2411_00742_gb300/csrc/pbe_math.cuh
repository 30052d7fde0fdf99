// Short-latency FP64 exp and log for the scalar kinetics chain.
//
// On GB300 every dependent FP64 operation costs ~65 cycles and every FP64
// instruction occupies the SM's FP64 pipe ~16 cycles, so the latency of the
// scalar chain between stages is set by the depth and the length of exp/log.
// These are written from the textbook constructions:
//   exp: Cody-Waite reduction x = k ln2 + r (|r| <= ln2/2, ln2 split in a
//        high part with trailing zero bits and a low part), exp(r) by its
//        Taylor polynomial of degree 13 evaluated with Estrin's scheme, and
//        the scale 2^k written into the exponent field;
//   exp_tab: the table-driven form (Tang's method): x = (64 m + j) ln2/64 + r,
//        exp x = 2^m 2^(j/64) exp(r), |r| <= ln2/128, exp(r) - 1 to r^5,
//        seven dependent FP64 operations;
//   log: x = 2^e m with m in [sqrt(1/2), sqrt(2)), log m = 2 atanh(z),
//        z = (m-1)/(m+1), by the odd Taylor series of atanh to z^23 (Estrin
//        in w = z^2), plus e ln2.
//   log_tab: the table-driven form (Tang's method): x = 2^e m, m in [1, 2),
//        the top 8 bits of m pick a centre c_j, log x = e ln2 + ln c_j +
//        log1p(r) with r = m / c_j - 1 (|r| <= 1/513) and log1p by its Taylor
//        polynomial to r^5 (Estrin), at an absolute (not relative) error of a
//        few 1e-16 near x = 1.
// The tables (pbe_log_table.h) are written by gen_log_table.py with 50-digit
// arithmetic.  Relative error is a few units of 2^-53 on the arguments the
// kinetics use (checked against the C library on the host by the tests).
// Arguments outside the handled ranges (non-positive or non-finite log input,
// exp of |x| > 700) return the IEEE limits of the function.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "pbe_log_table.h"

namespace pbe {

#ifdef __CUDACC__
static __constant__ double c_log_inv[256] = PBE_LOG_TAB_INV;
static __constant__ double c_log_ln[256] = PBE_LOG_TAB_LN;
static __constant__ double c_exp_tab[64] = PBE_EXP_TAB;
#endif
static const double h_log_inv[256] = PBE_LOG_TAB_INV;
static const double h_log_ln[256] = PBE_LOG_TAB_LN;
static const double h_exp_tab[64] = PBE_EXP_TAB;

__host__ __device__ __forceinline__ double pbe_bits_to_double(int64_t b)
{
#ifdef __CUDA_ARCH__
    return __longlong_as_double(b);
#else
    double d;
    memcpy(&d, &b, sizeof(d));
    return d;
#endif
}

__host__ __device__ __forceinline__ int64_t pbe_double_to_bits(double d)
{
#ifdef __CUDA_ARCH__
    return __double_as_longlong(d);
#else
    int64_t b;
    memcpy(&b, &d, sizeof(b));
    return b;
#endif
}

__host__ __device__ __forceinline__ double pbe_fma(double a, double b, double c)
{
#ifdef __CUDA_ARCH__
    return __fma_rn(a, b, c);
#else
    return __builtin_fma(a, b, c);
#endif
}

__host__ __device__ inline double pbe_exp(double x)
{
    if (!(x > -700.0)) return x != x ? x : 0.0;   // NaN stays NaN
    if (x > 700.0) return __builtin_huge_val();
    const double log2e = 1.4426950408889634;
    const double ln2_hi = 6.93147180369123816490e-01;   // 0x3fe62e42fee00000
    const double ln2_lo = 1.90821492927058770002e-10;   // ln2 - ln2_hi
    const double shifter = 6755399441055744.0;            // 1.5 * 2^52: rounds to an integer
    const double t = pbe_fma(x, log2e, shifter);
    const double kd = t - shifter;
    const int k = (int)(pbe_double_to_bits(t) & 0xffffffff) - (int)(pbe_double_to_bits(shifter) & 0xffffffff);
    double r = pbe_fma(-kd, ln2_hi, x);
    r = pbe_fma(-kd, ln2_lo, r);
    // Taylor coefficients 1/i!, i = 0..13
    const double c0 = 1.0, c1 = 1.0, c2 = 0.5, c3 = 1.6666666666666666e-01, c4 = 4.1666666666666664e-02,
                 c5 = 8.3333333333333332e-03, c6 = 1.3888888888888889e-03, c7 = 1.9841269841269841e-04,
                 c8 = 2.4801587301587302e-05, c9 = 2.7557319223985893e-06, c10 = 2.7557319223985888e-07,
                 c11 = 2.5052108385441720e-08, c12 = 2.0876756987868100e-09, c13 = 1.6059043836821613e-10;
    const double r2 = r * r, r4 = r2 * r2, r8 = r4 * r4;
    const double p01 = pbe_fma(c1, r, c0), p23 = pbe_fma(c3, r, c2), p45 = pbe_fma(c5, r, c4),
                 p67 = pbe_fma(c7, r, c6), p89 = pbe_fma(c9, r, c8), p1011 = pbe_fma(c11, r, c10),
                 p1213 = pbe_fma(c13, r, c12);
    const double q03 = pbe_fma(p23, r2, p01), q47 = pbe_fma(p67, r2, p45), q811 = pbe_fma(p1011, r2, p89);
    const double q07 = pbe_fma(q47, r4, q03), q813 = pbe_fma(p1213, r4, q811);
    const double p = pbe_fma(q813, r8, q07);
    // 2^k split in two factors so that k down to -1074 and up to 1023 stay exact
    const int k1 = k / 2, k2 = k - k1;
    const double s1 = pbe_bits_to_double((int64_t)(k1 + 1023) << 52);
    const double s2 = pbe_bits_to_double((int64_t)(k2 + 1023) << 52);
    return (p * s1) * s2;
}

// Table-driven exp (Tang's method): x = (64 m + j) ln2/64 + r with
// |r| <= ln2/128, exp x = 2^m 2^(j/64) exp(r), exp(r) - 1 by its Taylor
// polynomial to r^5 (the first omitted term, r^6/720, is below 4e-17).  The
// low part c = n (ln2/64)_lo of the reduction (|c| < 3e-14) enters only the
// linear term (r - c; the neglected c r is below 1.2e-16 even at |x| = 700,
// below 4e-18 for |x| < 20), so the polynomial starts one dependent operation
// earlier, and 2^m is added to the exponent field of the table value (exact:
// the result of an in-range argument is normal) instead of a multiplication:
// seven dependent FP64 operations.  The range test is an integer compare on
// the bits of x, applied to the result.
__host__ __device__ inline double pbe_exp_tab(double x)
{
    const double inv_l = 92.332482616893656;            // 64 / ln2
    const double shifter = 6755399441055744.0;            // 1.5 * 2^52: rounds to an integer
    const double t = pbe_fma(x, inv_l, shifter);
    const double nd = t - shifter;
    const int n = (int)(pbe_double_to_bits(t) & 0xffffffff) - (int)(pbe_double_to_bits(shifter) & 0xffffffff);
    const double r = pbe_fma(-nd, PBE_EXP_LN2_64_HI, x);
    const double c = nd * PBE_EXP_LN2_64_LO;
    const int j = n & 63, m = (n - j) / 64;
#ifdef __CUDA_ARCH__
    const double tj = c_exp_tab[j];
#else
    const double tj = h_exp_tab[j];
#endif
    const double tjs =
        pbe_bits_to_double((int64_t)((uint64_t)pbe_double_to_bits(tj) + ((uint64_t)(int64_t)m << 52)));   // tj 2^m
    const double a = pbe_fma(r, 1.0 / 6, 0.5), b = pbe_fma(r, 1.0 / 120, 1.0 / 24);
    const double r2 = r * r, rc = r - c;
    const double r4 = r2 * r2;
    const double u = pbe_fma(r4, b, pbe_fma(r2, a, rc));   // exp(r - c) - 1
    const double res = pbe_fma(tjs, u, tjs);
    const uint64_t ax = (uint64_t)pbe_double_to_bits(x) & 0x7fffffffffffffffULL;
    if (ax <= 0x4085E00000000000ULL) return res;   // |x| <= 700 (NaN has larger bits)
    if (x != x) return x;                          // NaN stays NaN
    return x > 0.0 ? __builtin_huge_val() : 0.0;
}

__host__ __device__ inline double pbe_log(double x)
{
    if (!(x > 0.0) || x == __builtin_huge_val()) {
        if (x == 0.0) return -__builtin_huge_val();
        if (x == __builtin_huge_val()) return x;
        return (x - x) / (x - x);   // NaN for negative or NaN input
    }
    int64_t b = pbe_double_to_bits(x);
    int e = (int)((b >> 52) & 0x7ff);
    if (e == 0) {                    // subnormal: scale into the normal range
        x *= 18014398509481984.0;    // 2^54
        b = pbe_double_to_bits(x);
        e = (int)((b >> 52) & 0x7ff) - 54;
    }
    e -= 1023;
    double m = pbe_bits_to_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);   // [1, 2)
    if (m > 1.4142135623730951) {
        m *= 0.5;
        e += 1;
    }
    const double f = m - 1.0;
    const double s = 2.0 + f;
    double z;
#ifdef __CUDA_ARCH__
    {
        double rc;
        asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(rc) : "d"(s));
        rc = pbe_fma(rc, pbe_fma(-s, rc, 1.0), rc);   // one Newton-Raphson step on 1/s
        const double q0 = f * rc;
        z = pbe_fma(rc, pbe_fma(-s, q0, f), q0);      // and one on the quotient
    }
#else
    z = f / s;
#endif
    const double w = z * z;
    // 2 atanh(z) = 2 z (1 + w/3 + w^2/5 + ... + w^11/23)
    const double a0 = 1.0, a1 = 1.0 / 3, a2 = 1.0 / 5, a3 = 1.0 / 7, a4 = 1.0 / 9, a5 = 1.0 / 11, a6 = 1.0 / 13,
                 a7 = 1.0 / 15, a8 = 1.0 / 17, a9 = 1.0 / 19, a10 = 1.0 / 21, a11 = 1.0 / 23;
    const double w2 = w * w, w4 = w2 * w2, w8 = w4 * w4;
    const double p01 = pbe_fma(a1, w, a0), p23 = pbe_fma(a3, w, a2), p45 = pbe_fma(a5, w, a4),
                 p67 = pbe_fma(a7, w, a6), p89 = pbe_fma(a9, w, a8), p1011 = pbe_fma(a11, w, a10);
    const double q03 = pbe_fma(p23, w2, p01), q47 = pbe_fma(p67, w2, p45), q811 = pbe_fma(p1011, w2, p89);
    const double q07 = pbe_fma(q47, w4, q03);
    const double P = pbe_fma(q811, w8, q07);
    const double ln2_hi = 6.93147180369123816490e-01, ln2_lo = 1.90821492927058770002e-10;
    const double ed = (double)e;
    const double two_z = z + z;
    // e ln2 + 2 z P, with the small terms first
    return pbe_fma(ed, ln2_hi, pbe_fma(two_z, P, ed * ln2_lo));
}

// log of the positive normal double with bits b, times 2^eadj
__host__ __device__ __forceinline__ double pbe_log_tab_bits(int64_t b, int eadj)
{
    const int e = (int)(b >> 52) - 1023 + eadj;
    const int j = (int)((b >> 44) & 255);
    const double m = pbe_bits_to_double((b & 0x000fffffffffffffLL) | 0x3ff0000000000000LL);   // [1, 2)
#ifdef __CUDA_ARCH__
    const double inv = c_log_inv[j], lnc = c_log_ln[j];
#else
    const double inv = h_log_inv[j], lnc = h_log_ln[j];
#endif
    const double ln2_hi = 6.93147180369123816490e-01, ln2_lo = 1.90821492927058770002e-10;
    const double ed = (double)e;
    const double H = pbe_fma(ed, ln2_hi, lnc);   // off the dependent chain
    const double r = pbe_fma(m, inv, -1.0);       // |r| <= 1/513
    // log1p(r) = r + r^2 (c2 + c3 r) + r^4 (c4 + c5 r), c_k = (-1)^(k+1) / k;
    // the first omitted term, r^6 / 6, is below 1e-17.  The small part
    // e ln2_lo joins r first, the large part H last: five dependent operations
    const double c2 = -0.5, c3 = 1.0 / 3, c4 = -0.25, c5 = 0.2;
    const double r2 = r * r;
    const double p23 = pbe_fma(c3, r, c2), p45 = pbe_fma(c5, r, c4);
    const double s1 = pbe_fma(ed, ln2_lo, r);
    const double r4 = r2 * r2;
    const double s2 = pbe_fma(r2, p23, s1);
    return H + pbe_fma(r4, p45, s2);
}

// The main path runs for every x; the classification of x is applied to the
// result, so it does not lengthen the dependent chain.
__host__ __device__ inline double pbe_log_tab(double x)
{
    const int64_t b = pbe_double_to_bits(x);
    const double res = pbe_log_tab_bits(b, 0);
    if (b >= 0x0010000000000000LL && b < 0x7ff0000000000000LL) return res;   // positive normal
    if (x == 0.0) return -__builtin_huge_val();
    if (x == __builtin_huge_val()) return x;
    if (!(x > 0.0)) return (x - x) / (x - x);   // NaN for negative or NaN input
    return pbe_log_tab_bits(pbe_double_to_bits(x * 18014398509481984.0), -54);   // subnormal, scaled by 2^54
}

}  // namespace pbe
