// Exact decisions of the growth rule on the device.
//
// Every decision of the method reduces to the sign of
//     Delta = log(a1/a2) - alpha * log(b1/b2),   a1, a2, b1, b2 positive int64 < 2^62,
// with alpha the exact binary64 value:
//   * add test (Eq. 2 > 0, strict):   a = (K+2d)/K, b = (V+k)/V
//   * remove test (Alg. 1, strict):   a = (K-2d)/K, b = (V-k)/V
//   * ranking factor 2 d / k^alpha of the max priority queue (Sec. 2):
//                                     a = d1/d2,   b = k1/k2
// The sign is the true mathematical sign, decided in stages:
//   1. integer shortcuts (b1 == b2 or a1 == a2);
//   1b. (add / remove tests) binary32 with a derived bound, see sign_delta32;
//   2. binary64 with a derived bound: each log-ratio term has absolute error
//      <= 13u|L| (u = 2^-53: 3u from the quotient, <= 1 ulp from log1p/log,
//      derivative bound 2 on the log1p branch, |L| > log 1.5 on the log
//      branch); the sign is taken when |Delta| > 2^-47 (|L1| + alpha|L2|);
//   3. exact tie test: alpha = P / 2^s with P odd, so Delta = 0 iff the
//      reduced b1/b2 is a 2^s-th power t^(2^s) of a reduced rational t and the
//      reduced a1/a2 equals t^P (unique factorisation);
//   4. double-double (error-free transformations of Dekker and Knuth; log by
//      exponent reduction and the series log x = 2 atanh((x-1)/(x+1))); the
//      sign is taken when |Delta| > 2^-92 (|L1| + alpha|L2|), otherwise the
//      decision is reported undecided (treated as a tie) and flagged.
#pragma once

#include "common.cuh"

#define EXACT_SLOW 1u       // a decision needed stage 3 or 4
#define EXACT_UNDECIDED 2u  // no stage settled a decision

namespace exact {

// ------------------------------------------------------------ double-double
struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
__device__ __forceinline__ dd fast_two_sum(double a, double b) {  // |a| >= |b|
    double s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ dd two_prod(double a, double b) {
    double p = a * b;
    return {p, fma(a, b, -p)};
}
__device__ __forceinline__ dd add(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    dd t = two_sum(x.lo, y.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd neg(dd x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dd mul(dd x, dd y) {
    dd p = two_prod(x.hi, y.hi);
    p.lo += x.hi * y.lo + x.lo * y.hi;
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd mul_d(dd x, double y) {
    dd p = two_prod(x.hi, y);
    p.lo += x.lo * y;
    return fast_two_sum(p.hi, p.lo);
}
__device__ __noinline__ dd div(dd x, dd y) {
    double q1 = x.hi / y.hi;
    dd r = add(x, neg(mul_d(y, q1)));
    double q2 = r.hi / y.hi;
    r = add(r, neg(mul_d(y, q2)));
    double q3 = r.hi / y.hi;
    return add(fast_two_sum(q1, q2), dd{q3, 0.0});
}
__device__ __forceinline__ dd from_i64(i64 a) {  // exact for |a| < 2^62
    double hi = (double)a;
    double lo = (double)(a - (i64)hi);
    return fast_two_sum(hi, lo);
}

// 2 atanh(z) = log((1+z)/(1-z)), |z| <= 1/3: odd power series, summed until
// the term falls below 2^-112 of the sum.
__device__ __noinline__ dd atanh2(dd z) {
    dd z2 = mul(z, z);
    dd term = z, sum = z;
    for (int j = 1; j < 90; ++j) {
        term = mul(term, z2);
        dd t = div(term, dd{(double)(2 * j + 1), 0.0});
        sum = add(sum, t);
        if (fabs(t.hi) <= 0x1p-112 * fabs(sum.hi)) break;
    }
    return mul_d(sum, 2.0);
}

// log(a1/a2) in double-double.
__device__ __noinline__ dd log_ratio(i64 a1, i64 a2) {
    i64 diff = a1 - a2;
    u64 ad = diff < 0 ? (u64)(-diff) : (u64)diff;
    if (ad <= (u64)a2 / 2) {
        // near 1: t = (a1-a2)/a2 keeps full relative precision, |t| <= 1/2
        dd t = div(from_i64(diff), from_i64(a2));
        dd z = div(t, add(dd{2.0, 0.0}, t));  // |z| <= 1/3
        return atanh2(z);
    }
    dd r = div(from_i64(a1), from_i64(a2));
    int e = ilogb(r.hi);
    dd m = {ldexp(r.hi, -e), ldexp(r.lo, -e)};  // m in [1, 2)
    if (m.hi > 1.4142135623730951) {
        m = {0.5 * m.hi, 0.5 * m.lo};
        e += 1;
    }
    dd z = div(add(m, dd{-1.0, 0.0}), add(m, dd{1.0, 0.0}));  // |z| <= 0.1716
    const dd LN2 = {0x1.62e42fefa39efp-1, 0x1.abc9e3b39803fp-56};  // ln 2 to 106 bits
    return add(atanh2(z), mul_d(LN2, (double)e));
}

// ------------------------------------------------------------ exact tie test
__device__ __forceinline__ i64 gcd64(i64 a, i64 b) {
    while (b) {
        i64 t = a % b;
        a = b;
        b = t;
    }
    return a;
}

// Root of x if x is a perfect square, else -1.
__device__ __forceinline__ i64 sqrt_exact(i64 x) {
    i64 r = (i64)sqrt((double)x);
    while (r > 0 && (unsigned __int128)r * (unsigned __int128)r > (unsigned __int128)x) --r;
    while ((unsigned __int128)(r + 1) * (unsigned __int128)(r + 1) <= (unsigned __int128)x) ++r;
    return ((unsigned __int128)r * (unsigned __int128)r == (unsigned __int128)x) ? r : -1;
}

// base^e == target (target < 2^63); stops as soon as the power exceeds it.
__device__ __forceinline__ bool power_is(i64 base, u64 e, i64 target) {
    if (base == 1) return target == 1;
    unsigned __int128 acc = 1;
    for (u64 i = 0; i < e; ++i) {
        acc *= (unsigned __int128)base;
        if (acc > (unsigned __int128)target) return false;
    }
    return acc == (unsigned __int128)target;
}

__device__ __noinline__ bool is_tie(i64 a1, i64 a2, i64 b1, i64 b2, double alpha) {
    i64 g = gcd64(a1, a2);
    i64 an = a1 / g, ad = a2 / g;
    g = gcd64(b1, b2);
    i64 bn = b1 / g, bd = b2 / g;
    if (bn == 1 && bd == 1) return an == 1 && ad == 1;
    // alpha = M 2^(E-1075) from its bits, reduced to P / 2^s with P odd
    u64 bits = (u64)__double_as_longlong(alpha);
    int E = (int)((bits >> 52) & 0x7ff);
    u64 M = bits & ((1ull << 52) - 1);
    if (E) M |= 1ull << 52;
    else E = 1;
    int tz = __ffsll((long long)M) - 1;
    u64 P = M >> tz;
    int s = 1075 - E - tz;
    u64 expo = P;
    if (s > 0) {
        for (int i = 0; i < s; ++i) {
            bn = sqrt_exact(bn);
            bd = sqrt_exact(bd);
            if (bn < 0 || bd < 0) return false;
            if (bn == 1 && bd == 1) return false;
        }
    } else {
        int sh = -s;
        expo = (sh >= 63 || P > (~0ull >> sh)) ? ~0ull : (P << sh);
    }
    return power_is(bn, expo, an) && power_is(bd, expo, ad);
}

// ------------------------------------------------------------ the sign
__device__ __forceinline__ double log_ratio_fast(i64 a1, i64 a2) {
    i64 diff = a1 - a2;
    u64 ad = diff < 0 ? (u64)(-diff) : (u64)diff;
    if (ad <= (u64)a2 / 2) return log1p((double)diff / (double)a2);
    return log((double)a1 / (double)a2);
}

// Stages 3 and 4.  The result is returned by value (the sign plus one, in
// bits 0-1, and the EXACT_* flags above it) so that no caller state has its
// address taken by this out-of-line function.
__device__ __noinline__ u32 sign_slow(i64 a1, i64 a2, i64 b1, i64 b2, double alpha) {
    const u32 slow = EXACT_SLOW << 2;
    if (is_tie(a1, a2, b1, b2, alpha)) return slow | 1u;
    dd L1 = log_ratio(a1, a2), L2 = log_ratio(b1, b2);
    dd D = add(L1, neg(mul_d(L2, alpha)));
    double E = 0x1p-92 * (fabs(L1.hi) + alpha * fabs(L2.hi));
    if (D.hi > E) return slow | 2u;
    if (D.hi < -E) return slow | 0u;
    return slow | (EXACT_UNDECIDED << 2) | 1u;
}

// Binary64 stage and beyond (integer shortcuts first).
__device__ __forceinline__ int sign_delta(i64 a1, i64 a2, i64 b1, i64 b2, double alpha, u32 &flags) {
    if (b1 == b2) return (a1 > a2) - (a1 < a2);
    if (a1 == a2) return (b2 > b1) - (b2 < b1);
    double L1 = log_ratio_fast(a1, a2), L2 = log_ratio_fast(b1, b2);
    double D = fma(-alpha, L2, L1);
    double E = 0x1p-47 * (fabs(L1) + alpha * fabs(L2));
    if (D > E) return 1;
    if (D < -E) return -1;
    const u32 r = sign_slow(a1, a2, b1, b2, alpha);
    flags |= r >> 2;
    return (int)(r & 3u) - 1;
}

// Binary32 stage in front of sign_delta (GB300 issues binary32 at many times
// the binary64 rate).  The same analysis as the binary64 stage with
// u32 = 2^-24: each log-ratio term is within 13 u32 |L| (quotient rounded
// three times, <= 1 ulp from log1pf / logf), alpha32 = fl(alpha) adds
// u32 alpha |L2|, the fused multiply-add one more rounding; the sign is taken
// when |Delta| > 2^-18 (|L1| + alpha |L2|) = 64 u32 (...).
// int64 -> binary32, rounded to nearest.  Values that fit 32 bits take the
// 32-bit conversion (same result; the 64-bit one is a slow instruction here).
__device__ __forceinline__ float i2f(i64 x) {
    return x == (i64)(int)x ? __int2float_rn((int)x) : __ll2float_rn(x);
}

__device__ __forceinline__ float log_ratio32(i64 a1, i64 a2) {
    i64 diff = a1 - a2;
    u64 ad = diff < 0 ? (u64)(-diff) : (u64)diff;
    if (ad <= (u64)a2 / 2) return log1pf(i2f(diff) / i2f(a2));
    return logf(i2f(a1) / i2f(a2));
}

__device__ __forceinline__ int sign_delta32(i64 a1, i64 a2, i64 b1, i64 b2, double alpha, float alpha32,
                                            u32 &flags) {
    if (b1 == b2) return (a1 > a2) - (a1 < a2);
    if (a1 == a2) return (b2 > b1) - (b2 < b1);
    float L1 = log_ratio32(a1, a2), L2 = log_ratio32(b1, b2);
    float D = fmaf(-alpha32, L2, L1);
    float E = 0x1p-18f * (fabsf(L1) + alpha32 * fabsf(L2));
    if (D > E) return 1;
    if (D < -E) return -1;
    return sign_delta(a1, a2, b1, b2, alpha, flags);
}

// Add test for a node outside c: (K+2d)/(V+k)^alpha > K/V^alpha.
__device__ __forceinline__ bool add_test(i64 K, i64 V, i64 d, i64 k, double alpha, float alpha32, u32 &flags) {
    if (K == 0) return true;  // f_c = 0 < f_{c+n} because d > 0
    return sign_delta32(K + 2 * d, K, V + k, V, alpha, alpha32, flags) > 0;
}

// Remove test for a member: (K-2d)/(V-k)^alpha > K/V^alpha.
__device__ __forceinline__ bool remove_test(i64 K, i64 V, i64 d, i64 k, double alpha, float alpha32, u32 &flags) {
    if (K == 0 || K - 2 * d == 0) return false;  // f_{c\n} = 0 <= f_c
    return sign_delta32(K - 2 * d, K, V - k, V, alpha, alpha32, flags) > 0;
}

// Necessary conditions (cheap filters, no transcendental): log1p(x) <= x and
// log1p(y) >= y/(1+y) give   add  => 2d(V+k) > alpha K k,
//                            remove => 2d(V-k) < alpha K k.
// Evaluated in binary32 (products stay below 2^125 < FLT_MAX); each side
// carries at most ~6 roundings of 2^-24 (alpha32 included), so a 2^-19
// margin keeps the filters one-sided.
__device__ __forceinline__ bool add_possible(i64 K, i64 V, i64 d, i64 k, float alpha32) {
    float lhs = 2.0f * i2f(d) * i2f(V + k);  // V + k formed exactly in int64
    float rhs = alpha32 * i2f(K) * i2f(k);
    return lhs > rhs * (1.0f - 0x1p-19f);
}
__device__ __forceinline__ bool remove_possible(i64 K, i64 V, i64 d, i64 k, float alpha32) {
    float lhs = 2.0f * i2f(d) * i2f(V - k);  // no cancellation: V - k exact in int64
    float rhs = alpha32 * i2f(K) * i2f(k);
    return lhs < rhs * (1.0f + 0x1p-19f);
}

}  // namespace exact
