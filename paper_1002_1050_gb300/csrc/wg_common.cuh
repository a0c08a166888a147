// wg_common.cuh -- device-side building blocks shared by the sm_103a kernels.
//
//  * double-double arithmetic from the published error-free transforms
//    (Knuth's TwoSum, Dekker's Fast2Sum, FMA-based TwoProd) for the seeds;
//  * per-angle quantities of Sec. 4.2.2's first precomputation (cos beta,
//    ln cos(beta/2), ln sin(beta/2)) evaluated with CUDA's math functions;
//  * the seed of Eqs. ini1-ini2 / logstart (Sec. 3.2) as a scaled double;
//  * exponent-field manipulation of doubles (exact multiplication by 2^k for
//    normal values, done on the integer pipe so the scarce FP64 pipe is left to
//    the recursion).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "wg_internal.h"

namespace wg {

// ---------------------------------------------------------------------------
// double-double (value = hi + lo, |lo| <= ulp(hi)/2)
// ---------------------------------------------------------------------------
struct dd {
    double hi, lo;
};

__device__ __forceinline__ dd two_sum(double a, double b) {
    double s = __dadd_rn(a, b);
    double bb = __dsub_rn(s, a);
    double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dd fast_two_sum(double a, double b) {  // |a| >= |b|
    double s = __dadd_rn(a, b);
    double e = __dsub_rn(b, __dsub_rn(s, a));
    return {s, e};
}

__device__ __forceinline__ dd two_prod(double a, double b) {
    double p = __dmul_rn(a, b);
    double e = __fma_rn(a, b, -p);
    return {p, e};
}

__device__ __forceinline__ dd dd_add(dd x, dd y) {
    dd s = two_sum(x.hi, y.hi);
    double e = __dadd_rn(s.lo, __dadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

__device__ __forceinline__ dd dd_neg(dd x) { return {-x.hi, -x.lo}; }

// x * k for a small integer k (|k| < 2^31): k is exact in double, product via TwoProd
__device__ __forceinline__ dd dd_mul_d(dd x, double k) {
    dd p = two_prod(x.hi, k);
    double e = __fma_rn(x.lo, k, p.lo);
    return fast_two_sum(p.hi, e);
}

// ---------------------------------------------------------------------------
// float-float (value = hi + lo in two floats, ~48 significant bits) on the FP32 pipe,
// from the same error-free transforms in single precision.  Used to move the weighted
// l-sum off GB300's narrow FP64 pipe.
// ---------------------------------------------------------------------------
struct ff {
    float hi, lo;
};

// Split a double into float hi + lo with integer and FP32 operations only (no
// double<->float conversion, which runs on the FP64 unit): hi = x truncated to 24
// significant bits, lo = the next 24 bits of the remainder.  Valid for
// 2^-100 <= |x| < 2^127; other inputs give garbage the caller must mask.
__device__ __forceinline__ ff split_ff(double x) {
    const long long b = __double_as_longlong(x);
    const int hi32 = (int)(b >> 32);
    const int eu = ((hi32 >> 20) & 0x7ff) - 1023;              // unbiased exponent
    const unsigned sign = (unsigned)hi32 & 0x80000000u;
    const unsigned long long mant = (unsigned long long)b & 0xfffffffffffffULL;
    ff r;
    r.hi = __uint_as_float(sign | ((unsigned)(eu + 127) << 23) | (unsigned)(mant >> 29));
    const unsigned rem = (unsigned)(mant & 0x1fffffffULL);      // 29 bits below hi's last bit
    // rem * 2^(eu - 52) = (rem * 2^-29) * 2^(eu - 23), both factors normal for eu >= -100
    const float scale = __uint_as_float(sign | ((unsigned)(eu - 23 + 127) << 23));
    r.lo = __fmul_rn(__fmul_rn(__uint2float_rn(rem), 0x1p-29f), scale);
    return r;
}

__device__ __forceinline__ ff ff_fast(float a, float b) {  // |a| >= |b|
    const float s = __fadd_rn(a, b);
    return ff{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ ff ff_add(ff x, ff y) {
    const float s = __fadd_rn(x.hi, y.hi);
    const float bb = __fsub_rn(s, x.hi);
    const float e = __fadd_rn(__fsub_rn(x.hi, __fsub_rn(s, bb)), __fsub_rn(y.hi, bb));
    return ff_fast(s, __fadd_rn(e, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }

__device__ __forceinline__ ff ff_mul(ff x, ff y) {
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return ff_fast(p, e);
}

__device__ __forceinline__ ff ff_of(float2 v) { return ff{v.x, v.y}; }

// a non-negative integer below 2^31 as float-float (exact)
__device__ __forceinline__ ff ff_int(long long n) {
    const float hi = __ll2float_rz(n);
    return ff{hi, __ll2float_rn(n - (long long)hi)};
}

// double -> float on the integer pipe, truncating; |x| < 2^-126 flushes to a signed zero,
// |x| >= 2^128 saturates to infinity.  (Used where float precision of the value suffices.)
__device__ __forceinline__ float d2f_trunc(double x) {
    const long long b = __double_as_longlong(x);
    const int hi = (int)(b >> 32);
    const int e = ((hi >> 20) & 0x7ff) - 1023;
    const unsigned sign = (unsigned)hi & 0x80000000u;
    if (e < -126) return __uint_as_float(sign);
    if (e > 127) return __uint_as_float(sign | 0x7f800000u);
    return __uint_as_float(sign | ((unsigned)(e + 127) << 23) |
                           (unsigned)(((unsigned long long)b & 0xfffffffffffffULL) >> 29));
}

// x 2^-shift as a float, rounded to nearest (ties to even), on the integer pipe: the
// exponent is re-biased in the double's bit pattern and the 29 dropped mantissa bits
// rounded (a carry out of the mantissa moves into the exponent, as it should).  Zero and
// subnormal doubles give a signed zero, results below 2^-126 flush to a signed zero, and
// results from 2^128 up (or an infinite or NaN x) are infinite or NaN.
__device__ __forceinline__ float d2f_rn_scaled(double x, int shift) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const unsigned sign = (unsigned)(b >> 32) & 0x80000000u;
    const int ef = (int)((b >> 52) & 0x7ff);
    if (ef == 0x7ff) return __uint_as_float(sign | ((b & 0xfffffffffffffULL) ? 0x7fc00000u : 0x7f800000u));
    const int e = ef - 1023 - shift;  // unbiased exponent of the result
    if (ef == 0 || e < -126) return __uint_as_float(sign);
    if (e > 127) return __uint_as_float(sign | 0x7f800000u);
    unsigned long long r = ((unsigned long long)(e + 127) << 52) | (b & 0xfffffffffffffULL);
    r += 0x0fffffffULL + ((r >> 29) & 1);
    return __uint_as_float(sign | (unsigned)(r >> 29));
}

// acc += w * u in float-float (Dekker product with FMA, Knuth TwoSum, Fast2Sum)
__device__ __forceinline__ void ff_mac(ff &acc, float wh, float wl, float uh, float ul) {
    const float p = __fmul_rn(wh, uh);
    float e = __fmaf_rn(wh, uh, -p);
    e = __fmaf_rn(wh, ul, e);
    e = __fmaf_rn(wl, uh, e);
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    const float lo = __fadd_rn(acc.lo, __fadd_rn(err, e));
    acc.hi = __fadd_rn(s, lo);
    acc.lo = __fsub_rn(lo, __fsub_rn(acc.hi, s));
}

// ff_mac on a (re, im) pair with the packed f32x2 instructions: the same rounding steps
// lane by lane (a - b is written fma(b, -1, a), which rounds a - b once, and p - bb as
// -(np + bb) with np = -p), so each lane equals ff_mac's result bit for bit, in 15
// instructions instead of 28.  (hi, lo): the accumulators; (wh, wl): the weight pair;
// (uh, ul): the value as float-float.
__device__ __forceinline__ void ff_mac2(float2 &hi, float2 &lo, float2 wh, float2 wl, float uh, float ul) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 Uh = make_float2(uh, uh), Ul = make_float2(ul, ul), nUh = make_float2(-uh, -uh);
    const float2 np = __fmul2_rn(wh, nUh);          // -p
    float2 e = __ffma2_rn(wh, Uh, np);              // wh uh - p, exact
    e = __ffma2_rn(wh, Ul, e);
    e = __ffma2_rn(wl, Uh, e);
    const float2 s = __ffma2_rn(np, m1, hi);        // hi + p
    const float2 bb = __ffma2_rn(hi, m1, s);        // s - hi
    const float2 t1 = __ffma2_rn(bb, m1, s);        // s - bb
    const float2 t2 = __ffma2_rn(t1, m1, hi);       // hi - (s - bb)
    const float2 q = __fadd2_rn(np, bb);            // -(p - bb)
    const float2 err = __ffma2_rn(q, m1, t2);       // t2 + (p - bb)
    const float2 l2 = __fadd2_rn(lo, __fadd2_rn(err, e));
    const float2 h2 = __fadd2_rn(s, l2);
    lo = __ffma2_rn(__ffma2_rn(s, m1, h2), m1, l2);  // l2 - (h2 - s)
    hi = h2;
}

// (x.hi, x.lo) += (y.hi, y.lo) in float-float for a pair of values with the packed f32x2
// instructions: per lane the steps of ff_add (TwoSum, then Fast2Sum), a - b written
// fma(b, -1, a) (one rounding, as a subtraction)
__device__ __forceinline__ void ff_add2(float2 &xh, float2 &xl, float2 yh, float2 yl) {
    const float2 m1 = make_float2(-1.f, -1.f);
    const float2 s = __fadd2_rn(xh, yh);
    const float2 bb = __ffma2_rn(xh, m1, s);                         // s - xh
    const float2 t1 = __ffma2_rn(__ffma2_rn(bb, m1, s), m1, xh);     // xh - (s - bb)
    const float2 e = __fadd2_rn(t1, __ffma2_rn(bb, m1, yh));         // + (yh - bb)
    const float2 e2 = __fadd2_rn(e, __fadd2_rn(xl, yl));
    const float2 h = __fadd2_rn(s, e2);
    xl = __ffma2_rn(__ffma2_rn(s, m1, h), m1, e2);                   // e2 - (h - s)
    xh = h;
}

// ---------------------------------------------------------------------------
// exponent-field helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int biased_exp(double x) { return (__double2hiint(x) >> 20) & 0x7ff; }

// x * 2^k for normal x whose result stays normal, by an integer add to the exponent field.
// Zero stays zero.  (Callers guarantee the range; see the scaled-double invariants.)
__device__ __forceinline__ double exp_shift(double x, int k) {
    int hi = __double2hiint(x);
    int lo = __double2loint(x);
    int nz = (hi & 0x7fffffff) | lo;
    hi += (nz != 0) ? (k << 20) : 0;
    return __hiloint2double(hi, lo);
}

// 2^k as a double for -1022 <= k <= 1023
__device__ __forceinline__ double pow2(int k) { return __hiloint2double((k + 1023) << 20, 0); }

// |x| >= y for y > 0, compared on the bit patterns with the sign bit shifted out.
// (A sign mask here is recognised as fabs and turned into an FP64 instruction, which
// costs a full slot of GB300's narrow FP64 pipe; the shift keeps it on the integer pipe.)
__device__ __forceinline__ bool abs_ge(double x, long long ybits) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) << 1;
    return b >= ((unsigned long long)ybits << 1);
}

// ---------------------------------------------------------------------------
// per-angle quantities (Sec. 4.2.2: cos beta, ln cos(beta/2), ln sin(beta/2))
// ---------------------------------------------------------------------------
struct Angle {
    double cb;    // cos(beta)
    double sb;    // sin(beta)
    double lnc;   // ln cos(beta/2)   (unused when c_zero)
    double lns;   // ln sin(beta/2)   (unused when s_zero)
    bool c_zero;  // beta == pi
    bool s_zero;  // beta == 0
    bool bad;     // beta outside [0, pi] or NaN
};

__device__ __forceinline__ Angle make_angle(double beta) {
    Angle t;
    t.bad = !(beta >= 0.0 && beta <= WG_PI_HI);
    double b = t.bad ? 1.0 : beta;
    double s, c;
    sincos(0.5 * b, &s, &c);
    t.cb = cos(b);
    t.sb = sin(b);
    t.s_zero = (s == 0.0);
    t.c_zero = (c <= 0.0);
    // the logarithm of the half-angle factor closer to 1 through log1p(-x^2)/2 keeps
    // full relative accuracy near the poles
    t.lnc = (c >= s) ? 0.5 * log1p(-s * s) : log(c);
    t.lns = (s >= c) ? 0.5 * log1p(-c * c) : log(s);
    return t;
}

// ---------------------------------------------------------------------------
// constant tables (device pointers, built once per device on the host)
// ---------------------------------------------------------------------------
struct Tables {
    const double *lnf_hi;  // ln n! = lnf_hi[n] + lnf_lo[n], n <= 2*lcap+1
    const double *lnf_lo;
    const double *P;       // P_i = sqrt(1/(i+1)),  i <= 2*lcap+1   (Sec. 4.2.2)
    const double *Q;       // Q_i = sqrt(i/(i+1))
    const double *R1;      // 1/(l(l+1)), l >= 1  (R1[0] = 0)
    const double *R2;      // (l+1)/l,    l >= 1  (R2[0] = 0)
    // float-float copies (hi, lo) for the FP32 form's set-up on the FP32 pipe; may be
    // null for paths that do not use them: ln n!, P_i, Q_i, E (2*lcap+2 each), R1, R2 (lcap+1)
    const float2 *lnf_f;
    const float2 *P_f;
    const float2 *Q_f;
    const float2 *R1_f;
    const float2 *R2_f;
    const float2 *E_f;     // E(n) = ln((n-1)!! / n!!), n <= 2*lcap+1 (FP32 form's sigma)
    int lcap;
    int *status;           // device status word (WG_DEVERR_* bits)
};

// ---------------------------------------------------------------------------
// Seed of a chain (Eqs. ini1-ini2 in log form, Eq. logstart) as a scaled double.
//   l0 = max(mb, ms), m = min(mb, ms)
//   ms >= mb : d^{l0}_{mb,l0} = A c^{l0+mb} s^{l0-mb}
//   mb >  ms : d^{l0}_{l0,ms} = A c^{l0+ms} (-s)^{l0-ms}
//   ln|d| = (ln (2l0)! - ln (l0+m)! - ln (l0-m)!)/2 + (l0+m) ln c + (l0-m) ln s
// evaluated in double-double.  Result: value = mant * 2^(90 n); plain (n = 0,
// mant = the value) when the value is >= 2^-810, else mant in [1, 2^90).
// ---------------------------------------------------------------------------
struct Scaled {
    double mant;
    int n;
    bool plain;
};

// The angle-independent part of ln|d^{l0}|, (ln (2l0)! - ln (l0+m)! - ln (l0-m)!)/2, in
// double-double: one value per chain column, shared by all its angles.
__device__ __forceinline__ dd seed_prefactor(int mb, int ms, const Tables &T) {
    const int l0 = mb > ms ? mb : ms;
    const int m = mb > ms ? ms : mb;
    const int p = l0 + m, q = l0 - m;
    dd x = {T.lnf_hi[2 * l0], T.lnf_lo[2 * l0]};
    x = dd_add(x, dd_neg(dd{T.lnf_hi[p], T.lnf_lo[p]}));
    x = dd_add(x, dd_neg(dd{T.lnf_hi[q], T.lnf_lo[q]}));
    x.hi *= 0.5;  // exact
    x.lo *= 0.5;
    return x;
}

// ln|d^{l0}| of the seed in double-double from the column's prefactor, its sign, and
// whether the value is exactly 0.
__device__ __forceinline__ dd seed_log_from(dd x, int mb, int ms, const Angle &t, double &sign, bool &zero) {
    const int l0 = mb > ms ? mb : ms;
    const int m = mb > ms ? ms : mb;
    const int p = l0 + m, q = l0 - m;
    zero = (p > 0 && t.c_zero) || (q > 0 && t.s_zero);  // a factor is exactly 0 (Sec. 3.2 early stop)
    sign = (mb > ms && (q & 1)) ? -1.0 : 1.0;
    if (p > 0 && !zero) x = dd_add(x, dd_mul_d(dd{t.lnc, 0.0}, (double)p));
    if (q > 0 && !zero) x = dd_add(x, dd_mul_d(dd{t.lns, 0.0}, (double)q));
    return x;
}

// ln|d^{l0}| of the seed in double-double, its sign, and whether the value is exactly 0.
__device__ __forceinline__ dd seed_log(int mb, int ms, const Angle &t, const Tables &T, double &sign, bool &zero) {
    return seed_log_from(seed_prefactor(mb, ms, T), mb, ms, t, sign, zero);
}

// The seed as a scaled double from ln|d^{l0}| (x), its sign and zero flag.
__device__ __forceinline__ Scaled seed_from_log(dd x, double sign, bool zero);

__device__ __forceinline__ Scaled seed_value_from(dd pre, int mb, int ms, const Angle &t) {
    double sign;
    bool zero;
    const dd x = seed_log_from(pre, mb, ms, t, sign, zero);
    return seed_from_log(x, sign, zero);
}

__device__ __forceinline__ Scaled seed_value(int mb, int ms, const Angle &t, const Tables &T) {
    return seed_value_from(seed_prefactor(mb, ms, T), mb, ms, t);
}

__device__ __forceinline__ Scaled seed_from_log(dd x, double sign, bool zero) {
    Scaled r;
    if (zero) {
        r.mant = 0.0;
        r.n = 0;
        r.plain = true;
        return r;
    }
    // split x = k * (90 ln 2) + rem, rem in [0, 90 ln 2)
    double k = floor(x.hi * WG_INV_LN_S);
    dd rem = dd_add(x, dd_mul_d(dd{WG_LN_S_HI, 0.0}, -k));  // k * LN_S_HI is exact (|k| < 2^17)
    rem = dd_add(rem, dd{-k * WG_LN_S_LO, 0.0});
    if (rem.hi < 0.0) {
        k -= 1.0;
        rem = dd_add(dd_add(rem, dd{WG_LN_S_HI, 0.0}), dd{WG_LN_S_LO, 0.0});
    } else if (rem.hi >= WG_LN_S_HI) {
        k += 1.0;
        rem = dd_add(dd_add(rem, dd{-WG_LN_S_HI, 0.0}), dd{-WG_LN_S_LO, 0.0});
    }
    double e = exp(rem.hi);
    double v = __fma_rn(e, rem.lo, e);  // exp(hi + lo) ~ exp(hi)(1 + lo)
    int kk = (int)k;
    if (kk >= WG_PLAIN_MIN_N) {
        r.mant = sign * v * pow2(90 * kk);
        r.n = 0;
        r.plain = true;
    } else {
        r.mant = sign * v;
        r.n = kk;
        r.plain = false;
    }
    return r;
}

// Value of a scaled double as a plain double (rounded; 0 below the double range).
__device__ __forceinline__ double scaled_to_double(double mant, int n) {
    if (n == 0) return mant;
    return scalbn(mant, 90 * n);
}

// The value to store for a chain in scaled mode (n < 0), mant * 2^(90 n), by integer
// arithmetic on the exponent field: no FP64 instruction, so a store that selects between
// the plain and the scaled value costs nothing on the FP64 pipe when the compiler
// evaluates both sides.  Exact while the result is a normal double; a result below
// 2^-1022 (the subnormal range) is stored as 0.
__device__ __forceinline__ double scaled_store(double mant, int n) {
    const int e = biased_exp(mant) + 90 * n;  // the result's biased exponent (0 stays below 1)
    return e >= 1 ? exp_shift(mant, 90 * n) : 0.0;
}

// ---------------------------------------------------------------------------
// Scaled-mode maintenance after a step (integer pipe only, except the one-time
// conversion to plain doubles).  (cur, prev) share the exponent n.
//   |cur| > 2^90  -> both * 2^-90, n += 1
//   0 < |cur| < 2^-90 -> both * 2^90, n -= 1
//   n >= WG_PLAIN_MIN_N (value >= 2^-900)  -> plain doubles from now on (Sec. 3.2)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void scaled_fixup(double &cur, double &prev, int &n, bool &plain) {
    const int e = biased_exp(cur);
    if (e > 1023 + 90) {
        cur = exp_shift(cur, -90);
        prev = exp_shift(prev, -90);
        n += 1;
        if (n >= WG_PLAIN_MIN_N) {
            const double f = pow2(90 * n);  // 2^(90n) >= 2^-810
            cur *= f;
            prev *= f;
            n = 0;
            plain = true;
        }
    } else if (e < 1023 - 90 && e > 0) {
        cur = exp_shift(cur, 90);
        prev = exp_shift(prev, 90);
        n -= 1;
    }
}

// ---------------------------------------------------------------------------
// F0_l, G_l = F0_l F1_l, F2_l for orders (mb, ms) at order l (Sec. 4.2.2):
//   F0 = (l+1)(2l+1) P_{l+mb} P_{l-mb} P_{l+ms} P_{l-ms},  F1 = mb ms / (l(l+1)),
//   F2 = Q_{l+mb} Q_{l-mb} Q_{l+ms} Q_{l-ms} (l+1)/l
// so that Eq. lrec reads d^{l+1} = (F0 cos(beta) - G) d^l - F2 d^{l-1}.
// Requires l >= max(mb, ms); at l = 0 and at l = max(mb, ms) the F2 factor is 0.
// ---------------------------------------------------------------------------
// k as a double, exact for 0 <= k < 2^53, by integer operations on the bits (no
// conversion instruction on the FP64 pipe)
__device__ __forceinline__ double exact_double(long long k) {
    if (k <= 0) return 0.0;
    const int e = 63 - __clzll(k);
    const unsigned long long m = ((unsigned long long)k << (52 - e)) & 0xFFFFFFFFFFFFFull;
    return __longlong_as_double((long long)(((unsigned long long)(1023 + e) << 52) | m));
}

__device__ __forceinline__ void lrec_coefficients(int l, int mb, int ms, const Tables &T, double &f0,
                                                  double &g, double &f2) {
    const double pp = (T.P[l + mb] * T.P[l - mb]) * (T.P[l + ms] * T.P[l - ms]);
    const double qq = (T.Q[l + mb] * T.Q[l - mb]) * (T.Q[l + ms] * T.Q[l - ms]);
    // (l+1)(2l+1) and mb ms are exact integers, so these are the products
    // ((double)(l+1) (double)(2l+1)) pp and ((double)mb (double)ms) R1_l, bit for bit
    f0 = exact_double((long long)(l + 1) * (long long)(2 * l + 1)) * pp;
    g = f0 * (exact_double((long long)mb * (long long)ms) * T.R1[l]);
    f2 = T.R2[l] * qq;
}

// ---------------------------------------------------------------------------
// status word
// ---------------------------------------------------------------------------
__device__ __forceinline__ void raise_status(int *status, int bit) {
    if (status) atomicOr(status, bit);
}

}  // namespace wg
