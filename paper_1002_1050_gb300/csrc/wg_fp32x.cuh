// wg_fp32x.cu -- the FP32 form: recursion body in float with an int32 exponent carry.
//
// Precision design (see the FP32 accuracy study recorded with the project):
//  * Seeds (Eqs. ini1-ini2, logstart) in double-double, split into a float mantissa
//    and an int32 count n of factors 2^64:  value = mant * 2^(64 n).
//  * The coefficient tables of Sec. 4.2.2 (F0, F0*F1, F2) are built in double and
//    combined, still in double, into the coefficients of a difference form of
//    Eq. lrec before rounding to float:
//        Delta_{l+1} = F2_l Delta_l + (K_l - 2 F0_l x^2) d^l,   d^{l+1} = d^l + Delta_{l+1},
//    with Delta_l = d^l - d^{l-1}, x^2 = sin^2(beta/2), K_l = F0_l (1 - F1_l) - 1 - F2_l.
//    Straight float recursion loses all accuracy near the poles (cos beta rounds to
//    1 and the two roots of the recursion merge); in this form the small quantities
//    (x^2, K_l) carry their own relative precision.  For beta > pi/2 the same form runs
//    on e^l = (-1)^l d^l, which obeys Eq. lrec with cos beta -> -cos beta and
//    F1 -> -F1: x^2 = cos^2(beta/2), K_l = F0_l (1 + F1_l) - 1 - F2_l.
//  * Scaled mode while the value is below 2^-64: mantissa kept in [2^-64, 2^64] by
//    joint rescaling of (d, Delta) on the integer pipe; plain floats after that.
//  * Sum C = sum_l w_l d^l in float: terms go into two per-parity partial sums
//    (even/odd l, so the (-1)^l of the mirrored chains is applied once per tile), and
//    each tile's partials are added into a Neumaier-compensated float accumulator.
//    Terms start with the first plain value (|d| >= 2^-64; the paper's 1e-30 skip
//    drops terms below the FP32 form's resolution anyway).
#pragma once

#include <cuda_runtime.h>

#include "wg_common.cuh"
#include "wg_conv_fp64.cuh"  // flush_counters

namespace wg {

#define WG_LN_S32_HI 0x1.62e42fefa0000p+5     /* 64 ln 2, leading 36 bits */
#define WG_LN_S32_LO 0x1.cf79abc9e3b3ap-34    /* 64 ln 2 - WG_LN_S32_HI   */
#define WG_INV_LN_S32 0.022542110013890053

struct Seed32 {
    float mant;
    int n;  // value = mant * 2^(64 n); n == 0: plain
};

// 64 ln 2 in three floats: HI has 11 significant bits so k * HI is exact for |k| < 2^13
#define WG_LN64F_HI 0x1.62cp+5f
#define WG_LN64F_MID 0x1.217f7ep-6f
#define WG_LN64F_LO (-0x1.c610cap-31f)
#define WG_INV_LN64F 0.022542110013890053f

// Per-angle quantities of the FP32 form (Sec. 4.2.2's precomputation), built once per
// angle per work item: x^2 of the difference form, the mirrored flag, and the
// half-angle logarithms as float-float for the seeds.
struct Angle32 {
    float x2;     // sin^2(beta/2) (beta <= pi/2) or cos^2(beta/2) (mirrored chain)
    bool high;    // beta > pi/2: the chain runs on e^l = (-1)^l d^l
    bool bad;     // beta outside [0, pi] or NaN
    bool c_zero, s_zero;
    ff lnc, lns;  // ln cos(beta/2), ln sin(beta/2)
};

__device__ __forceinline__ ff dbl_ff(double x) {
    const float hi = __double2float_rn(x);
    return ff{hi, __double2float_rn(x - (double)hi)};
}

__device__ __forceinline__ Angle32 make_angle32(double beta) {
    Angle32 t;
    t.bad = !(beta >= 0.0 && beta <= WG_PI_HI);
    const double b = t.bad ? 1.0 : beta;
    double s, c;
    sincos(0.5 * b, &s, &c);
    t.high = c < s;
    t.x2 = __double2float_rn(t.high ? c * c : s * s);
    t.s_zero = (s == 0.0);
    t.c_zero = (c <= 0.0);
    t.lnc = dbl_ff((c >= s) ? 0.5 * log1p(-s * s) : log(c));
    t.lns = dbl_ff((s >= c) ? 0.5 * log1p(-c * c) : log(s));
    return t;
}

// Seed (Eqs. ini1-ini2 in log form, Eq. logstart) in float-float on the FP32 pipe,
// split into a float mantissa and a count n of factors 2^64: value = mant * 2^(64 n).
// The logarithm is good to ~2^-48 relative, the exponential to a few float ulps.
__device__ __forceinline__ Seed32 seed32(int mb, int ms, const Angle32 &t, const Tables &T) {
    const int l0 = mb > ms ? mb : ms;
    const int m = mb > ms ? ms : mb;
    const int p = l0 + m, q = l0 - m;
    Seed32 r;
    if ((p > 0 && t.c_zero) || (q > 0 && t.s_zero)) {
        r.mant = 0.0f;
        r.n = 0;
        return r;
    }
    const float sign = (mb > ms && (q & 1)) ? -1.0f : 1.0f;
    ff x = ff_add(ff_of(T.lnf_f[2 * l0]), ff_neg(ff_of(T.lnf_f[p])));
    x = ff_add(x, ff_neg(ff_of(T.lnf_f[q])));
    x.hi *= 0.5f;
    x.lo *= 0.5f;
    if (p > 0) x = ff_add(x, ff_mul(t.lnc, ff_int(p)));
    if (q > 0) x = ff_add(x, ff_mul(t.lns, ff_int(q)));
    float k = floorf(x.hi * WG_INV_LN64F);
    ff rem = ff_add(x, ff{-k * WG_LN64F_HI, 0.0f});
    rem = ff_add(rem, ff_mul(ff{-k, 0.0f}, ff{WG_LN64F_MID, WG_LN64F_LO}));
    if (rem.hi < 0.0f) {
        k -= 1.0f;
        rem = ff_add(rem, ff{WG_LN64F_HI, 0.0f});
        rem = ff_add(rem, ff{WG_LN64F_MID, WG_LN64F_LO});
    } else if (rem.hi >= WG_LN64F_HI + WG_LN64F_MID) {
        k += 1.0f;
        rem = ff_add(rem, ff{-WG_LN64F_HI, 0.0f});
        rem = ff_add(rem, ff{-WG_LN64F_MID, -WG_LN64F_LO});
    }
    const float e = expf(rem.hi);
    float v = sign * __fmaf_rn(e, rem.lo, e);  // in [1, 2^64)
    int kk = (int)k;
    if (kk >= -1) {  // value >= 2^-64: plain
        v *= (kk == 0) ? 1.0f : 0x1p-64f;
        kk = 0;
    }
    r.mant = v;
    r.n = kk;
    return r;
}

// exponent-field shift of a normal float (zero stays zero)
__device__ __forceinline__ float fexp_shift(float x, int k) {
    int b = __float_as_int(x);
    b += ((b & 0x7fffffff) != 0) ? (k << 23) : 0;
    return __int_as_float(b);
}

// scaled-mode maintenance for the pair (cur, aux) sharing the count n (integer pipe)
__device__ __forceinline__ void fixup32(float &cur, float &aux, int &n) {
    const int e = (__float_as_int(cur) >> 23) & 0xff;
    if (e >= 127 + 64) {
        cur = fexp_shift(cur, -64);
        aux = fexp_shift(aux, -64);
        n += 1;
        if (n == -1) {  // value >= 2^-64: leave scaled mode
            cur *= 0x1p-64f;
            aux *= 0x1p-64f;
            n = 0;
        }
    } else if (e < 127 - 64 && e > 0) {
        cur = fexp_shift(cur, 64);
        aux = fexp_shift(aux, 64);
        n -= 1;
    }
}

struct Tile32 {
    float4 *t;  // (A = -2 F0, F2, K0, K1) per l
    float2 *w;  // (w_re, w_im) per l
};

// Coefficients of the difference form at order l (A = -2 F0, F2, K0, K1), built in
// float-float on the FP32 pipe from the float-float tables and rounded to float:
// K0 = F0 (1 - F1) - 1 - F2 and K1 = F0 (1 + F1) - 1 - F2 are small where the form
// matters and keep their relative precision because the cancellation happens in ff.
__device__ __forceinline__ float4 diff_coefficients(int l, int L, int mb, int ms, const Tables &T) {
    if (l >= L) return make_float4(0.f, 0.f, 0.f, 0.f);
    const ff pp = ff_mul(ff_mul(ff_of(T.P_f[l + mb]), ff_of(T.P_f[l - mb])),
                         ff_mul(ff_of(T.P_f[l + ms]), ff_of(T.P_f[l - ms])));
    const ff qq = ff_mul(ff_mul(ff_of(T.Q_f[l + mb]), ff_of(T.Q_f[l - mb])),
                         ff_mul(ff_of(T.Q_f[l + ms]), ff_of(T.Q_f[l - ms])));
    const ff f0 = ff_mul(ff_int((long long)(l + 1) * (2 * l + 1)), pp);
    const ff g = ff_mul(f0, ff_mul(ff_int((long long)mb * ms), ff_of(T.R1_f[l])));
    const ff f2 = ff_mul(ff_of(T.R2_f[l]), qq);
    const ff base = ff_add(ff_add(f0, ff{-1.0f, 0.0f}), ff_neg(f2));
    const ff k0 = ff_add(base, ff_neg(g));
    const ff k1 = ff_add(base, g);
    return make_float4(-2.0f * f0.hi, f2.hi, __fadd_rn(k0.hi, k0.lo), __fadd_rn(k1.hi, k1.lo));
}

// Neumaier-compensated float accumulation: (s, c) += v
__device__ __forceinline__ void neumaier_add(float &s, float &c, float v) {
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}

// One l-step of CPT chains: term l into the partial of parity PAR, then the
// difference-form step to l+1.  x2s carries x^2 with the sign bit set for mirrored
// chains (beta > pi/2); the sign selects K1 over K0 with one bitwise operation.
// MASKED: some chain of the warp may still be scaled (value < 2^-64); those add no
// term, and a chain whose mantissa leaves [2^-64, 2^64) is rescaled (rarely taken
// branch).  lpl records the l at which a chain turned plain.
template <int CPT, int PAR, bool MASKED>
__device__ __forceinline__ void step32(const float4 tc, const float2 w, const float (&x2s)[CPT], float (&cur)[CPT],
                                       float (&aux)[CPT], int (&nsc)[CPT], int (&lpl)[CPT], int l,
                                       float (&pr)[2][CPT], float (&pi)[2][CPT]) {
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const float cm = (!MASKED || nsc[c] == 0) ? cur[c] : 0.f;
        pr[PAR][c] = fmaf(w.x, cm, pr[PAR][c]);
        pi[PAR][c] = fmaf(w.y, cm, pi[PAR][c]);
        const int hm = __float_as_int(x2s[c]) >> 31;  // all ones for a mirrored chain
        const float kk = __int_as_float((__float_as_int(tc.z) & ~hm) | (__float_as_int(tc.w) & hm));
        const float coef = fmaf(tc.x, fabsf(x2s[c]), kk);
        aux[c] = fmaf(tc.y, aux[c], coef * cur[c]);
        cur[c] = cur[c] + aux[c];
        if (MASKED) {
            const int e = (__float_as_int(cur[c]) >> 23) & 0xff;
            if (nsc[c] != 0 && (unsigned)(e - 63) > 127u) {
                fixup32(cur[c], aux[c], nsc[c]);
                if (nsc[c] == 0) lpl[c] = l + 1;
            }
        }
    }
}

template <int TL>
struct SmemFp32 {
    float4 sT[TL];
    float2 sW[TL];
};

// One work item of the FP32 form: chain columns k in [k_begin, k_end) (m_sky-major
// order) for the angle chunk `chunk` (NT*CPT angles).  Every thread of the CTA calls it.
template <int NT, int CPT, int TL>
__device__ __forceinline__ void conv_fp32x_item(const ConvArgs &A, const Tables &T, int chunk, int k_begin,
                                                int k_end, SmemFp32<TL> &sm, unsigned long long &n_elem,
                                                unsigned long long &n_sum) {
    static_assert(TL % 2 == 0, "tile length must be even (parity of l is tracked per tile)");
    const int MB1 = A.mb_max + 1;
    const int L = A.l_max;
    const int NB = A.n_beta;
    const int tid = threadIdx.x;
    float4 *sT = sm.sT;
    float2 *sW = sm.sW;

    int jj[CPT];
    bool valid[CPT], high[CPT], bad[CPT];
    float x2s[CPT];
    Angle32 ang[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        jj[c] = chunk * NT * CPT + c * NT + tid;
        valid[c] = jj[c] < NB;
        ang[c] = make_angle32(valid[c] ? A.beta[jj[c]] : 1.0);
        bad[c] = ang[c].bad;
        if (valid[c] && bad[c]) raise_status(T.status, WG_DEVERR_BETA);
        high[c] = ang[c].high;
        x2s[c] = high[c] ? -ang[c].x2 : ang[c].x2;
    }

    for (int k = k_begin; k < k_end; ++k) {
        const int ms = k / MB1, mb = k - ms * MB1;
        const int l0 = mb > ms ? mb : ms;

        float cur[CPT], aux[CPT], pr[2][CPT], pi[2][CPT], sr[CPT], cr[CPT], si[CPT], ci[CPT];
        int nsc[CPT], lpl[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const Seed32 s = seed32(mb, ms, ang[c], T);
            // mirrored chains start from e^{l0} = (-1)^{l0} d^{l0}
            cur[c] = (high[c] && (l0 & 1)) ? -s.mant : s.mant;
            aux[c] = cur[c];  // Delta_{l0} = d^{l0} - d^{l0-1} = d^{l0}
            nsc[c] = s.n;
            lpl[c] = (s.n == 0) ? l0 : L + 1;
            sr[c] = cr[c] = si[c] = ci[c] = 0.f;
        }
        bool warp_plain = false;

        for (int ts = l0; ts <= L; ts += TL) {
            __syncthreads();
            for (int i = tid; i < TL; i += NT) {
                const int l = ts + i;
                float2 w = make_float2(0.f, 0.f);
                if (l <= L) {
                    const double2 av = reinterpret_cast<const double2 *>(A.a)[(size_t)l * (A.ms_max + 1) + ms];
                    const double2 bv = reinterpret_cast<const double2 *>(A.b)[(size_t)l * MB1 + mb];
                    const float ar = d2f_trunc(av.x), ai = d2f_trunc(av.y);
                    const float br = d2f_trunc(bv.x), bi = d2f_trunc(bv.y);
                    w = make_float2(__fmaf_rn(br, ar, bi * ai), __fmaf_rn(br, ai, -(bi * ar)));
                }
                sT[i] = (l <= L) ? diff_coefficients(l, L, mb, ms, T) : make_float4(0.f, 0.f, 0.f, 0.f);
                sW[i] = w;
            }
            __syncthreads();
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                pr[0][c] = pr[1][c] = pi[0][c] = pi[1][c] = 0.f;
            }
            const int nl = min(TL, L + 1 - ts);
            if (!warp_plain) {
                bool p = true;
#pragma unroll
                for (int c = 0; c < CPT; ++c) p = p && (nsc[c] == 0);
                warp_plain = __all_sync(0xffffffffu, p);
            }
            int i = 0;
            if (warp_plain) {  // every chain of the warp is a plain float from here on
                for (; i + 1 < nl; i += 2) {
                    step32<CPT, 0, false>(sT[i], sW[i], x2s, cur, aux, nsc, lpl, ts + i, pr, pi);
                    step32<CPT, 1, false>(sT[i + 1], sW[i + 1], x2s, cur, aux, nsc, lpl, ts + i + 1, pr, pi);
                }
                if (i < nl) step32<CPT, 0, false>(sT[i], sW[i], x2s, cur, aux, nsc, lpl, ts + i, pr, pi);
            } else {
                for (; i + 1 < nl; i += 2) {
                    step32<CPT, 0, true>(sT[i], sW[i], x2s, cur, aux, nsc, lpl, ts + i, pr, pi);
                    step32<CPT, 1, true>(sT[i + 1], sW[i + 1], x2s, cur, aux, nsc, lpl, ts + i + 1, pr, pi);
                }
                if (i < nl) step32<CPT, 0, true>(sT[i], sW[i], x2s, cur, aux, nsc, lpl, ts + i, pr, pi);
            }
            // partials of this tile into the compensated accumulators; the sign of the
            // odd-offset partial is (-1) for mirrored chains, and the tile's start parity
            // (that of l0, as TL is even) is applied at the end
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const float sg = high[c] ? -1.f : 1.f;
                neumaier_add(sr[c], cr[c], pr[0][c] + sg * pr[1][c]);
                neumaier_add(si[c], ci[c], pi[0][c] + sg * pi[1][c]);
            }
        }
        double2 *out = reinterpret_cast<double2 *>(A.c_out) + ((size_t)mb * (A.ms_max + 1) + ms) * NB;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            if (valid[c]) {
                const double sg = (high[c] && (l0 & 1)) ? -1.0 : 1.0;
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                const double re = sg * ((double)sr[c] + (double)cr[c]);
                const double im = sg * ((double)si[c] + (double)ci[c]);
                out[jj[c]] = bad[c] ? make_double2(nan, nan) : make_double2(re, im);
                n_elem += (unsigned long long)(L + 1 - l0);
                n_sum += (unsigned long long)(L + 1 - min(lpl[c], L + 1));
            }
        }
    }
}

}  // namespace wg
