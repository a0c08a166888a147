// wg_fp32x.cuh -- the FP32 form: recursion body in float with an int32 exponent carry.
//
// Precision design:
//  * Seeds (Eqs. ini1-ini2, logstart) in float-float on the FP32 pipe from float-float
//    tables of ln n! and per-angle half-angle logarithms, split into a float mantissa
//    and an int32 count n of factors 2^64:  value = mant * 2^(64 n).
//  * The coefficients of Sec. 4.2.2 (F0, F0*F1, F2) are built in float-float from the
//    float-float tables P, Q, 1/(l(l+1)), (l+1)/l and combined, still in float-float,
//    into the coefficients of a difference form of Eq. lrec before rounding to float:
//        Delta_{l+1} = F2_l Delta_l + (K_l - 2 F0_l x^2) d^l,   d^{l+1} = d^l + Delta_{l+1},
//    with Delta_l = d^l - d^{l-1}, x^2 = sin^2(beta/2), K_l = F0_l (1 - F1_l) - 1 - F2_l.
//    Straight float recursion loses all accuracy near the poles (cos beta rounds to
//    1 and the two roots of the recursion merge); in this form the small quantities
//    (x^2, K_l) carry their own relative precision.  For beta > pi/2 the same form runs
//    on e^l = (-1)^l d^l, which obeys Eq. lrec with cos beta -> -cos beta and
//    F1 -> -F1: x^2 = cos^2(beta/2), K_l = F0_l (1 + F1_l) - 1 - F2_l.
//  * Scaled mode while the value is below 2^-64: every fourth step the pair (d, Delta)
//    is scaled jointly by 2^-64 or 2^64 when the mantissa has left [2^-64, 2^64); a
//    chain whose value has reached 2^-64 turns into a plain float at the next l-tile.
//    A warp whose chains are all plain runs the step without any of this.
//  * Sum C = sum_l w_l d^l in float: terms go into two per-parity partial sums
//    (even/odd l, so the (-1)^l of the mirrored chains is applied once per tile), and
//    each tile's partials are added into a Neumaier-compensated float accumulator.
//    Terms start once the value reaches 2^-128 (below it their factor 2^(64 n) is 0;
//    the paper's 1e-30 skip of Sec. 4.2.1 drops terms below the FP32 form's resolution
//    anyway), and a warp whose chains are all below it steps without the sum.
#pragma once

#include <cuda_runtime.h>

#include "wg_common.cuh"
#include "wg_conv_fp64.cuh"  // flush_counters

namespace wg {

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
    float cb;     // cos(beta)
    float sb;     // sin(beta)
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
    t.cb = __double2float_rn((c - s) * (c + s));
    t.sb = __double2float_rn(2.0 * s * c);
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

// Coefficients of the difference form at order l (A = -2 F0, F2, K0, K1), built in
// float-float on the FP32 pipe from the float-float tables and rounded to float:
// K0 = F0 (1 - F1) - 1 - F2 and K1 = F0 (1 + F1) - 1 - F2 are small where the form
// matters and keep their relative precision because the cancellation happens in ff.
// F0 and G = F0 F1 of Eq. lrec at order l < l_max in float-float (Sec. 4.2.2's tables)
__device__ __forceinline__ void f0g_ff(int l, int mb, int ms, const Tables &T, ff &f0, ff &g) {
    const ff pp = ff_mul(ff_mul(ff_of(T.P_f[l + mb]), ff_of(T.P_f[l - mb])),
                         ff_mul(ff_of(T.P_f[l + ms]), ff_of(T.P_f[l - ms])));
    f0 = ff_mul(ff_int((long long)(l + 1) * (2 * l + 1)), pp);
    g = ff_mul(f0, ff_mul(ff_int((long long)mb * ms), ff_of(T.R1_f[l])));
}

__device__ __forceinline__ float4 diff_coefficients(int l, int L, int mb, int ms, const Tables &T, float4 &raw) {
    if (l >= L) {
        raw = make_float4(0.f, 0.f, 1.f, 0.f);
        return make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const ff qq = ff_mul(ff_mul(ff_of(T.Q_f[l + mb]), ff_of(T.Q_f[l - mb])),
                         ff_mul(ff_of(T.Q_f[l + ms]), ff_of(T.Q_f[l - ms])));
    ff f0, g;
    f0g_ff(l, mb, ms, T, f0, g);
    const ff f2 = ff_mul(ff_of(T.R2_f[l]), qq);
    const ff base = ff_add(ff_add(f0, ff{-1.0f, 0.0f}), ff_neg(f2));
    const ff k0 = ff_add(base, ff_neg(g));
    const ff k1 = ff_add(base, g);
    raw = make_float4(f0.hi, g.hi, f2.hi, f2.lo);  // F0, G = F0 F1, F2 (float-float)
    return make_float4(-2.0f * f0.hi, f2.hi, __fadd_rn(k0.hi, k0.lo), __fadd_rn(k1.hi, k1.lo));
}

// Neumaier-compensated float accumulation: (s, c) += v
__device__ __forceinline__ void neumaier_add(float &s, float &c, float v) {
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}

// The chains of a thread are processed in pairs with the packed two-lane float
// instructions of sm_100+ (__ffma2_rn, __fmul2_rn, __fadd2_rn: per component the same
// IEEE operation as fmaf, *, +), so one instruction advances two chains.  The per-l
// operands are stored duplicated in shared memory, (A, A, F2, F2), (K0, K0, K1, K1),
// (w_re, w_re, w_im, w_im), and reach the pair as 64-bit register pairs.

// One l-step of the NP chain pairs: term l into the partial of parity PAR, then the
// difference-form step to l+1.  kp[p]: the K coefficient of each chain of pair p (K0,
// or K1 for a mirrored chain).  MASKED: some chain of the warp is still scaled; its term
// is cur * sp, where sp = 2^(64 n) for the count n of 2^64 factors (1 for a plain chain,
// 2^-64 for n = -1, 0 below: those terms are < 2^-64 |w|).
template <int NP, int PAR, bool MASKED>
__device__ __forceinline__ void step_pairs(const float4 a4, const float2 (&kp)[NP], const float4 w4,
                                           const float2 (&x2p)[NP], float2 (&cur)[NP], float2 (&aux)[NP],
                                           const float2 (&sp)[NP], float2 (&pr)[2][NP], float2 (&pi)[2][NP]) {
    const float2 A = make_float2(a4.x, a4.y), F2 = make_float2(a4.z, a4.w);
    const float2 WR = make_float2(w4.x, w4.y), WI = make_float2(w4.z, w4.w);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 cm = MASKED ? __fmul2_rn(cur[p], sp[p]) : cur[p];
        pr[PAR][p] = __ffma2_rn(WR, cm, pr[PAR][p]);
        pi[PAR][p] = __ffma2_rn(WI, cm, pi[PAR][p]);
        const float2 coef = __ffma2_rn(A, x2p[p], kp[p]);
        aux[p] = __ffma2_rn(F2, aux[p], __fmul2_rn(coef, cur[p]));
        cur[p] = __fadd2_rn(cur[p], aux[p]);
    }
}

// The difference-form step without its term, for warps whose chains are all below
// 2^-128 (sp = 0: their terms are zero)
template <int NP>
__device__ __forceinline__ void step_pairs_rec(const float4 a4, const float2 (&kp)[NP], const float2 (&x2p)[NP],
                                               float2 (&cur)[NP], float2 (&aux)[NP]) {
    const float2 A = make_float2(a4.x, a4.y), F2 = make_float2(a4.z, a4.w);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 coef = __ffma2_rn(A, x2p[p], kp[p]);
        aux[p] = __ffma2_rn(F2, aux[p], __fmul2_rn(coef, cur[p]));
        cur[p] = __fadd2_rn(cur[p], aux[p]);
    }
}

// whether some chain of the warp has a non-zero term factor sp (warp-uniform)
template <int NP>
__device__ __forceinline__ bool warp_terms_live(const float2 (&sp)[NP]) {
    bool any = false;
#pragma unroll
    for (int p = 0; p < NP; ++p) any = any || sp[p].x != 0.0f || sp[p].y != 0.0f;
    return __any_sync(0xffffffffu, any);
}

// Rescaling of one scaled chain, run every 4 or 8 steps of a masked tile: a mantissa at
// or above 2^64 is scaled by 2^-64 (n += 1), one of a scaled chain below 2^-64 by 2^64
// (n -= 1), jointly with aux; then sp = 2^(64 n) (0 for n <= -2).  No branch.  Between
// two calls the mantissa changes by less than 2^60: the ratio of consecutive values is
// at most |F0 (cos b - F1)| + 1 <= 2 (l0 + 1) / (k + 1) + 1 at l = l0 + k (largest for
// m_b = m_sky = l0; 4 (l0 + 1) / (k + 1) + 1 in the normalised form, whose rho <= 2),
// so four steps from any l0 <= 32767 grow it by at most 2^64 / 24, eight steps by at
// most 181^8 < 2^60 once k >= (l0 + 1) / 45, and sixteen steps of the normalised form by
// at most 13^16 < 2^60 once k >= (l0 + 1) / 3 (rescale_period; the difference form keeps
// groups of at most 8); a mantissa left in [2^-64, 2^64) stays a normal float.
__host__ __device__ __forceinline__ int rescale_period(int l0, int k) {
    return 3 * k >= l0 + 1 ? 16 : (45 * k >= l0 + 1 ? 8 : 4);
}
__device__ __forceinline__ void rescale32(float &cur, float &aux, int &n, float &sp) {
    const float m = fabsf(cur);
    const bool dn = m >= 0x1p64f;
    const bool up = (m < 0x1p-64f) && (n != 0);
    const float f = dn ? 0x1p-64f : (up ? 0x1p64f : 1.0f);
    cur *= f;
    aux *= f;
    n += (int)dn - (int)up;
    sp = __int_as_float(max(0, 127 + 64 * n) << 23);
}

template <int NP>
__device__ __forceinline__ void rescale_pairs(float2 (&cur)[NP], float2 (&aux)[NP], int (&nsc)[2 * NP],
                                              float2 (&sp)[NP]) {
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        rescale32(cur[p].x, aux[p].x, nsc[2 * p], sp[p].x);
        rescale32(cur[p].y, aux[p].y, nsc[2 * p + 1], sp[p].y);
    }
}

// the normalised step without its term (a warp whose chains are all below 2^-128)
template <int NP>
__device__ __forceinline__ void step_norm_rec(const float4 n4, const float2 (&cbp)[NP], float2 (&u)[NP],
                                              float2 (&up)[NP]) {
    const float2 F = make_float2(n4.x, n4.y), NG = make_float2(n4.z, n4.w);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 y = __ffma2_rn(F, cbp[p], NG);
        const float2 nx = __ffma2_rn(y, u[p], up[p]);
        up[p] = u[p];
        u[p] = nx;
    }
}

// One l-step of the NP chain pairs in the normalised form (bulk angles): with u^l =
// d^l / sigma_l (sigma_{l0} = sigma_{l0+1} = 1, sigma_{l+1} = F2_l sigma_{l-1}), Eq. lrec
// reads u^{l+1} = (F0'_l cos b - G'_l) u^l - u^{l-1}, F0' = F0 rho_l, G' = G rho_l,
// rho_l = sigma_l / sigma_{l+1}; the chain is carried as v^l = s_k u^l, s_k = +1, +1,
// -1, -1, ... for k = l - l0, which obeys v^{l+1} = (-1)^k (F0'_l cos b - G'_l) v^l +
// v^{l-1}: two packed FMAs per pair for the recursion, two for the sum of (w_l sigma_l
// s_k) v^l.  n4 = (-1)^k (F0', F0', -G', -G'), w4 = (w sigma s)(re, re, im, im).
template <int NP, int PAR, bool MASKED>
__device__ __forceinline__ void step_norm(const float4 n4, const float4 w4, const float2 (&cbp)[NP],
                                          float2 (&u)[NP], float2 (&up)[NP], const float2 (&sp)[NP],
                                          float2 (&pr)[2][NP], float2 (&pi)[2][NP]) {
    const float2 F = make_float2(n4.x, n4.y), NG = make_float2(n4.z, n4.w);
    const float2 WR = make_float2(w4.x, w4.y), WI = make_float2(w4.z, w4.w);
#pragma unroll
    for (int p = 0; p < NP; ++p) {
        const float2 cm = MASKED ? __fmul2_rn(u[p], sp[p]) : u[p];
        pr[PAR][p] = __ffma2_rn(WR, cm, pr[PAR][p]);
        pi[PAR][p] = __ffma2_rn(WI, cm, pi[PAR][p]);
        const float2 y = __ffma2_rn(F, cbp[p], NG);
        const float2 nx = __ffma2_rn(y, u[p], up[p]);
        up[p] = u[p];
        u[p] = nx;
    }
}

// Shared memory of one FP32-form CTA: two buffers of each form's l-tile operands (the
// tile after the current one is built while other warps still step the current one),
// and the per-chain state that is touched once per column or per tile (kept out of
// registers so that more warps fit on an SM): the seeds' half-angle logarithms and
// flags, and the Neumaier-compensated sums.
template <int NT, int CPT, int TL>
struct SmemFp32 {
    float4 sA[2][TL];       // difference form: (A, A, F2, F2), A = -2 F0
    float4 sK[2][TL];       // (K0, K0, K1, K1)
    float4 sW[2][TL];       // (w_re, w_re, w_im, w_im)
    float4 sN[2][TL];       // normalised form: (F0', F0', -G', -G')
    float4 sWn[2][TL];      // (w sigma s)(re, re, im, im)
    float4 sKc;             // the column's S(l0), S(l0 + 1) (float-float; see sigma_log)
    float4 sLog[CPT][NT];   // (ln cos(b/2) hi, lo, ln sin(b/2) hi, lo)
    int sFlag[CPT][NT];     // bit 0: bad angle, 1: mirrored, 2: cos(b/2) = 0, 3: sin(b/2) = 0
    float4 sAcc[CPT][NT];   // compensated sums (re, re carry, im, im carry)
};

// The normalisation sigma of the normalised form in closed form.  sigma_{l0} =
// sigma_{l0+1} = 1 and sigma_{l+1} = F2_l sigma_{l-1}; with h_l = sqrt((l^2 - mb^2)(l^2 -
// ms^2)) / l, Eq. lrec's F2_l = h_l / h_{l+1}, so along each parity of l the product
// telescopes into alternating logarithms of h, and those of each factor l +- m of h
// into logarithms of double factorials: ln sigma_l = S(l) - S(l0 + ((l - l0) & 1)) with
//   S(n) = (E(n - mb) + E(n + mb) + E(n - ms) + E(n + ms)) / 2 - E(n),
//   E(n) = ln((n-1)!! / n!!)   (a host table, float-float).
// Each entry of a tile is then independent of the others (no scan along l).
__device__ __forceinline__ ff sigma_log(int n, int mb, int ms, const float2 *E) {
    ff s = ff_add(ff_add(ff_of(E[n - mb]), ff_of(E[n + mb])), ff_add(ff_of(E[n - ms]), ff_of(E[n + ms])));
    s.hi *= 0.5f;
    s.lo *= 0.5f;
    return ff_add(s, ff_neg(ff_of(E[n])));
}

// e^x of a float-float argument, to float accuracy
__device__ __forceinline__ float ff_expf(ff x) {
    const float e = expf(x.hi);
    return __fmaf_rn(e, x.lo, e);
}

// The operands of the l-tile starting at order ts into buffer buf, for the forms in use
// (need_diff, need_norm: CTA-uniform).  Warp w builds entries 31 w + lane (lane < 31);
// each lane also forms S(l) of its order for the normalised form, and takes S(l+1)
// from the next lane (lane 31 forms the first order of the next warp's entries).
// sm.sKc holds S(l0) and S(l0 + 1).  F0 = G = 0 from l_max on (the chain's last step is
// never used).
template <int NT, int CPT, int TL>
__device__ __forceinline__ void build_tile(const ConvArgs &A, const Tables &T, int ts, int l0, int mb, int ms,
                                           bool need_diff, bool need_norm, SmemFp32<NT, CPT, TL> &sm, int buf) {
    constexpr int PER = 31 * (NT / 32);
    const int L = A.l_max, MB1 = A.mb_max + 1;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < TL; base += PER) {
        const int i = base + 31 * w + lane;
        const int l = ts + i;
        ff s{0.0f, 0.0f};
        if (need_norm && i <= TL && l <= L + 1) s = sigma_log(l, mb, ms, T.E_f);
        const ff sn{__shfl_down_sync(0xffffffffu, s.hi, 1), __shfl_down_sync(0xffffffffu, s.lo, 1)};
        if (lane == 31 || i >= TL || l > L) continue;
        const double2 av = reinterpret_cast<const double2 *>(A.a)[(size_t)l * (A.ms_max + 1) + ms];
        const double2 bv = reinterpret_cast<const double2 *>(A.b)[(size_t)l * MB1 + mb];
        const int sa = A.ea ? A.ea[ms] : 0, sb = A.eb ? A.eb[mb] : 0;
        const float ar = d2f_rn_scaled(av.x, sa), ai = d2f_rn_scaled(av.y, sa);
        const float br = d2f_rn_scaled(bv.x, sb), bi = d2f_rn_scaled(bv.y, sb);
        const float wr = __fmaf_rn(br, ar, bi * ai), wi = __fmaf_rn(br, ai, -(bi * ar));
        float f0 = 0.0f, g = 0.0f;
        if (need_diff) {
            float4 raw;
            const float4 c = diff_coefficients(l, L, mb, ms, T, raw);
            sm.sA[buf][i] = make_float4(c.x, c.x, c.y, c.y);
            sm.sK[buf][i] = make_float4(c.z, c.z, c.w, c.w);
            sm.sW[buf][i] = make_float4(wr, wr, wi, wi);
            f0 = raw.x;
            g = raw.y;
        } else if (l < L) {
            ff f0f, gf;
            f0g_ff(l, mb, ms, T, f0f, gf);
            f0 = f0f.hi;
            g = gf.hi;
        }
        if (need_norm) {
            const float4 kc = sm.sKc;
            const int k = l - l0;
            const ff ke{(k & 1) ? kc.z : kc.x, (k & 1) ? kc.w : kc.y}, ko{(k & 1) ? kc.x : kc.z, (k & 1) ? kc.y : kc.w};
            const ff ls = ff_add(s, ff_neg(ke));
            const ff lsn = ff_add(sn, ff_neg(ko));
            const float sig = ff_expf(ls);                      // sigma_l
            const float rho = ff_expf(ff_add(ls, ff_neg(lsn)));  // sigma_l / sigma_{l+1}
            // the chain is carried as v = s_k u with s_k = +1, +1, -1, -1, ... (k = l - l0):
            // v^{l+1} = (-1)^k y_l v^l + v^{l-1}, so the step takes no negation, and
            // d^l = sigma_l s_k v^l
            const float f0p = ((k & 1) ? -f0 : f0) * rho, gp = ((k & 1) ? -g : g) * rho;
            const float ws = (k & 2) ? -sig : sig;
            sm.sN[buf][i] = make_float4(f0p, f0p, -gp, -gp);
            sm.sWn[buf][i] = make_float4(wr * ws, wr * ws, wi * ws, wi * ws);
        }
    }
}

// the K pair of each chain pair at tile entry i: the thread's common K (UNIFORM: all its
// chains on the same side of pi/2) or each chain's own (bit c of hbits: chain c is
// mirrored and takes K1, at index 2 of (K0, K0, K1, K1))
template <int NP, bool UNIFORM>
__device__ __forceinline__ void k_pairs(const float4 &k4, int thigh, int hbits, float2 (&kp)[NP]) {
    if (UNIFORM) {
        const float2 k = reinterpret_cast<const float2 *>(&k4)[thigh];
#pragma unroll
        for (int p = 0; p < NP; ++p) kp[p] = k;
    } else {
        const float *kq = reinterpret_cast<const float *>(&k4);
#pragma unroll
        for (int p = 0; p < NP; ++p)
            kp[p] = make_float2(kq[((hbits >> (2 * p)) & 1) << 1], kq[((hbits >> (2 * p + 1)) & 1) << 1]);
    }
}

// The steps of one l-tile (nl orders) in the difference form for every chain of the thread.
template <int NP, int TL, bool UNIFORM>
__device__ __forceinline__ void tile_steps(const float4 *sA, const float4 *sK, const float4 *sW, int nl, bool plain,
                                           int period, int thigh, int hbits, const float2 (&x2p)[NP],
                                           float2 (&cur)[NP], float2 (&aux)[NP], int (&nsc)[2 * NP],
                                           float2 (&sp)[NP], float2 (&pr)[2][NP], float2 (&pi)[2][NP]) {
    float2 kp[NP];
    int i = 0;
    if (plain) {  // every chain of the warp is a plain float
        for (; i + 1 < nl; i += 2) {
            k_pairs<NP, UNIFORM>(sK[i], thigh, hbits, kp);
            step_pairs<NP, 0, false>(sA[i], kp, sW[i], x2p, cur, aux, sp, pr, pi);
            k_pairs<NP, UNIFORM>(sK[i + 1], thigh, hbits, kp);
            step_pairs<NP, 1, false>(sA[i + 1], kp, sW[i + 1], x2p, cur, aux, sp, pr, pi);
        }
        if (i < nl) {
            k_pairs<NP, UNIFORM>(sK[i], thigh, hbits, kp);
            step_pairs<NP, 0, false>(sA[i], kp, sW[i], x2p, cur, aux, sp, pr, pi);
        }
    } else {
        // groups of 8 steps between rescales where rescale_period allows, else of 4
        if (period >= 8) {
            for (; i + 7 < nl; i += 8) {
                if (warp_terms_live(sp)) {
#pragma unroll
                    for (int q = 0; q < 8; q += 2) {
                        k_pairs<NP, UNIFORM>(sK[i + q], thigh, hbits, kp);
                        step_pairs<NP, 0, true>(sA[i + q], kp, sW[i + q], x2p, cur, aux, sp, pr, pi);
                        k_pairs<NP, UNIFORM>(sK[i + q + 1], thigh, hbits, kp);
                        step_pairs<NP, 1, true>(sA[i + q + 1], kp, sW[i + q + 1], x2p, cur, aux, sp, pr, pi);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        k_pairs<NP, UNIFORM>(sK[i + q], thigh, hbits, kp);
                        step_pairs_rec<NP>(sA[i + q], kp, x2p, cur, aux);
                    }
                }
                rescale_pairs(cur, aux, nsc, sp);
            }
        }
        for (; i + 3 < nl; i += 4) {
            if (warp_terms_live(sp)) {
#pragma unroll
                for (int q = 0; q < 4; q += 2) {
                    k_pairs<NP, UNIFORM>(sK[i + q], thigh, hbits, kp);
                    step_pairs<NP, 0, true>(sA[i + q], kp, sW[i + q], x2p, cur, aux, sp, pr, pi);
                    k_pairs<NP, UNIFORM>(sK[i + q + 1], thigh, hbits, kp);
                    step_pairs<NP, 1, true>(sA[i + q + 1], kp, sW[i + q + 1], x2p, cur, aux, sp, pr, pi);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    k_pairs<NP, UNIFORM>(sK[i + q], thigh, hbits, kp);
                    step_pairs_rec<NP>(sA[i + q], kp, x2p, cur, aux);
                }
            }
            rescale_pairs(cur, aux, nsc, sp);
        }
        if (i < nl) {
            k_pairs<NP, UNIFORM>(sK[i], thigh, hbits, kp);
            step_pairs<NP, 0, true>(sA[i], kp, sW[i], x2p, cur, aux, sp, pr, pi);
            if (i + 1 < nl) {
                k_pairs<NP, UNIFORM>(sK[i + 1], thigh, hbits, kp);
                step_pairs<NP, 1, true>(sA[i + 1], kp, sW[i + 1], x2p, cur, aux, sp, pr, pi);
            }
            if (i + 2 < nl) {
                k_pairs<NP, UNIFORM>(sK[i + 2], thigh, hbits, kp);
                step_pairs<NP, 0, true>(sA[i + 2], kp, sW[i + 2], x2p, cur, aux, sp, pr, pi);
            }
            rescale_pairs(cur, aux, nsc, sp);
        }
    }
}

// The steps of one l-tile in the normalised form ((cur, aux) hold (u^l, u^{l-1})).
template <int NP, int TL>
__device__ __forceinline__ void tile_steps_norm(const float4 *sN, const float4 *sWn, int nl, bool plain, int period,
                                                const float2 (&cbp)[NP], float2 (&cur)[NP], float2 (&aux)[NP],
                                                int (&nsc)[2 * NP], float2 (&sp)[NP], float2 (&pr)[2][NP],
                                                float2 (&pi)[2][NP]) {
    int i = 0;
    if (plain) {
        for (; i + 1 < nl; i += 2) {
            step_norm<NP, 0, false>(sN[i], sWn[i], cbp, cur, aux, sp, pr, pi);
            step_norm<NP, 1, false>(sN[i + 1], sWn[i + 1], cbp, cur, aux, sp, pr, pi);
        }
        if (i < nl) step_norm<NP, 0, false>(sN[i], sWn[i], cbp, cur, aux, sp, pr, pi);
    } else {
        if (period == 16) {
            for (; i + 15 < nl; i += 16) {
                if (warp_terms_live(sp)) {
#pragma unroll
                    for (int q = 0; q < 16; q += 2) {
                        step_norm<NP, 0, true>(sN[i + q], sWn[i + q], cbp, cur, aux, sp, pr, pi);
                        step_norm<NP, 1, true>(sN[i + q + 1], sWn[i + q + 1], cbp, cur, aux, sp, pr, pi);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) step_norm_rec<NP>(sN[i + q], cbp, cur, aux);
                }
                rescale_pairs(cur, aux, nsc, sp);
            }
        }
        if (period >= 8) {
            for (; i + 7 < nl; i += 8) {
                if (warp_terms_live(sp)) {
#pragma unroll
                    for (int q = 0; q < 8; q += 2) {
                        step_norm<NP, 0, true>(sN[i + q], sWn[i + q], cbp, cur, aux, sp, pr, pi);
                        step_norm<NP, 1, true>(sN[i + q + 1], sWn[i + q + 1], cbp, cur, aux, sp, pr, pi);
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) step_norm_rec<NP>(sN[i + q], cbp, cur, aux);
                }
                rescale_pairs(cur, aux, nsc, sp);
            }
        }
        for (; i + 3 < nl; i += 4) {
            if (warp_terms_live(sp)) {
#pragma unroll
                for (int q = 0; q < 4; q += 2) {
                    step_norm<NP, 0, true>(sN[i + q], sWn[i + q], cbp, cur, aux, sp, pr, pi);
                    step_norm<NP, 1, true>(sN[i + q + 1], sWn[i + q + 1], cbp, cur, aux, sp, pr, pi);
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q) step_norm_rec<NP>(sN[i + q], cbp, cur, aux);
            }
            rescale_pairs(cur, aux, nsc, sp);
        }
        if (i < nl) {
            step_norm<NP, 0, true>(sN[i], sWn[i], cbp, cur, aux, sp, pr, pi);
            if (i + 1 < nl) step_norm<NP, 1, true>(sN[i + 1], sWn[i + 1], cbp, cur, aux, sp, pr, pi);
            if (i + 2 < nl) step_norm<NP, 0, true>(sN[i + 2], sWn[i + 2], cbp, cur, aux, sp, pr, pi);
            rescale_pairs(cur, aux, nsc, sp);
        }
    }
}

// Angles where the normalised float recursion is used: sin(beta) >= max(0.1, 1.2e-5 l_max).
// There its error stays near 3e-5 (emulated against the FP64 oracle: it grows like
// l / sin(beta)); closer to the poles the difference form runs.  Chains starting at
// l0 >= 8192 also run the difference form: the growth bound of the four steps between
// rescales holds for the normalised form (ratio <= 4 F0 + 1 with rho <= 2) only below.
__device__ __forceinline__ float bulk_sin_threshold(int L) { return fmaxf(0.1f, 1.2e-5f * (float)L); }
constexpr int NORM_L0_LIMIT = 8192;

// One work item of the FP32 form: chain columns k in [k_begin, k_end) (m_sky-major
// order) for the angle chunk `chunk` (NT*CPT angles).  Every thread of the CTA calls it.
template <int NT, int CPT, int TL>
__device__ __forceinline__ void conv_fp32x_item(const ConvArgs &A, const Tables &T, int chunk, int k_begin,
                                                int k_end, SmemFp32<NT, CPT, TL> &sm, unsigned long long &n_elem,
                                                unsigned long long &n_sum) {
    static_assert(TL % 4 == 0, "tile length must be a multiple of 4 (parity of l and the rescale period)");
    static_assert(CPT % 2 == 0, "chains are processed in pairs");
    constexpr int NP = CPT / 2;
    const int MB1 = A.mb_max + 1;
    const int L = A.l_max;
    const int NB = A.n_beta;
    const int tid = threadIdx.x;
    // a thread's chains are CPT adjacent angles, a warp's 32 CPT consecutive ones, so that
    // only the warps that hold angles near a pole take the difference form
    const int j0 = chunk * NT * CPT + tid * CPT;  // angle of chain c: j0 + c

    int hbits = 0;    // bit c: chain c is mirrored (beta > pi/2)
    bool bulk = true;
    const float sthr = bulk_sin_threshold(L);
    float2 x2p[NP], cbp[NP];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        const bool valid = j0 + c < NB;
        const Angle32 t = make_angle32(valid ? A.beta[j0 + c] : 1.0);
        if (valid && t.bad) raise_status(T.status, WG_DEVERR_BETA);
        hbits |= (t.high ? 1 : 0) << c;
        bulk = bulk && (t.sb >= sthr) && !t.bad;
        if (c & 1) {
            x2p[c / 2].y = t.x2;
            cbp[c / 2].y = t.cb;
        } else {
            x2p[c / 2].x = t.x2;
            cbp[c / 2].x = t.cb;
        }
        sm.sLog[c][tid] = make_float4(t.lnc.hi, t.lnc.lo, t.lns.hi, t.lns.lo);
        sm.sFlag[c][tid] = (t.bad ? 1 : 0) | (t.high ? 2 : 0) | (t.c_zero ? 4 : 0) | (t.s_zero ? 8 : 0);
    }
    const int thigh = hbits & 1;                             // the thread's side when uniform
    const bool same = hbits == 0 || hbits == (1 << CPT) - 1;
    const bool uniform = __all_sync(0xffffffffu, same);      // warp-uniform code paths
    const bool wbulk = __all_sync(0xffffffffu, bulk);
    // one float per chain stays live: cos(beta) for warps of the normalised form (whose
    // rare columns from l0 >= 8192 take x^2 = (1 - |cos beta|) / 2, accurate there as
    // sin(beta) >= 0.1), x^2 for the others
    float2 xr[NP];
#pragma unroll
    for (int p = 0; p < NP; ++p) xr[p] = wbulk ? cbp[p] : x2p[p];

    for (int k = k_begin; k < k_end; ++k) {
        const int ms = k / MB1, mb = k - ms * MB1;
        const int l0 = mb > ms ? mb : ms;
        const bool norm = wbulk && l0 < NORM_L0_LIMIT;  // this warp runs the normalised form
        if (tid == 0) {  // read by build_tile after the barrier below
            const ff k0 = sigma_log(l0, mb, ms, T.E_f), k1 = sigma_log(l0 + 1, mb, ms, T.E_f);
            sm.sKc = make_float4(k0.hi, k0.lo, k1.hi, k1.lo);
        }
        const int n_norm = __syncthreads_count(norm);  // warp-uniform: a warp runs one form
        const bool need_norm = n_norm > 0, need_diff = n_norm < NT;

        float2 cur[NP], aux[NP], sp[NP], pr[2][NP], pi[2][NP];
        float2 xv[NP];  // per chain: cos(beta) (normalised form) or x^2 (difference form)
#pragma unroll
        for (int p = 0; p < NP; ++p)
            xv[p] = (norm || !wbulk) ? xr[p]
                                     : make_float2(0.5f * (1.0f - fabsf(xr[p].x)), 0.5f * (1.0f - fabsf(xr[p].y)));
        int nsc[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const float4 lg = sm.sLog[c][tid];
            const int fl = sm.sFlag[c][tid];
            Angle32 t;
            t.lnc = ff{lg.x, lg.y};
            t.lns = ff{lg.z, lg.w};
            t.c_zero = (fl & 4) != 0;
            t.s_zero = (fl & 8) != 0;
            const Seed32 s = seed32(mb, ms, t, T);
            // difference form: mirrored chains start from e^{l0} = (-1)^{l0} d^{l0},
            // Delta_{l0} = d^{l0}; normalised form: u^{l0} = d^{l0}, u^{l0-1} = 0
            const float v = (!norm && (fl & 2) && (l0 & 1)) ? -s.mant : s.mant;
            const float av = norm ? 0.0f : v;
            const float spv = (s.n == 0) ? 1.0f : 0.0f;  // a scaled seed has n <= -2
            if (c & 1) {
                cur[c / 2].y = v;
                aux[c / 2].y = av;
                sp[c / 2].y = spv;
            } else {
                cur[c / 2].x = v;
                aux[c / 2].x = av;
                sp[c / 2].x = spv;
            }
            nsc[c] = s.n;
            if (s.n == 0 && j0 + c < NB) n_sum += (unsigned long long)(L + 1 - l0);
            sm.sAcc[c][tid] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
        bool warp_plain = false;

        // first tile's operands into buffer 0
        build_tile<NT, CPT, TL>(A, T, l0, l0, mb, ms, need_diff, need_norm, sm, 0);
        __syncthreads();

        int buf = 0;
        for (int ts = l0; ts <= L; ts += TL, buf ^= 1) {
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                pr[0][p] = pr[1][p] = pi[0][p] = pi[1][p] = make_float2(0.f, 0.f);
            }
            const int nl = min(TL, L + 1 - ts);
            if (!warp_plain) {
                // a chain with n = -1 (value >= 2^-64) becomes a plain float here, at the
                // tile boundary (exact: a power-of-two scaling of normal floats)
                bool p = true;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    if (nsc[c] == -1) {
                        float &cu = (c & 1) ? cur[c / 2].y : cur[c / 2].x;
                        float &au = (c & 1) ? aux[c / 2].y : aux[c / 2].x;
                        float &su = (c & 1) ? sp[c / 2].y : sp[c / 2].x;
                        cu *= 0x1p-64f;
                        au *= 0x1p-64f;
                        su = 1.0f;
                        nsc[c] = 0;
                        if (j0 + c < NB) n_sum += (unsigned long long)(L + 1 - ts);
                    }
                    p = p && (nsc[c] == 0);
                }
                warp_plain = __all_sync(0xffffffffu, p);
            }
            const int period = rescale_period(l0, ts - l0);
            if (norm)
                tile_steps_norm<NP, TL>(sm.sN[buf], sm.sWn[buf], nl, warp_plain, period, xv, cur, aux, nsc, sp, pr,
                                        pi);
            else if (uniform)
                tile_steps<NP, TL, true>(sm.sA[buf], sm.sK[buf], sm.sW[buf], nl, warp_plain, period, thigh, hbits, xv, cur,
                                         aux, nsc, sp, pr, pi);
            else
                tile_steps<NP, TL, false>(sm.sA[buf], sm.sK[buf], sm.sW[buf], nl, warp_plain, period, thigh, hbits, xv, cur,
                                          aux, nsc, sp, pr, pi);
            // partials of this tile into the compensated sums; the sign of the odd-offset
            // partial is (-1) for mirrored chains of the difference form, and the tile's
            // start parity (that of l0, as TL is even) is applied at the end
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                const float sg = (((hbits >> c) & 1) && !norm) ? -1.f : 1.f;
                const float p0r = (c & 1) ? pr[0][c / 2].y : pr[0][c / 2].x;
                const float p1r = (c & 1) ? pr[1][c / 2].y : pr[1][c / 2].x;
                const float p0i = (c & 1) ? pi[0][c / 2].y : pi[0][c / 2].x;
                const float p1i = (c & 1) ? pi[1][c / 2].y : pi[1][c / 2].x;
                float4 acc = sm.sAcc[c][tid];
                neumaier_add(acc.x, acc.y, p0r + sg * p1r);
                neumaier_add(acc.z, acc.w, p0i + sg * p1i);
                sm.sAcc[c][tid] = acc;
            }
            // the next tile: its operands into the other buffer (their previous readers
            // passed the barrier at the end of the last tile) as soon as this warp is done
            // with the current one, then the tile's one barrier
            const int tn = ts + TL;
            if (tn <= L) {
                build_tile<NT, CPT, TL>(A, T, tn, l0, mb, ms, need_diff, need_norm, sm, buf ^ 1);
                __syncthreads();
            }
        }
        double2 *out = reinterpret_cast<double2 *>(A.c_out) + ((size_t)mb * (A.ms_max + 1) + ms) * NB;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const int j = j0 + c;
            if (j < NB) {
                const int fl = sm.sFlag[c][tid];
                const float4 acc = sm.sAcc[c][tid];
                const double sg = (!norm && (fl & 2) && (l0 & 1)) ? -1.0 : 1.0;
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                // the weights' power-of-two scales back (two exact factors within the
                // double range)
                const int k = (A.ea ? A.ea[ms] : 0) + (A.eb ? A.eb[mb] : 0);
                const int k1 = min(1023, max(-1022, k / 2)), k2 = min(1023, max(-1022, k - k1));
                const double re = sg * ((((double)acc.x + (double)acc.y) * pow2(k1)) * pow2(k2));
                const double im = sg * ((((double)acc.z + (double)acc.w) * pow2(k1)) * pow2(k2));
                out[j] = (fl & 1) ? make_double2(nan, nan) : make_double2(re, im);
                n_elem += (unsigned long long)(L + 1 - l0);
            }
        }
        __syncthreads();  // the sums and buffers are reused by the next column
    }
}

}  // namespace wg
