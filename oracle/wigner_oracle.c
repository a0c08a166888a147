/*
 * wigner_oracle.c -- plain CPU oracle for the reduced Wigner matrices and the
 * beam-convolution l-sum (Prezeau & Reinecke, "Algorithm for the evaluation of
 * reduced Wigner matrices").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package smoke check and the
 * bench's CPU-baseline leg may load this file's library.  It shares no code,
 * header, table or constant with the CUDA path, and is deliberately slow and
 * literal:
 *
 *   - seeds follow Eqs. ini1-ini2 (Sec. 3.2) in log form, Eq. logstart, with
 *     ln n! from lgammal and the half-angle logarithms in long double
 *     (the paper's "extended IEEE precision" for the seed, Sec. 3.2);
 *   - the l-recursion is Eq. lrec solved for d^{l+1}, with its coefficients
 *     computed straight from the equation (square roots of integer products,
 *     one division per step) in IEEE double -- not from the paper's P/Q/F tables
 *     of Sec. 4.2.2, so the two routes round differently;
 *   - values are kept as scaled doubles v = d * S^n with S = 2^90 (Sec. 3.2),
 *     the pair (d^l, d^{l-1}) rescaled jointly whenever the newest value leaves
 *     [S^-1, S]; this is done at every step, all the way to l_max (power-of-two
 *     scaling is exact, so this equals the paper's switch to plain doubles at
 *     2^-900 wherever neither form under- or overflows);
 *   - the weighted sum of Eq. convdef, C = sum_l conj(b_{l m_b}) a_{l m_sky} d^l,
 *     runs over every l >= max(m_b, m_sky) (no epsilon threshold);
 *   - the beta-derivative used for gradients is the tangent-linear recurrence
 *     (Eq. lrec differentiated in beta), a different route from the m'-neighbour
 *     relation Eq. mrec.
 *
 * Orders: 0 <= m_b <= mb_max, 0 <= m_sky <= ms_max, both <= l_max.
 * Layouts (row-major, complex = interleaved re,im doubles):
 *   d   [mb_max+1][ms_max+1][l_max+1][n_beta]   (zero where l < max(m_b, m_sky))
 *   a   [l_max+1][ms_max+1] complex,  b [l_max+1][mb_max+1] complex
 *   C   [mb_max+1][ms_max+1][n_beta] complex
 * Compile: gcc -O2 -ffp-contract=off -fno-fast-math -fopenmp -shared -fPIC.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORACLE_LOG2_S 90 /* S = 2^90, Sec. 3.2 */

/* ORACLE_PLANT = k > 0 compiles a copy with one deliberate mistake, for the test
 * that shows the pins catch it (tests/test_oracle_plants.py).  0 = the oracle. */
#ifndef ORACLE_PLANT
#define ORACLE_PLANT 0
#endif

typedef long double ldbl;

/* ---- per-angle half-angle logarithms (Sec. 4.2.2, first precomputation) ---- */
typedef struct {
    double cosb;   /* cos(beta), rounded to double from long double */
    double sinb;   /* sin(beta) */
    ldbl lnc;      /* ln cos(beta/2)  (-inf at beta = pi) */
    ldbl lns;      /* ln sin(beta/2)  (-inf at beta = 0)  */
    ldbl tan_h;    /* tan(beta/2) */
} angle_t;

static angle_t make_angle(double beta) {
    angle_t t;
    ldbl hb = (ldbl)beta / 2.0L;
    ldbl c = cosl(hb), s = sinl(hb);
    t.cosb = (double)cosl((ldbl)beta);
    t.sinb = (double)sinl((ldbl)beta);
    t.lnc = (c > 0.0L) ? logl(c) : -INFINITY;
    t.lns = (s > 0.0L) ? logl(s) : -INFINITY;
    t.tan_h = s / c;
    return t;
}

static ldbl ln_fact(int n) { return lgammal((ldbl)n + 1.0L); }

/* ---- seed: d^{l0}_{m,mp}(beta), l0 = max(|m|, |mp|)  (Eqs. ini1-ini2, logstart) ----
 * With c = cos(beta/2), s = sin(beta/2) the four edge values of Sec. 3.2 are
 *   mp =  l0 (|m| <= l0): d^{l0}_{m, l0}  = A c^{l0+m}  s^{l0-m},     A = sqrt((2l0)!/((l0+m)!(l0-m)!))
 *   mp = -l0 (|m| <= l0): d^{l0}_{m,-l0}  = A c^{l0-m}  (-s)^{l0+m}
 *   m  =  l0 (|mp| < l0): d^{l0}_{l0, mp} = A c^{l0+mp} (-s)^{l0-mp}, A = sqrt((2l0)!/((l0+mp)!(l0-mp)!))
 *   m  = -l0 (|mp| < l0): d^{l0}_{-l0,mp} = A c^{l0-mp} s^{l0+mp}
 * (for m, mp >= 0 only the first and third occur).
 * Returns the scaled pair (mant, n): value = mant * 2^(90 n), mant in [1, 2^90) or 0.
 * pc, ps receive the exponents of c and s (for the derivative of the seed). */
static void seed_scaled(int m, int mp, const angle_t *t, double *mant, int *n, int *pc, int *ps) {
    int am = m < 0 ? -m : m, amp = mp < 0 ? -mp : mp;
    int l0 = am > amp ? am : amp;
    int k;   /* the order that is not at the edge: A = sqrt((2l0)!/((l0+k)!(l0-k)!)) */
    int p, q, neg_s;
    if (amp >= am) {
        k = m;
        if (mp >= 0) { p = l0 + m; q = l0 - m; neg_s = 0; }
        else         { p = l0 - m; q = l0 + m; neg_s = 1; }
    } else {
        k = mp;
        if (m >= 0)  { p = l0 + mp; q = l0 - mp; neg_s = 1; }
        else         { p = l0 - mp; q = l0 + mp; neg_s = 0; }
    }
    int sign = (neg_s && (q & 1)) ? -1 : 1;
#if ORACLE_PLANT == 2
    sign = 1; /* planted: sign of (-sin(beta/2))^(l-m) dropped */
#endif
    *pc = p;
    *ps = q;
    ldbl r = 0.5L * (ln_fact(2 * l0) - ln_fact(l0 + k) - ln_fact(l0 - k));
    /* a zero power contributes nothing even where the logarithm is -inf */
    if (p > 0) {
        if (isinf(t->lnc)) { *mant = 0.0; *n = 0; return; } /* early stop: all values 0 (Sec. 3.2) */
        r += (ldbl)p * t->lnc;
    }
    if (q > 0) {
        if (isinf(t->lns)) { *mant = 0.0; *n = 0; return; }
#if ORACLE_PLANT == 3
        r += (ldbl)q * t->lnc; /* planted: cos where sin belongs */
#else
        r += (ldbl)q * t->lns;
#endif
    }
    ldbl ln_s = (ldbl)ORACLE_LOG2_S * logl(2.0L);
    ldbl kk_ = floorl(r / ln_s);
    ldbl rem = r - kk_ * ln_s; /* in [0, ln S) up to rounding */
    ldbl v = expl(rem);
    int kk = (int)kk_;
    /* renormalise if rounding pushed v just outside [1, S) */
    if (v >= ldexpl(1.0L, ORACLE_LOG2_S)) { v = ldexpl(v, -ORACLE_LOG2_S); kk += 1; }
    if (v < 1.0L) { v = ldexpl(v, ORACLE_LOG2_S); kk -= 1; }
    *mant = (double)(sign * v);
    *n = kk;
}

/* ---- coefficients of Eq. lrec at order l for orders (m, m') ----
 * [cos b - m m'/(l(l+1))] d^l = alpha_l d^{l-1} + gamma_l d^{l+1}
 * alpha_l = sqrt((l^2-m^2)(l^2-m'^2)) / (l (2l+1)),
 * gamma_l = sqrt(((l+1)^2-m^2)((l+1)^2-m'^2)) / ((l+1)(2l+1)).
 * At l = 0 (only m = m' = 0) the 0/0 terms are 0 (d^{-1} = 0). */
typedef struct { double f1, alpha, gamma; } lrec_coef;

static lrec_coef coef_at(int l, int m, int mp) {
    lrec_coef c;
    if (l == 0) {
        c.f1 = 0.0;
        c.alpha = 0.0;
    } else {
        c.f1 = ((double)m * (double)mp) / ((double)l * (double)(l + 1));
        int64_t num = ((int64_t)l * l - (int64_t)m * m) * ((int64_t)l * l - (int64_t)mp * mp);
        c.alpha = sqrt((double)num) / ((double)l * (double)(2 * l + 1));
    }
    int64_t l1 = l + 1;
    int64_t num1 = (l1 * l1 - (int64_t)m * m) * (l1 * l1 - (int64_t)mp * mp);
    c.gamma = sqrt((double)num1) / ((double)l1 * (double)(2 * l + 1));
    return c;
}

static const double S_UP = 0x1p90;    /* S    */
static const double S_DOWN = 0x1p-90; /* 1/S  */

/* One chain d^l_{mb,ms}(beta), l = l0..l_max.  Calls back per l with the scaled
 * value (mant, n) and, when dmant != NULL, the scaled beta-derivative.  The
 * `scaling` flag exists for the test that checks scaled == unscaled bitwise. */
typedef struct {
    int l_max, mb, ms;
    const angle_t *t;
    int scaling;
    int with_deriv;
} chain_spec;

typedef void (*chain_visit)(void *ctx, int l, double mant, double dmant, int n);

static void run_chain(const chain_spec *cs, chain_visit visit, void *ctx) {
    int amb = cs->mb < 0 ? -cs->mb : cs->mb, ams = cs->ms < 0 ? -cs->ms : cs->ms;
    int l0 = amb > ams ? amb : ams;
    if (l0 > cs->l_max) return;
    double cur, prev = 0.0, dcur = 0.0, dprev = 0.0;
    int n, pc, ps;
    seed_scaled(cs->mb, cs->ms, cs->t, &cur, &n, &pc, &ps);
    if (!cs->scaling) {
        cur = ldexp(cur, ORACLE_LOG2_S * n);
        n = 0;
    }
    if (cs->with_deriv && cur != 0.0) {
        /* d/dbeta of A c^p s^q = A c^p s^q (-(p/2) tan(b/2) + (q/2) cot(b/2)) */
        ldbl th = cs->t->tan_h;
        ldbl fac = -0.5L * (ldbl)pc * th + 0.5L * (ldbl)ps / th;
        dcur = (double)((ldbl)cur * fac);
    }
    const double cb = cs->t->cosb, sb = cs->t->sinb;
    for (int l = l0;; ++l) {
        visit(ctx, l, cur, dcur, n);
        if (l == cs->l_max) break;
        lrec_coef k = coef_at(l, cs->mb, cs->ms);
        double tl = cb - k.f1;
#if ORACLE_PLANT == 1
        double next = (tl * cur) / k.gamma; /* planted: d^{l-1} term dropped */
#elif ORACLE_PLANT == 4
        lrec_coef k1 = coef_at(l + 1, cs->mb, cs->ms); /* planted: coefficient one order off */
        double next = (tl * cur - k1.alpha * prev) / k.gamma;
#else
        double next = (tl * cur - k.alpha * prev) / k.gamma;
#endif
        double dnext = 0.0;
        if (cs->with_deriv) dnext = (-sb * cur + tl * dcur - k.alpha * dprev) / k.gamma;
        prev = cur;
        cur = next;
        dprev = dcur;
        dcur = dnext;
        if (cs->scaling) {
            double a = fabs(cur);
            if (a > S_UP) {
#if ORACLE_PLANT == 5
                cur *= S_DOWN; dcur *= S_DOWN; dprev *= S_DOWN; n += 1; /* planted: pair not rescaled jointly */
#else
                cur *= S_DOWN; prev *= S_DOWN; dcur *= S_DOWN; dprev *= S_DOWN; n += 1;
#endif
            } else if (a != 0.0 && a < S_DOWN) {
                cur *= S_UP; prev *= S_UP; dcur *= S_UP; dprev *= S_UP; n -= 1;
            }
        }
    }
}

static inline double unscale(double mant, int n) { return ldexp(mant, ORACLE_LOG2_S * n); }

/* ------------------------------------------------------------------------- */
/* d-table                                                                    */
/* ------------------------------------------------------------------------- */
typedef struct { double *col; int n_beta; int j; } dtab_ctx;

static void dtab_visit(void *vctx, int l, double mant, double dmant, int n) {
    (void)dmant;
    dtab_ctx *c = (dtab_ctx *)vctx;
    c->col[(size_t)l * c->n_beta + c->j] = unscale(mant, n);
}

static int check_orders(int l_max, int mb_max, int ms_max, int n_beta) {
    if (l_max < 0 || mb_max < 0 || ms_max < 0 || n_beta < 0) return -1;
    if (mb_max > l_max || ms_max > l_max) return -1;
    if (l_max > 100000) return -1;
    return 0;
}

/* d[mb][ms][l][j] for all 0<=mb<=mb_max, 0<=ms<=ms_max, 0<=l<=l_max, beta_j.
 * scaling = 1 for the paper's scaled doubles, 0 for a plain unscaled recurrence. */
int oracle_d_table(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                   int scaling, double *d_out) {
    if (check_orders(l_max, mb_max, ms_max, n_beta)) return -1;
    size_t col_len = (size_t)(l_max + 1) * n_beta;
    angle_t *ang = (angle_t *)malloc(sizeof(angle_t) * (n_beta ? n_beta : 1));
    for (int j = 0; j < n_beta; ++j) ang[j] = make_angle(beta[j]);
    int ncol = (mb_max + 1) * (ms_max + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < ncol; ++c) {
        int mb = c / (ms_max + 1), ms = c % (ms_max + 1);
        double *col = d_out + (size_t)c * col_len;
        memset(col, 0, sizeof(double) * col_len);
        for (int j = 0; j < n_beta; ++j) {
            chain_spec cs = {l_max, mb, ms, &ang[j], scaling, 0};
            dtab_ctx ctx = {col, n_beta, j};
            run_chain(&cs, dtab_visit, &ctx);
        }
    }
    free(ang);
    return 0;
}

/* One chain column d[l][j] = d^l_{mb,ms}(beta_j), l = 0..l_max (zero below max(mb, ms)). */
int oracle_d_column(int l_max, int mb, int ms, int n_beta, const double *beta, double *d_out) {
    if (l_max < 0 || mb < 0 || ms < 0 || mb > l_max || ms > l_max || n_beta < 0) return -1;
    memset(d_out, 0, sizeof(double) * (size_t)(l_max + 1) * n_beta);
#pragma omp parallel for schedule(dynamic, 4)
    for (int j = 0; j < n_beta; ++j) {
        angle_t t = make_angle(beta[j]);
        chain_spec cs = {l_max, mb, ms, &t, 1, 0};
        dtab_ctx ctx = {d_out, n_beta, j};
        run_chain(&cs, dtab_visit, &ctx);
    }
    return 0;
}

/* Single element d^l_{m m'}(beta) for |m|, |m'| <= l (used by sampled checks). */
typedef struct { int want_l; double val; } one_ctx;

static void one_visit(void *vctx, int l, double mant, double dmant, int n) {
    (void)dmant;
    one_ctx *c = (one_ctx *)vctx;
    if (l == c->want_l) c->val = unscale(mant, n);
}

double oracle_d_single(int l, int m, int mp, double beta) {
    if (m < -l || mp < -l || m > l || mp > l) return NAN;
    angle_t t = make_angle(beta);
    chain_spec cs = {l, m, mp, &t, 1, 0};
    one_ctx ctx = {l, 0.0};
    run_chain(&cs, one_visit, &ctx);
    return ctx.val;
}

/* The rows 0 <= m <= m_max of the matrix d^l(beta_j) at one l, every -l <= m' <= l:
 * d_out[m][m' + l][j], shape (m_max+1, 2l+1, n_beta).  Each element is the end of its
 * own l-chain from the general edge seed at l0 = max(|m|, |m'|) (the definition through
 * the pinned chain code; no m-recursion, no ratios, no symmetry). */
int oracle_d_matrix(int l, int m_max, int n_beta, const double *beta, double *d_out) {
    if (l < 0 || l > 100000 || m_max < 0 || m_max > l || n_beta < 0) return -1;
    angle_t *ang = (angle_t *)malloc(sizeof(angle_t) * (n_beta ? n_beta : 1));
    for (int j = 0; j < n_beta; ++j) ang[j] = make_angle(beta[j]);
    int nmp = 2 * l + 1;
    long ncell = (long)(m_max + 1) * nmp;
#pragma omp parallel for schedule(dynamic, 16)
    for (long c = 0; c < ncell; ++c) {
        int m = (int)(c / nmp), mp = (int)(c % nmp) - l;
        for (int j = 0; j < n_beta; ++j) {
#if ORACLE_PLANT == 10
            chain_spec cs = {l, mp, m, &ang[j], 1, 0}; /* planted: row and column orders swapped */
#else
            chain_spec cs = {l, m, mp, &ang[j], 1, 0};
#endif
            one_ctx ctx = {l, 0.0};
            run_chain(&cs, one_visit, &ctx);
            d_out[(size_t)c * n_beta + j] = ctx.val;
        }
    }
    free(ang);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The l_min cut of Sec. 4.2.1 (Eq. lmin, its second, approximate line): in the */
/* chain (m_b, m', beta) the terms with l below                                 */
/*     l_min = (sqrt(m'^2 + m_b^2 - 2 m' m_b cos beta) - offset) / sin beta      */
/* lie in the non-classical, exponentially small region (Eq. classiccond) and   */
/* are left out of the sum; offset > 0 moves the cut away from the turning      */
/* point.  At sin beta = 0 (beta = 0) d = delta_{m_b m'}: the chain is left out */
/* unless m_b = m'.  Returns the first l of the sum: l0 = max(|m_b|, |m'|) when */
/* nothing is cut, l_max + 1 when the whole chain is.  Double precision, no     */
/* contraction (the compile flags say so), every operation rounded once.        */
/* ------------------------------------------------------------------------- */
static int l_first(int l_max, int l0, int mb, int mp, const angle_t *t, double offset) {
    if (t->sinb == 0.0) return (mb == mp) ? l0 : l_max + 1;
    double q = (double)mb * (double)mb + (double)mp * (double)mp;
#if ORACLE_PLANT == 8
    q = q + (2.0 * (double)mb * (double)mp) * t->cosb; /* planted: sign of the cos term */
#else
    q = q - (2.0 * (double)mb * (double)mp) * t->cosb;
#endif
    double x = (sqrt(q) - offset) / t->sinb;
    if (!(x <= (double)l_max)) return l_max + 1;
    if (x <= (double)l0) return l0;
    return (int)ceil(x);
}

int oracle_l_first(int l_max, int mb, int mp, double beta, double offset) {
    int amb = mb < 0 ? -mb : mb, amp = mp < 0 ? -mp : mp;
    int l0 = amb > amp ? amb : amp;
    angle_t t = make_angle(beta);
    return l_first(l_max, l0, mb, mp, &t, offset);
}

/* ------------------------------------------------------------------------- */
/* beam-convolution l-sum, Eq. convdef                                        */
/* ------------------------------------------------------------------------- */
typedef struct {
    const double *a, *b; /* interleaved complex */
    int ms_max1, mb_max1, mb, ms;
    double cre, cim;      /* C accumulator */
    double ere, eim;      /* sum of w * d/dbeta accumulator */
    int lfirst;           /* terms with l < lfirst are left out (the l_min cut; 0 = none) */
} sum_ctx;

static void sum_visit(void *vctx, int l, double mant, double dmant, int n) {
    sum_ctx *c = (sum_ctx *)vctx;
    if (l < c->lfirst) return;
    const double *al = c->a + 2 * ((size_t)l * c->ms_max1 + c->ms);
#if ORACLE_PLANT == 7
    const double *bl = c->b + 2 * ((size_t)l * c->mb_max1 + (c->mb_max1 - 1 - c->mb)); /* planted: wrong beam column */
#else
    const double *bl = c->b + 2 * ((size_t)l * c->mb_max1 + c->mb);
#endif
    /* w = conj(b) * a */
#if ORACLE_PLANT == 6
    double wre = bl[0] * al[0] - bl[1] * al[1]; /* planted: b not conjugated */
    double wim = bl[0] * al[1] + bl[1] * al[0];
#else
    double wre = bl[0] * al[0] + bl[1] * al[1];
    double wim = bl[0] * al[1] - bl[1] * al[0];
#endif
    double d = unscale(mant, n);
    double dd = unscale(dmant, n);
    c->cre += wre * d;
    c->cim += wim * d;
    c->ere += wre * dd;
    c->eim += wim * dd;
}

/* C[mb][ms][j] = sum_{l=max(mb,ms)}^{l_max} conj(b[l][mb]) a[l][ms] d^l_{mb ms}(beta_j);
 * cut != 0: the sum starts at the l_min of Eq. lmin for that offset. */
static int conv_sum_impl(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                         const double *a, const double *b, int cut, double offset, double *c_out) {
    if (check_orders(l_max, mb_max, ms_max, n_beta)) return -1;
    angle_t *ang = (angle_t *)malloc(sizeof(angle_t) * (n_beta ? n_beta : 1));
    for (int j = 0; j < n_beta; ++j) ang[j] = make_angle(beta[j]);
    int ncol = (mb_max + 1) * (ms_max + 1);
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < ncol; ++c) {
        int mb = c / (ms_max + 1), ms = c % (ms_max + 1);
        int l0 = mb > ms ? mb : ms;
        for (int j = 0; j < n_beta; ++j) {
            chain_spec cs = {l_max, mb, ms, &ang[j], 1, 0};
            sum_ctx ctx = {a, b, ms_max + 1, mb_max + 1, mb, ms, 0.0, 0.0, 0.0, 0.0, 0};
            if (cut) ctx.lfirst = l_first(l_max, l0, mb, ms, &ang[j], offset);
            if (ctx.lfirst <= l_max) run_chain(&cs, sum_visit, &ctx);
            double *o = c_out + 2 * ((size_t)c * n_beta + j);
            o[0] = ctx.cre;
            o[1] = ctx.cim;
        }
    }
    free(ang);
    return 0;
}

int oracle_conv_sum(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                    const double *a, const double *b, double *c_out) {
    return conv_sum_impl(l_max, mb_max, ms_max, n_beta, beta, a, b, 0, 0.0, c_out);
}

int oracle_conv_sum_lmin(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                         const double *a, const double *b, double offset, double *c_out) {
    return conv_sum_impl(l_max, mb_max, ms_max, n_beta, beta, a, b, 1, offset, c_out);
}

/* The sum over every sky order, -ms_max <= m_sky <= ms_max, for a real sky field:
 * s_{l,-m} = (-1)^m conj(s_{l m}) (Sec. 4.2, the b/s symmetry relation), so only the
 * m_sky >= 0 coefficients a[l][m] are passed.  Each negative order runs its own chain
 * d^l_{m_b,m_sky}(beta), m_sky < 0, from the general seed above.
 * C[mb][ms + ms_max][j], shape (mb_max+1, 2 ms_max+1, n_beta). */
typedef struct {
    const double *a, *b;
    int ms_max1, mb_max1, mb, ms;  /* ms may be negative */
    double cre, cim;
    int lfirst;                    /* as in sum_ctx */
} full_ctx;

static void full_visit(void *vctx, int l, double mant, double dmant, int n) {
    (void)dmant;
    full_ctx *c = (full_ctx *)vctx;
    if (l < c->lfirst) return;
    int am = c->ms < 0 ? -c->ms : c->ms;
    const double *al = c->a + 2 * ((size_t)l * c->ms_max1 + am);
    double sre = al[0], sim = al[1];
    if (c->ms < 0) {  /* (-1)^m conj(a_{l,|m|}) */
#if ORACLE_PLANT == 9
        double sg = 1.0; /* planted: the (-1)^m of the real-sky relation dropped */
#else
        double sg = (am & 1) ? -1.0 : 1.0;
#endif
        sre = sg * al[0];
        sim = -sg * al[1];
    }
    const double *bl = c->b + 2 * ((size_t)l * c->mb_max1 + c->mb);
    double wre = bl[0] * sre + bl[1] * sim;  /* conj(b) * s */
    double wim = bl[0] * sim - bl[1] * sre;
    double d = unscale(mant, n);
    c->cre += wre * d;
    c->cim += wim * d;
}

static int conv_sum_full_impl(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                              const double *a, const double *b, int cut, double offset, double *c_out) {
    if (check_orders(l_max, mb_max, ms_max, n_beta)) return -1;
    angle_t *ang = (angle_t *)malloc(sizeof(angle_t) * (n_beta ? n_beta : 1));
    for (int j = 0; j < n_beta; ++j) ang[j] = make_angle(beta[j]);
    int ns = 2 * ms_max + 1;
    int ncol = (mb_max + 1) * ns;
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < ncol; ++c) {
        int mb = c / ns, ms = c % ns - ms_max;
        int ams = ms < 0 ? -ms : ms, l0 = mb > ams ? mb : ams;
        for (int j = 0; j < n_beta; ++j) {
            chain_spec cs = {l_max, mb, ms, &ang[j], 1, 0};
            full_ctx ctx = {a, b, ms_max + 1, mb_max + 1, mb, ms, 0.0, 0.0, 0};
            if (cut) ctx.lfirst = l_first(l_max, l0, mb, ms, &ang[j], offset);
            if (ctx.lfirst <= l_max) run_chain(&cs, full_visit, &ctx);
            double *o = c_out + 2 * ((size_t)c * n_beta + j);
            o[0] = ctx.cre;
            o[1] = ctx.cim;
        }
    }
    free(ang);
    return 0;
}

int oracle_conv_sum_full(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                         const double *a, const double *b, double *c_out) {
    return conv_sum_full_impl(l_max, mb_max, ms_max, n_beta, beta, a, b, 0, 0.0, c_out);
}

int oracle_conv_sum_full_lmin(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                              const double *a, const double *b, double offset, double *c_out) {
    return conv_sum_full_impl(l_max, mb_max, ms_max, n_beta, beta, a, b, 1, offset, c_out);
}

/* Same sum restricted to a list of (mb, ms, j) triples (sampled checks at full size).
 * idx has 3*n_samples ints; out has 2*n_samples doubles. */
int oracle_conv_sum_sampled(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                            const double *a, const double *b, int n_samples, const int *idx,
                            double *out) {
    if (check_orders(l_max, mb_max, ms_max, n_beta)) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < n_samples; ++s) {
        int mb = idx[3 * s], ms = idx[3 * s + 1], j = idx[3 * s + 2];
        if (mb < 0 || mb > mb_max || ms < 0 || ms > ms_max || j < 0 || j >= n_beta) {
            out[2 * s] = NAN;
            out[2 * s + 1] = NAN;
            continue;
        }
        angle_t t = make_angle(beta[j]);
        chain_spec cs = {l_max, mb, ms, &t, 1, 0};
        sum_ctx ctx = {a, b, ms_max + 1, mb_max + 1, mb, ms, 0.0, 0.0, 0.0, 0.0, 0};
        run_chain(&cs, sum_visit, &ctx);
        out[2 * s] = ctx.cre;
        out[2 * s + 1] = ctx.cim;
    }
    return 0;
}

/* oracle_conv_sum_full at a list of (mb, ms, j) triples, -ms_max <= ms <= ms_max;
 * cut != 0: with the l_min cut of Eq. lmin for that offset. */
static int full_sampled_impl(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                             const double *a, const double *b, int n_samples, const int *idx,
                             int cut, double offset, double *out) {
    if (check_orders(l_max, mb_max, ms_max, n_beta)) return -1;
#pragma omp parallel for schedule(dynamic, 1)
    for (int s = 0; s < n_samples; ++s) {
        int mb = idx[3 * s], ms = idx[3 * s + 1], j = idx[3 * s + 2];
        if (mb < 0 || mb > mb_max || ms < -ms_max || ms > ms_max || j < 0 || j >= n_beta) {
            out[2 * s] = NAN;
            out[2 * s + 1] = NAN;
            continue;
        }
        angle_t t = make_angle(beta[j]);
        chain_spec cs = {l_max, mb, ms, &t, 1, 0};
        full_ctx ctx = {a, b, ms_max + 1, mb_max + 1, mb, ms, 0.0, 0.0, 0};
        int ams = ms < 0 ? -ms : ms, l0 = mb > ams ? mb : ams;
        if (cut) ctx.lfirst = l_first(l_max, l0, mb, ms, &t, offset);
        if (ctx.lfirst <= l_max) run_chain(&cs, full_visit, &ctx);
        out[2 * s] = ctx.cre;
        out[2 * s + 1] = ctx.cim;
    }
    return 0;
}

int oracle_conv_sum_full_sampled(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                                 const double *a, const double *b, int n_samples, const int *idx,
                                 double *out) {
    return full_sampled_impl(l_max, mb_max, ms_max, n_beta, beta, a, b, n_samples, idx, 0, 0.0, out);
}

int oracle_conv_sum_full_sampled_lmin(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                                      const double *a, const double *b, int n_samples, const int *idx,
                                      double offset, double *out) {
    return full_sampled_impl(l_max, mb_max, ms_max, n_beta, beta, a, b, n_samples, idx, 1, offset, out);
}

/* ------------------------------------------------------------------------- */
/* gradients of a real loss through C (PyTorch's convention for complex        */
/* tensors: grad = dL/dRe + i dL/dIm).                                        */
/*   grad_a[l][ms]  = sum_mb b[l][mb] S[l][mb][ms],   S = sum_j G[mb][ms][j] d^l(beta_j)
 *   grad_b[l][mb]  = sum_ms a[l][ms] conj(S[l][mb][ms])
 *   grad_beta[j]   = Re sum_{mb,ms} conj(G[mb][ms][j]) sum_l w_l d/dbeta d^l(beta_j)
 * with d/dbeta d^l from the tangent-linear recurrence.  Any output may be NULL.
 * Interior angles only: the seed derivative is singular at beta = 0 and pi. */
typedef struct {
    const double *g; /* G column for this (mb, ms): [n_beta] complex */
    double *s_col;   /* S[l] for this (mb, ms): [l_max+1] complex (per-thread scratch) */
    int j;
} grad_ctx;

static void grad_visit(void *vctx, int l, double mant, double dmant, int n) {
    (void)dmant;
    grad_ctx *c = (grad_ctx *)vctx;
    double d = unscale(mant, n);
    c->s_col[2 * l] += c->g[2 * c->j] * d;
    c->s_col[2 * l + 1] += c->g[2 * c->j + 1] * d;
}

int oracle_conv_grad(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                     const double *a, const double *b, const double *grad_c,
                     double *grad_a, double *grad_b, double *grad_beta) {
    if (check_orders(l_max, mb_max, ms_max, n_beta)) return -1;
    angle_t *ang = (angle_t *)malloc(sizeof(angle_t) * (n_beta ? n_beta : 1));
    for (int j = 0; j < n_beta; ++j) ang[j] = make_angle(beta[j]);
    int ncol = (mb_max + 1) * (ms_max + 1);
    size_t s_len = (size_t)(l_max + 1) * 2;
    double *S = (double *)calloc((size_t)ncol * s_len, sizeof(double));
    double *gb_cols = (double *)calloc((size_t)ncol * n_beta + 1, sizeof(double));
#pragma omp parallel for schedule(dynamic, 1)
    for (int c = 0; c < ncol; ++c) {
        int mb = c / (ms_max + 1), ms = c % (ms_max + 1);
        const double *g = grad_c + 2 * (size_t)c * n_beta;
        for (int j = 0; j < n_beta; ++j) {
            if (grad_a || grad_b) {
                chain_spec cs = {l_max, mb, ms, &ang[j], 1, 0};
                grad_ctx ctx = {g, S + (size_t)c * s_len, j};
                run_chain(&cs, grad_visit, &ctx);
            }
            if (grad_beta) {
                chain_spec cs = {l_max, mb, ms, &ang[j], 1, 1};
                sum_ctx ctx = {a, b, ms_max + 1, mb_max + 1, mb, ms, 0.0, 0.0, 0.0, 0.0, 0};
                run_chain(&cs, sum_visit, &ctx);
                /* Re(conj(G) * E) */
                gb_cols[(size_t)c * n_beta + j] = g[2 * j] * ctx.ere + g[2 * j + 1] * ctx.eim;
            }
        }
    }
    if (grad_a) {
        for (int l = 0; l <= l_max; ++l)
            for (int ms = 0; ms <= ms_max; ++ms) {
                double re = 0.0, im = 0.0;
                for (int mb = 0; mb <= mb_max; ++mb) {
                    const double *bl = b + 2 * ((size_t)l * (mb_max + 1) + mb);
                    const double *s = S + (size_t)(mb * (ms_max + 1) + ms) * s_len + 2 * l;
                    re += bl[0] * s[0] - bl[1] * s[1];
                    im += bl[0] * s[1] + bl[1] * s[0];
                }
                grad_a[2 * ((size_t)l * (ms_max + 1) + ms)] = re;
                grad_a[2 * ((size_t)l * (ms_max + 1) + ms) + 1] = im;
            }
    }
    if (grad_b) {
        for (int l = 0; l <= l_max; ++l)
            for (int mb = 0; mb <= mb_max; ++mb) {
                double re = 0.0, im = 0.0;
                for (int ms = 0; ms <= ms_max; ++ms) {
                    const double *al = a + 2 * ((size_t)l * (ms_max + 1) + ms);
                    const double *s = S + (size_t)(mb * (ms_max + 1) + ms) * s_len + 2 * l;
                    /* a * conj(S) */
                    re += al[0] * s[0] + al[1] * s[1];
                    im += al[1] * s[0] - al[0] * s[1];
                }
                grad_b[2 * ((size_t)l * (mb_max + 1) + mb)] = re;
                grad_b[2 * ((size_t)l * (mb_max + 1) + mb) + 1] = im;
            }
    }
    if (grad_beta) {
        for (int j = 0; j < n_beta; ++j) {
            double acc = 0.0;
            for (int c = 0; c < ncol; ++c) acc += gb_cols[(size_t)c * n_beta + j];
            grad_beta[j] = acc;
        }
    }
    free(S);
    free(gb_cols);
    free(ang);
    return 0;
}

/* Number of threads OpenMP will use (for reporting the CPU baseline's cores). */
int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
