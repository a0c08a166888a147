// wg_dtable.cu -- the full d-table d^l_{mb,ms}(beta_j) (Sec. 3.2 l-recursion).
//
// The d-table is short chains in great number (at l_max = 256: 82k chains of ~130 steps),
// so two things decide its speed on GB300, whose FP64 pipe takes a warp instruction per
// 64 cycles on each scheduler: how much FP64 work each element costs, and how evenly the
// chains are spread over the 608 schedulers.
//   * The FP64 pipe runs the recursion and little else: Eq. lrec's step is one DMUL and
//     two DFMA.  The step's coefficients (F0, G = F0 F1, F2 of Sec. 4.2.2) are formed in
//     double once per column and order by a set-up kernel (not once per 32 angles).  The
//     seeds (Eqs. ini1-ini2, logstart) take ~10 FP64 instructions instead of the
//     double-double seed's ~70: ln|d^{l0}| = pre + p ln c + q ln s in double (the
//     column's prefactor pre from the set-up kernel, the half-angle logarithms from the
//     angle's set-up), the reduction x = k ln 2 + r in double (Cody-Waite), and e^r in
//     float-float on the FP32 pipe by an exponential of the project's own (a Taylor
//     polynomial), made a double by integer operations.  A logarithm in double carries
//     an absolute error near |terms| 2^-53, the same order as the double-double seed's,
//     whose half-angle logarithms are doubles too.  (Coefficients and seed logarithms in
//     float-float, ~2^-47, were tried first: the chains' errors follow the coefficients'
//     and the seeds' and reached 7e-11 at l_max = 300.)
//   * Work is handed out per warp: an item is one chain column (mb, ms) for 32 angles,
//     items are ordered longest chain first, and each warp of a persistent grid takes
//     the next item from an atomic counter, so the schedulers stay evenly loaded down to
//     the shortest chains at the end.
// The per-angle quantities (cos beta, the half-angle logarithms), the per-column part of
// the seed logarithm and the coefficient tables are formed once per call by a set-up
// kernel laid out for the FP64 pipe (its comment says how).
#include <climits>
#include <cuda_runtime.h>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_internal.h"

namespace wg {

int host_pool(cudaMemPool_t *pool);  // wg_host.cu

// hi + lo (a float-float with |lo| <= ulp(hi)/2, hi normal or 0) as a double, by integer
// operations: the two significands are aligned in one 64-bit integer and added; bits
// below the double's last place are dropped (an error below 1 ulp).
__device__ __forceinline__ double ff_to_double(float hi, float lo) {
    const unsigned bh = __float_as_uint(hi), bl = __float_as_uint(lo);
    const int eh = (int)((bh >> 23) & 0xff);
    if (eh == 0) return 0.0;
    long long m = (long long)((bh & 0x7fffffu) | 0x800000u) << 29;  // value = m 2^(eh - 127 - 52)
    int e = eh;
    const int el = (int)((bl >> 23) & 0xff);
    if (el != 0) {
        long long ml = (long long)((bl & 0x7fffffu) | 0x800000u);  // value = ml 2^(el - 127 - 23)
        const int sft = el - eh + 29;                               // <= 5 as |lo| <= ulp(hi)/2
        ml = sft >= 0 ? (ml << sft) : (sft > -40 ? (ml >> -sft) : 0);
        m += ((bl ^ bh) >> 31) ? -ml : ml;
        if (m >= (1LL << 53)) {
            m >>= 1;
            e += 1;
        } else if (m < (1LL << 52)) {
            m <<= 1;
            e -= 1;
        }
    }
    return __longlong_as_double((long long)((unsigned long long)(bh >> 31) << 63 |
                                            (unsigned long long)(e - 127 + 1023) << 52 |
                                            ((unsigned long long)m & 0xfffffffffffffULL)));
}

// e^r for |r| <= ln 2 / 2 (+ a little) in float-float: the Taylor polynomial of degree
// 12 by Horner's rule (the first term left out, r^13 / 13!, is below 2^-52)
__device__ __forceinline__ ff ff_exp_reduced(ff r) {
    // 1/n!, n = 12 .. 0, as float-float
    const float2 c[13] = {
        {0x1.1eed8ep-29f, 0x1.ff1b12p-54f},  {0x1.ae6456p-26f, 0x1.fd5138p-52f},
        {0x1.27e4fcp-22f, -0x1.10ec14p-47f}, {0x1.71de3ap-19f, 0x1.55b1ccp-45f},
        {0x1.a01a02p-16f, -0x1.7f97fap-42f}, {0x1.a01a02p-13f, -0x1.7f97fap-39f},
        {0x1.6c16c2p-10f, -0x1.27d27ep-35f}, {0x1.111112p-7f, -0x1.dddddep-32f},
        {0x1.555556p-5f, -0x1.555556p-30f},  {0x1.555556p-3f, -0x1.555556p-28f},
        {0x1.0p-1f, 0.0f},                   {0x1.0p+0f, 0.0f},
        {0x1.0p+0f, 0.0f}};
    ff p{c[0].x, c[0].y};
#pragma unroll
    for (int i = 1; i < 13; ++i) p = ff_add(ff_mul(p, r), ff{c[i].x, c[i].y});
    return p;
}

// ln 2 in two doubles (Cody-Waite): HI has 32 significant bits, so k HI is exact for
// |k| < 2^21
#define WG_LN2_HI 0x1.62e42feep-1
#define WG_LN2_LO 0x1.a39ef35793c76p-33
#define WG_INV_LN2 0x1.71547652b82fep+0

// Per-angle quantities from the set-up kernel: the FP64 path's Angle, and its half-angle
// logarithms as float-float (their magnitudes bound the seed logarithm's terms).
struct DtAngle {
    Angle t;
    float lnc_hi, lnc_lo, lns_hi, lns_lo;
};

// Per-column part of the seed logarithm, (ln (2l0)! - ln (l0+m)! - ln (l0-m)!)/2, as
// double-double (and its magnitude as float-float).
struct DtCol {
    dd pre;
    float pre_hi, pre_lo;
};

// Chain column of item-order index c: the columns in order of l0 = max(mb, ms)
// ascending (longest chains first).  N(v) = min(v, MB+1) min(v, MS+1) columns have
// l0 < v; those with l0 = v are (v, ms) for ms <= min(v, MS) (if v <= MB), then (mb, v)
// for mb <= min(v-1, MB) (if v <= MS).
__device__ __forceinline__ void column_of(int c, int MB, int MS, int &mb, int &ms) {
    int lo = 0, hi = max(MB, MS);  // the largest v with N(v) <= c
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((long long)min(mid, MB + 1) * (long long)min(mid, MS + 1) <= (long long)c)
            lo = mid;
        else
            hi = mid - 1;
    }
    const int v = lo;
    const int r = c - min(v, MB + 1) * min(v, MS + 1);
    const int ca = (v <= MB) ? min(v, MS) + 1 : 0;
    if (r < ca) {
        mb = v;
        ms = r;
    } else {
        mb = r - ca;
        ms = v;
    }
}

// The coefficient tables of the set-up kernel: F0, G, F2 of column c at order l
// (l0 <= l < l_max) at index c l_max + l of each array.
struct DtCoef {
    double *f0, *g, *f2;
};

// One angle's quantities for the d-table: cos beta from the half angle (1 - 2 sin^2 or
// 2 cos^2 - 1, whichever has no cancellation: an absolute error of about one rounding
// unit), the half-angle logarithms as in make_angle but with one log and one log1p per
// angle (the smaller half-angle factor x takes log x, the larger ln sqrt(1 - x^2)), so a
// warp evaluates two logarithms whatever the mix of its angles.
__device__ __forceinline__ DtAngle dtable_angle(double beta) {
    DtAngle d;
    Angle &t = d.t;
    t.bad = !(beta >= 0.0 && beta <= WG_PI_HI);
    const double b = t.bad ? 1.0 : beta;
    double s, c;
    sincos(0.5 * b, &s, &c);
    t.cb = (s <= c) ? fma(-2.0 * s, s, 1.0) : fma(2.0 * c, c, -1.0);
    t.sb = 2.0 * s * c;
    t.s_zero = (s == 0.0);
    t.c_zero = (c <= 0.0);
    const double x = fmin(s, c);
    const double lx = log(x), ly = 0.5 * log1p(-x * x);
    t.lnc = (c >= s) ? ly : lx;
    t.lns = (s >= c) ? ly : lx;
    d.lnc_hi = d.lnc_lo = d.lns_hi = d.lns_lo = 0.0f;  // unused where the factor is 0
    if (!t.bad && !t.c_zero) {
        d.lnc_hi = __double2float_rn(t.lnc);
        d.lnc_lo = __double2float_rn(t.lnc - (double)d.lnc_hi);
    }
    if (!t.bad && !t.s_zero) {
        d.lns_hi = __double2float_rn(t.lns);
        d.lns_lo = __double2float_rn(t.lns - (double)d.lns_hi);
    }
    return d;
}

// The set-up of one call, one CTA of DTS_THREADS per SM (at 52 registers a thread two
// such CTAs do not fit one SM).  Its FP64 work is what costs: on GB300 each warp
// instruction of the FP64 pipe holds its scheduler for 64 cycles whatever the number of
// active lanes (measured), so a warp's latency is its FP64 instruction count times 64
// cycles times the number of warps sharing the scheduler.  The angles (a sincos and two
// logarithms: ~6k cycles for a warp alone on its scheduler, measured) therefore run in
// CTAs of their own, one warp per scheduler; the coefficients (10 FP64 multiplications per column and order, the integer
// factors made doubles by bit operations; 3 doubles stored) and the column prefactors
// (double-double, a few per CTA) fill the other CTAs.  Measured at the L = 256 workload:
// 10 us against 15-18 us for a grid of 128-thread CTAs in which the angle and prefactor
// warps shared their schedulers with up to 16 coefficient warps.
constexpr int DTS_THREADS = 1024;

__global__ void __launch_bounds__(DTS_THREADS, 1) dtable_setup_kernel(DTableArgs A, Tables T, DtAngle *ang,
                                                                      DtCol *cols, DtCoef cf, int *next, int n_ang) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if ((int)blockIdx.x < n_ang) {  // angle CTAs: warps 0..3, one per scheduler, 32 angles at a time
        const int n_chunks = (A.n_beta + 31) >> 5;
        if (warp < 4)
            for (int ch = (int)blockIdx.x * 4 + warp; ch < n_chunks; ch += n_ang * 4) {
                const int i = ch * 32 + lane;
                if (i < A.n_beta) {
                    const DtAngle d = dtable_angle(A.beta[i]);
                    if (d.t.bad) raise_status(T.status, WG_DEVERR_BETA);
                    ang[i] = d;
                }
            }
        return;
    }
    const long long i0 = (long long)(blockIdx.x - n_ang) * DTS_THREADS + threadIdx.x;
    const long long stride = (long long)(gridDim.x - n_ang) * DTS_THREADS;
    const int MS1 = A.ms_max + 1, ncol = (A.mb_max + 1) * MS1;
    const int L = A.l_max;
    if (i0 == 0) *next = 0;
    // column c's prefactor on CTA c mod n_cta, thread c / n_cta: a few per CTA, so that the
    // double-double work is spread over all schedulers (32 warps of one CTA doing it
    // share four schedulers and take ~8 us)
    const int n_cta = (int)gridDim.x - n_ang;
    for (long long i = (long long)threadIdx.x * n_cta + (blockIdx.x - n_ang); i < ncol;
         i += (long long)DTS_THREADS * n_cta) {
        const int mb = (int)i / MS1, ms = (int)i - mb * MS1;
        DtCol c;
        c.pre = seed_prefactor(mb, ms, T);
        c.pre_hi = __double2float_rn(c.pre.hi);
        c.pre_lo = __double2float_rn((c.pre.hi - (double)c.pre_hi) + c.pre.lo);
        cols[i] = c;
    }
    if (L == 0) return;
    for (long long e = i0; e < (long long)ncol * L; e += stride) {
        const int c = (int)(e / L), l = (int)(e - (long long)c * L);
        const int mb = c / MS1, ms = c - mb * MS1;
        if (l >= (mb > ms ? mb : ms)) {
            double f0, g, f2;
            lrec_coefficients(l, mb, ms, T, f0, g, f2);
            cf.f0[e] = f0;
            cf.g[e] = g;
            cf.f2[e] = f2;
        }
    }
}

// The seed of chain (mb, ms) at one angle as a scaled double (value = mant 2^(90 n);
// plain when the value is >= 2^-810): x = ln|d^{l0}| in double, x = k ln 2 + r, e^r in
// float-float.  dd_path: the double-double seed of the fused kernels instead
// (warp-uniform; taken where |x| may reach 2^20 ln 2).
__device__ __forceinline__ Scaled dtable_seed(int mb, int ms, const DtAngle &a, const DtCol &col, bool dd_path) {
    if (dd_path) return seed_value_from(col.pre, mb, ms, a.t);
    const int l0 = mb > ms ? mb : ms;
    const int m = mb > ms ? ms : mb;
    const int p = l0 + m, q = l0 - m;
    Scaled s;
    if ((p > 0 && a.t.c_zero) || (q > 0 && a.t.s_zero)) {
        s.mant = 0.0;
        s.n = 0;
        s.plain = true;
        return s;
    }
    const double lp = p > 0 ? (double)p * a.t.lnc : 0.0;
    const double t = q > 0 ? fma((double)q, a.t.lns, lp) : lp;
    const double x = (t + col.pre.lo) + col.pre.hi;
    const double kd = rint(x * WG_INV_LN2);
    const double r = fma(-kd, WG_LN2_LO, fma(-kd, WG_LN2_HI, x));  // |r| <= ln 2 / 2 + a little
    const ff rf = (biased_exp(r) >= 1023 - 100) ? split_ff(r) : ff{0.0f, 0.0f};  // e^r = 1 below 2^-100
    const ff e = ff_exp_reduced(rf);                                            // in [0.70, 1.42]
    double mant = ff_to_double(e.hi, e.lo);
    if (mb > ms && (q & 1)) mant = -mant;
    const int kk = (int)kd;
    const int n = kk >= 0 ? kk / 90 : -((-kk + 89) / 90);  // floor(kk / 90)
    if (n >= WG_PLAIN_MIN_N) {  // >= 2^-810: a normal double
        s.mant = exp_shift(mant, kk);
        s.n = 0;
        s.plain = true;
    } else {
        s.mant = exp_shift(mant, kk - 90 * n);  // in [0.7, 2^90)
        s.n = n;
        s.plain = false;
    }
    return s;
}

constexpr int DT_WARPS = 4;  // warps per CTA of the persistent grid

// YLM: each d^l is stored times sqrt((2l+1)/(4 pi)): with ms_max = 0 the table is then the
// theta part of the spherical harmonics, Y_l^m(theta, phi) = sqrt((2l+1)/(4 pi)) d^l_{m0}(theta)
// e^{i m phi} (the Condon-Shortley phase comes with d).
template <bool YLM>
__global__ void __launch_bounds__(32 * DT_WARPS) dtable_fp64_kernel(DTableArgs A, Tables T, const DtAngle *ang,
                                                                          const DtCol *cols, DtCoef cf, int *next,
                                                                          int n_items, int n_chunks) {
    __shared__ double sF0[DT_WARPS][32], sG[DT_WARPS][32], sF2[DT_WARPS][32], sN[DT_WARPS][YLM ? 32 : 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int MS1 = A.ms_max + 1;
    const int L = A.l_max;
    const size_t NB = (size_t)A.n_beta;
    int it_next = -1;  // lane 0: the item taken during the last tile of the current one
    for (;;) {
        int it = 0;
        if (lane == 0) it = it_next >= 0 ? it_next : atomicAdd(next, 1);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        it_next = -1;
        const int cidx = it / n_chunks, chunk = it - cidx * n_chunks;
        int mb, ms;
        column_of(cidx, A.mb_max, A.ms_max, mb, ms);
        const int col = mb * MS1 + ms;
        const int l0 = mb > ms ? mb : ms;
        const int m = mb > ms ? ms : mb;
        const int j = chunk * 32 + lane;
        const bool valid = j < A.n_beta;
        const DtAngle a = ang[valid ? j : 0];
        const DtCol cc = cols[col];
        // the seed: the double-double form only where the logarithm may be huge
        const float big = fabsf(cc.pre_hi) + (float)(l0 + m) * fabsf(a.lnc_hi) + (float)(l0 - m) * fabsf(a.lns_hi);
        const bool dd_path = __any_sync(0xffffffffu, valid && big > 700000.0f);
        const Scaled sd = dtable_seed(mb, ms, a, cc, dd_path);
        double cur = a.t.bad ? __longlong_as_double(0x7ff8000000000000LL) : sd.mant;
        double prev = 0.0;
        int n = a.t.bad ? 0 : sd.n;
        bool plain = a.t.bad ? true : sd.plain;

        double *out = A.d_out + (size_t)col * (size_t)(L + 1) * NB;
        // the coefficients of a tile: lane i holds order ts + i, loaded one tile ahead
        const size_t cbase = (size_t)col * L;
        double nf0 = 0.0, ng = 0.0, nf2 = 0.0;
        if (l0 + lane < L) {
            nf0 = cf.f0[cbase + l0 + lane];
            ng = cf.g[cbase + l0 + lane];
            nf2 = cf.f2[cbase + l0 + lane];
        }
        for (int ts = l0; ts <= L; ts += 32) {
            __syncwarp();  // the previous tile's coefficients have been read
            sF0[w][lane] = nf0;
            sG[w][lane] = ng;
            sF2[w][lane] = nf2;
            if (YLM) sN[w][lane] = sqrt((double)(2 * (ts + lane) + 1) * WG_INV_4PI);
            __syncwarp();
            const int ln = ts + 32 + lane;
            nf0 = ng = nf2 = 0.0;
            if (ln < L) {
                nf0 = cf.f0[cbase + ln];
                ng = cf.g[cbase + ln];
                nf2 = cf.f2[cbase + ln];
            }
            const int nl = min(32, L + 1 - ts);
            // the last tile: take the next item now, its atomic's latency hidden by the steps
            if (lane == 0 && ts + 32 > L) it_next = atomicAdd(next, 1);
            for (int i = 0; i < nl; ++i) {
                const int l = ts + i;
                if (valid) {
                    const double v = plain ? cur : scaled_store(cur, n);
                    out[(size_t)l * NB + j] = YLM ? v * sN[w][i] : v;
                }
                if (l < L) {
                    const double y = fma(sF0[w][i], a.t.cb, -sG[w][i]);
                    const double nx = fma(y, cur, -(sF2[w][i] * prev));
                    prev = cur;
                    cur = nx;
                    if (!plain) scaled_fixup(cur, prev, n, plain);
                }
            }
        }
        // The zeros of rows l < l0, written after the chain for another column: the item of
        // (mb, ms), ms >= 1, zeroes column (mb, ms_max + 1 - ms) (a bijection of 1..ms_max),
        // the item of (mb, 0) its own.  Items run longest chain first, and the columns with
        // the longest chains have the fewest zero rows; paired this way the early items
        // write the many zeros and the short items at the end of the queue few, instead of
        // ending the kernel with stores while the FP64 pipe idles.
        {
            const int msz = ms == 0 ? 0 : A.ms_max + 1 - ms;
            const int zn = mb > msz ? mb : msz;
            double *z = A.d_out + (size_t)(mb * MS1 + msz) * (size_t)(L + 1) * NB + j;
            if (valid)
                for (int l = 0; l < zn; ++l) z[(size_t)l * NB] = 0.0;
        }
        if (A.counters && lane == 0) {
            const int nvalid = min(32, A.n_beta - chunk * 32);
            atomicAdd(&A.counters[0], (unsigned long long)nvalid * (unsigned long long)(L + 1 - l0));
        }
    }
}

// CTAs of the persistent grid per SM
constexpr int DT_BLOCKS_PER_SM = 2;

template <bool YLM>
static int launch_dtable_t(const DTableArgs &a, const Tables &t, void *stream) {
    if (a.n_beta == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    const int ncol = (a.mb_max + 1) * (a.ms_max + 1);
    const int n_chunks = (a.n_beta + 31) / 32;
    const long long n_items = (long long)ncol * n_chunks;
    if (n_items > INT_MAX) return (int)cudaErrorInvalidValue;
    int dev = 0, n_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    // stream-ordered scratch: the item counter, the angles' and the columns' set-up values
    cudaMemPool_t pool;
    if (host_pool(&pool) != WG_OK) return (int)cudaErrorMemoryAllocation;
    const size_t off_ang = 256, off_col = off_ang + (((size_t)a.n_beta * sizeof(DtAngle) + 255) / 256) * 256;
    const size_t off_cf = off_col + (((size_t)ncol * sizeof(DtCol) + 255) / 256) * 256;
    const size_t n_cf = (size_t)ncol * a.l_max;  // entries of each coefficient array
    const size_t bytes = off_cf + 3 * n_cf * sizeof(double);
    char *sc = nullptr;
    e = alloc_injected() ? cudaErrorMemoryAllocation : cudaMallocFromPoolAsync((void **)&sc, bytes, pool, s);
    if (e != cudaSuccess) return (int)e;
    int *next = reinterpret_cast<int *>(sc);
    DtAngle *ang = reinterpret_cast<DtAngle *>(sc + off_ang);
    DtCol *cols = reinterpret_cast<DtCol *>(sc + off_col);
    DtCoef cf;
    cf.f0 = reinterpret_cast<double *>(sc + off_cf);
    cf.g = cf.f0 + n_cf;
    cf.f2 = cf.g + n_cf;
    // the set-up grid: one CTA per SM, the first n_ang of them for the angles (4 chunks of 32
    // angles each per pass), at most half the SMs
    int n_ang = (n_chunks + 3) / 4;
    if (n_ang > n_sm / 2) n_ang = n_sm / 2 > 1 ? n_sm / 2 : 1;
    const int setup_grid = n_sm > n_ang + 1 ? n_sm : n_ang + 1;
    dtable_setup_kernel<<<(unsigned)setup_grid, DTS_THREADS, 0, s>>>(a, t, ang, cols, cf, next, n_ang);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        long long grid = (long long)n_sm * DT_BLOCKS_PER_SM;
        const long long need = (n_items + DT_WARPS - 1) / DT_WARPS;
        if (grid > need) grid = need;
        dtable_fp64_kernel<YLM><<<(unsigned)grid, 32 * DT_WARPS, 0, s>>>(a, t, ang, cols, cf, next, (int)n_items,
                                                                         n_chunks);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(sc, s);
    return (int)(e != cudaSuccess ? e : ef);
}

int launch_dtable_fp64(const DTableArgs &a, const Tables &t, void *stream) { return launch_dtable_t<false>(a, t, stream); }

// out[m][l][j] = sqrt((2l+1)/(4 pi)) d^l_{m0}(theta_j) (a.ms_max must be 0)
int launch_ylm(const DTableArgs &a, const Tables &t, void *stream) { return launch_dtable_t<true>(a, t, stream); }

}  // namespace wg
