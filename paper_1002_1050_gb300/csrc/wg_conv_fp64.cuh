// wg_conv_fp64.cuh -- fused l-recursion + weighted l-sum in IEEE double
// (Sec. 4.1 Eq. convdef evaluated with the Sec. 3.2 recursion, Sec. 4.2.2 tables).
//
// Work decomposition
//   A work item = (a group of G consecutive chain columns, a chunk of NT*CPT angles).
//   Columns k are ordered m_sky-major (k = ms*(mb_max+1) + mb), so low k means a low
//   start l0 = max(mb, ms) and a long chain; blockIdx.x walks the items in that
//   order, longest first.  Each thread holds CPT chains; a warp holds 32*CPT
//   consecutive angles (lane i: j0 + i and j0 + 32 + i for CPT = 2), and every thread
//   keeps its per-angle quantities (cos beta, half-angle logs) in registers across
//   the G columns.  For each column the CTA walks l in tiles of TL: it builds the
//   coefficient table and the weights w_l = conj(b_{l,mb}) a_{l,ms} of the tile in
//   shared memory once, and every chain of the CTA reads them as broadcasts.
//
// Per element (chain, l): the chain is carried normalised, u^l = d^l / sigma_l, so
// Eq. lrec takes two FP64 FMAs, y = fma(F0', cos b, -G'), u' = fma(y, u, -u_prev);
// then, from the first |d| >= 1e-30 on (Sec. 4.2.1), C += (w_l sigma_l) u (two FP64
// FMAs).  The threshold test, the scaled-double bookkeeping and the switch to plain
// doubles (Sec. 3.2) are integer operations on the exponent field, so the FP64 pipe --
// the scarce unit of this GPU -- sees only these FMAs.  A warp skips the sum only while
// none of its chains has crossed the threshold; with consecutive angles in a warp the
// crossings lie close together.
#pragma once

#include <cuda_runtime.h>

#include "wg_common.cuh"
#include "wg_tma.cuh"

namespace wg {

// ===========================================================================
// The FP64 kernels: two FP64 instructions per recursion step.
//
// The chain is carried as u^l = d^l / sigma_l with sigma_{l0} = sigma_{l0+1} = 1 and
// sigma_{l+1} = F2_l sigma_{l-1}; then Eq. lrec reads
//     u^{l+1} = (F0'_l cos b - G'_l) u^l - u^{l-1},   F0' = F0 rho_l, G' = G rho_l,
//     rho_l = sigma_l / sigma_{l+1},
// so a step is two FP64 FMAs (the F2 d^{l-1} product of the plain form disappears into
// the normalisation; sigma_{l+1} = fl(F2_l sigma_{l-1}) is formed in the same order as
// that product would be, so the rounding per step is unchanged).  The term
// w_l d^l = (w_l sigma_l) u^l is summed
//   * SUM_FF = false: with two FP64 FMAs (every operation IEEE double: form WG_FP64);
//   * SUM_FF = true: in float-float on the FP32 pipe, u split into two floats by integer
//     operations (form WG_FP64S), so the FP64 pipe -- 2 lanes per clock per SM on
//     GB300 -- runs only the recursion; the float-float products and sums are ~48-bit
//     accurate, far below the FP64 path's 1e-11 bar on C.
// sigma_l is a product of the F2 coefficients along each parity of l (between 0.01 and
// 1 for the orders used), computed per l-tile by one thread and applied to the tile's
// tables.  The threshold |d| >= 1e-30 of Sec. 4.2.1 becomes |u| >= 1e-30 / sigma_l.
// ===========================================================================
template <int TL>
struct SmemFp64 {
    double2 sA[TL];        // (F0', G')   (phase 1: (F0, G))
    double2 sWd[TL];       // w_l = conj(b) a (phase 1), then w_l sigma_l
    float4 sW[TL];         // w_l sigma_l as float-float (re hi, lo, im hi, lo)
    double2 sWnd[TL];      // FULL: weights of the order -m_sky at pi - beta (then times sigma_l)
    float4 sWn[TL];        // FULL: the same as float-float
    long long sT[TL];      // bit pattern of 1e-30 / sigma_l
    double sF2[TL];        // F2_l (phase 1)
    double sSig[TL + 1];   // sigma_{ts + i}
};

// TMA staging of the weights: two buffers of the l-tile's a and b boxes (the tile after
// next is requested as soon as a buffer's tile has been read), one mbarrier each.
template <int TL>
struct SmemTma {
    alignas(128) double2 sAw[2][TL];
    alignas(128) double2 sBw[2][TL];
    unsigned long long mbar[2];
};

__device__ __forceinline__ void dbl_to_ff(double x, float &hi, float &lo) {
    hi = __double2float_rn(x);
    lo = __double2float_rn(x - (double)hi);
}

// The l_min cut of Sec. 4.2.1 (Eq. lmin, its approximate line): the chain (m_b, m_sky,
// beta) sums from l_min = (sqrt(q) - offset) / sin beta, q = m_sky^2 + m_b^2 -
// 2 m_sky m_b cos beta; the terms below lie in the non-classical region.  At sin beta = 0
// (beta = 0, d = delta) the chain is left out unless m_b = m_sky.  Returns the first l of
// the sum, l0 (nothing cut) up to L + 1 (the whole chain cut).  Every operation is
// rounded once, without contraction.  The chain's mirror (m_b, -m_sky, pi - beta) has
// the same q and sin, so one value serves both halves of the sum over every sky order.
__device__ __forceinline__ int lmin_first(int L, int l0, int mb, int ms, const Angle &t, double offset) {
    if (t.sb == 0.0) return mb == ms ? l0 : L + 1;
    const double q0 = __dadd_rn(__dmul_rn((double)mb, (double)mb), __dmul_rn((double)ms, (double)ms));
    const double q = __dsub_rn(q0, __dmul_rn(__dmul_rn(__dmul_rn(2.0, (double)mb), (double)ms), t.cb));
    const double x = __ddiv_rn(__dsub_rn(__dsqrt_rn(q), offset), t.sb);
    if (!(x <= (double)L)) return L + 1;
    if (x <= (double)l0) return l0;
    return (int)ceil(x);
}

// The outputs of column k (and, FULL, of its mirrored order) for this thread's chains
// set to NaN: the column was abandoned after a bounded wait gave up.
template <int CPT, bool FULL>
__device__ __forceinline__ void abandon_column(const ConvArgs &A, int k, const int *jj, const bool *valid) {
    const int MB1 = A.mb_max + 1;
    const int ms = k / MB1, mb = k - ms * MB1;
    const int NB = A.n_beta;
    const size_t NS = FULL ? (size_t)2 * A.ms_max + 1 : (size_t)A.ms_max + 1;
    const size_t col = (size_t)mb * NS + (FULL ? (size_t)(A.ms_max + ms) : (size_t)ms);
    double2 *out = reinterpret_cast<double2 *>(A.c_out) + col * NB;
    double2 *outn = reinterpret_cast<double2 *>(A.c_out) + ((size_t)mb * NS + (size_t)(A.ms_max - ms)) * NB;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        if (!valid[c]) continue;
        out[jj[c]] = make_double2(nan, nan);
        if (FULL && ms > 0) outn[NB - 1 - jj[c]] = make_double2(nan, nan);
    }
}

// TMA: the weights arrive by TMA (wm, st; the mbarriers initialised by the caller, their
// phases in ph), else by plain loads.  Returns false if a TMA wait gave up after
// A.wait_tries tries: the status word then has WG_DEVERR_TIMEOUT, the copies already
// issued have been waited for (default limit), and the outputs of the abandoned
// columns of this CTA's chains are NaN.
// FULL: the sum over every sky order (the data cube of Sec. 4.1, m_sky from -ms_max to
// ms_max) for a mirror-symmetric angle grid (beta_{N-1-j} = pi - beta_j).  The chain of
// (m_b, m_sky) at beta_j also gives the order -m_sky at pi - beta_j through the
// appendix identity d^l_{m,-m'}(pi - beta) = (-1)^{l+m} d^l_{m m'}(beta) (corrected
// sign): a second weighted sum with w^-_l = conj(b_{l m_b}) s_{l,-m_sky} (-1)^{l+m_b},
// s_{l,-m} = (-1)^m conj(s_{l m}) for a real sky.  c_out is then [m_b][m_sky + ms_max][j].
// LMIN: the sum of each chain starts at lmin_first (offset A.offset); a CTA whose chains
// are all cut skips the column (no tables, no copies), a warp whose chains are all cut
// skips its recursion steps, and a cut chain's C is 0.
template <int NT, int CPT, int TL, bool SUM_FF, bool TMA = false, bool FULL = false, bool LMIN = false>
__device__ __forceinline__ bool conv_fp64_item(const ConvArgs &A, const Tables &T, int chunk, int k_begin,
                                                 int k_end, SmemFp64<TL> &sm, unsigned long long &n_elem,
                                                 unsigned long long &n_sum, const WeightMaps *wm = nullptr,
                                                 SmemTma<TL> *st = nullptr, unsigned *ph = nullptr) {
    const int MB1 = A.mb_max + 1;
    const int L = A.l_max;
    const int NB = A.n_beta;
    const int tid = threadIdx.x;

    int jj[CPT];
    bool valid[CPT];
    Angle ang[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        // a warp's chains lie close together in sin(beta), so their 1e-30 crossings (at
        // l ~ m_sky / sin(beta); with LMIN, their cuts) do too: the warp starts its sum
        // late when all its chains do, and a cut tends to remove whole warps.  With two
        // chains and the sum in double a thread takes the angles j and N-1-j (pi - beta_j
        // on a symmetric grid, the same sin(beta)), a warp 32 consecutive j of the grid's
        // first half (measured 940.3 ms against 947.8 ms at the L = 4096 workload; the
        // split-pipe form measured 618.9 against 615.5 ms and keeps the other map); else a
        // warp takes 32 CPT consecutive angles.
        if (CPT == 2 && !SUM_FF) {
            const int jl = chunk * NT + tid;
            jj[c] = c == 0 ? jl : NB - 1 - jl;
            valid[c] = 2 * jl + c < NB;  // jl < N - 1 - jl for the second chain (the middle angle once)
        } else {
            jj[c] = chunk * NT * CPT + (tid >> 5) * (32 * CPT) + c * 32 + (tid & 31);
            valid[c] = jj[c] < NB;
        }
        ang[c] = make_angle(valid[c] ? A.beta[jj[c]] : 1.0);
        if (valid[c] && ang[c].bad) raise_status(T.status, WG_DEVERR_BETA);
    }

    for (int k = k_begin; k < k_end; ++k) {
        const int ms = k / MB1, mb = k - ms * MB1;
        const int l0 = mb > ms ? mb : ms;

        double u[CPT], up[CPT], cre[CPT], cim[CPT], nre[CPT], nim[CPT];
        ff are[CPT], aim[CPT], bre[CPT], bim[CPT];
        int nsc[CPT], lsum[CPT];
        bool plain[CPT], summing[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const Scaled s = seed_value(mb, ms, ang[c], T);
            u[c] = s.mant;  // sigma_{l0} = 1
            nsc[c] = s.n;
            plain[c] = s.plain;
            up[c] = 0.0;
            cre[c] = 0.0;
            cim[c] = 0.0;
            are[c] = ff{0.f, 0.f};
            aim[c] = ff{0.f, 0.f};
            nre[c] = nim[c] = 0.0;
            bre[c] = bim[c] = ff{0.f, 0.f};
            summing[c] = false;
            lsum[c] = L + 1;
        }
        int lfirst[CPT];
        bool cta_live = true, warp_live = true;
        if (LMIN) {
            bool live = false;
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                lfirst[c] = lmin_first(L, l0, mb, ms, ang[c], A.offset);
                live |= valid[c] && lfirst[c] <= L;
            }
            cta_live = __syncthreads_or(live);
            warp_live = __any_sync(0xffffffffu, live);
        }
        bool warp_sum = false;
        double sig_m1 = 0.0, sig_0 = 1.0;  // thread 0's carry: sigma_{ts-1}, sigma_{ts}
        bool inflight[2] = {false, false};  // TMA: a tile requested and not yet waited for
        if (TMA && cta_live) {
            if (tid == 0) {
                tma_weights<TL>(wm, mb, ms, l0, st->sAw[0], st->sBw[0], &st->mbar[0]);
                if (l0 + TL <= L) tma_weights<TL>(wm, mb, ms, l0 + TL, st->sAw[1], st->sBw[1], &st->mbar[1]);
            }
            inflight[0] = true;
            inflight[1] = l0 + TL <= L;
        }

        int tix = 0;
        for (int ts = l0; cta_live && ts <= L; ts += TL, ++tix) {
            const int buf = tix & 1;
            bool ok = true;
            if (TMA) {
                ok = mbar_wait(&st->mbar[buf], ph[buf], A.wait_tries);
                if (ok) {
                    inflight[buf] = false;
                    ph[buf] ^= 1u;
                }
            }
            if (!__syncthreads_and(ok)) {
                // a TMA wait gave up: record it, let the copies already issued land (each
                // drain wait with the default limit, whatever the launch's limit), mark
                // this column and the group's later columns NaN for this CTA's chains,
                // and leave
                if (tid == 0) {
                    raise_status(T.status, WG_DEVERR_TIMEOUT);
                    for (int b2 = 0; b2 < 2; ++b2)
                        if (inflight[b2] && mbar_wait(&st->mbar[b2], ph[b2], TMA_WAIT_ITERS)) ph[b2] ^= 1u;
                }
                __syncthreads();
                for (int k2 = k; k2 < k_end; ++k2) abandon_column<CPT, FULL>(A, k2, jj, valid);
                return false;
            }
            for (int i = tid; i < TL; i += NT) {  // phase 1: F0, G, F2, w
                const int l = ts + i;
                double f0 = 0.0, g = 0.0, f2 = 0.0;
                double2 w = make_double2(0.0, 0.0), wn = make_double2(0.0, 0.0);
                if (l <= L) {
                    if (l < L) lrec_coefficients(l, mb, ms, T, f0, g, f2);
                    double2 av, bv;
                    if (TMA) {
                        av = st->sAw[buf][i];
                        bv = st->sBw[buf][i];
                    } else {
                        av = reinterpret_cast<const double2 *>(A.a)[(size_t)l * (A.ms_max + 1) + ms];
                        bv = reinterpret_cast<const double2 *>(A.b)[(size_t)l * MB1 + mb];
                    }
                    w = make_double2(bv.x * av.x + bv.y * av.y, bv.x * av.y - bv.y * av.x);
                    if (FULL) {  // (-1)^{l + m_b + m_sky} conj(b a)
                        const double sg = ((l + mb + ms) & 1) ? -1.0 : 1.0;
                        wn = make_double2(sg * (bv.x * av.x - bv.y * av.y), -sg * (bv.x * av.y + bv.y * av.x));
                    }
                }
                sm.sA[i] = make_double2(f0, g);
                sm.sF2[i] = f2;
                sm.sWd[i] = w;
                if (FULL) sm.sWnd[i] = wn;
            }
            __syncthreads();
            if (TMA && ts + 2 * TL <= L) {  // this buffer has been read: request the tile after next
                if (tid == 0) tma_weights<TL>(wm, mb, ms, ts + 2 * TL, st->sAw[buf], st->sBw[buf], &st->mbar[buf]);
                inflight[buf] = true;
            }
            if (tid == 0) {  // phase 2: sigma_{ts+i}, i = 0..TL
                double sm1 = sig_m1, s0 = sig_0;
                sm.sSig[0] = s0;
                for (int i = 0; i < TL; ++i) {
                    const int l = ts + i;
                    double nx;
                    if (l == l0 || l >= L)
                        nx = s0;  // sigma_{l0+1} = 1; past l_max: unused, kept finite
                    else
                        nx = sm.sF2[i] * sm1;
                    sm.sSig[i + 1] = nx;
                    sm1 = s0;
                    s0 = nx;
                }
                sig_m1 = sm1;
                sig_0 = s0;
            }
            __syncthreads();
            for (int i = tid; i < TL; i += NT) {  // phase 3: normalised tables
                const int l = ts + i;
                const double sg = sm.sSig[i];
                double2 fg = sm.sA[i];
                if (l < L) {
                    const double rho = sg / sm.sSig[i + 1];
                    fg.x *= rho;
                    fg.y *= rho;
                }
                double2 w = sm.sWd[i];
                w.x *= sg;
                w.y *= sg;
                sm.sA[i] = fg;
                if (SUM_FF) {
                    float4 wf;
                    dbl_to_ff(w.x, wf.x, wf.y);
                    dbl_to_ff(w.y, wf.z, wf.w);
                    sm.sW[i] = wf;
                } else {
                    sm.sWd[i] = w;
                }
                if (FULL) {
                    double2 wn = sm.sWnd[i];
                    wn.x *= sg;
                    wn.y *= sg;
                    if (SUM_FF) {
                        float4 wf;
                        dbl_to_ff(wn.x, wf.x, wf.y);
                        dbl_to_ff(wn.y, wf.z, wf.w);
                        sm.sWn[i] = wf;
                    } else {
                        sm.sWnd[i] = wn;
                    }
                }
                sm.sT[i] = __double_as_longlong(WG_EPS_SUM / sg);
            }
            __syncthreads();
            const int nl = warp_live ? min(TL, L + 1 - ts) : 0;
            for (int i = 0; i < nl; ++i) {
                const double2 fg = sm.sA[i];
                const long long thr = sm.sT[i];
                bool any = false;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    if (!summing[c] && plain[c] && (!LMIN || ts + i >= lfirst[c]) && abs_ge(u[c], thr)) {
                        summing[c] = true;
                        lsum[c] = ts + i;
                    }
                    any |= summing[c];
                }
                if (!warp_sum) warp_sum = __any_sync(0xffffffffu, any);
                if (warp_sum) {
                    if (SUM_FF) {
                        const float4 w = sm.sW[i];
                        float4 wn;
                        if (FULL) wn = sm.sWn[i];
#pragma unroll
                        for (int c = 0; c < CPT; ++c) {
                            ff uu = split_ff(u[c]);
                            if (!summing[c]) uu = ff{0.f, 0.f};
                            ff_mac(are[c], w.x, w.y, uu.hi, uu.lo);
                            ff_mac(aim[c], w.z, w.w, uu.hi, uu.lo);
                            if (FULL) {
                                ff_mac(bre[c], wn.x, wn.y, uu.hi, uu.lo);
                                ff_mac(bim[c], wn.z, wn.w, uu.hi, uu.lo);
                            }
                        }
                    } else {
                        const double2 w = sm.sWd[i];
                        double2 wn;
                        if (FULL) wn = sm.sWnd[i];
#pragma unroll
                        for (int c = 0; c < CPT; ++c) {
                            const double um = summing[c] ? u[c] : 0.0;
                            cre[c] = fma(w.x, um, cre[c]);
                            cim[c] = fma(w.y, um, cim[c]);
                            if (FULL) {
                                nre[c] = fma(wn.x, um, nre[c]);
                                nim[c] = fma(wn.y, um, nim[c]);
                            }
                        }
                    }
                }
                if (ts + i < L) {
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        const double y = fma(fg.x, ang[c].cb, -fg.y);
                        const double nx = fma(y, u[c], -up[c]);
                        up[c] = u[c];
                        u[c] = nx;
                        if (!plain[c]) scaled_fixup(u[c], up[c], nsc[c], plain[c]);
                    }
                }
            }
        }
        // output columns: m_sky (and, FULL, -m_sky at the mirrored angle N-1-j)
        const size_t NS = FULL ? (size_t)2 * A.ms_max + 1 : (size_t)A.ms_max + 1;
        const size_t col = (size_t)mb * NS + (FULL ? (size_t)(A.ms_max + ms) : (size_t)ms);
        double2 *out = reinterpret_cast<double2 *>(A.c_out) + col * NB;
        double2 *outn = reinterpret_cast<double2 *>(A.c_out) + ((size_t)mb * NS + (size_t)(A.ms_max - ms)) * NB;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            if (valid[c]) {
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                double re = cre[c], im = cim[c];
                if (SUM_FF) {
                    re = (double)are[c].hi + (double)are[c].lo;
                    im = (double)aim[c].hi + (double)aim[c].lo;
                }
                out[jj[c]] = ang[c].bad ? make_double2(nan, nan) : make_double2(re, im);
                if (FULL && ms > 0) {
                    double nr = nre[c], ni = nim[c];
                    if (SUM_FF) {
                        nr = (double)bre[c].hi + (double)bre[c].lo;
                        ni = (double)bim[c].hi + (double)bim[c].lo;
                    }
                    // the mirrored angle must be pi - beta_j (to rounding): else NaN and a status bit
                    const int jm = NB - 1 - jj[c];
                    const double bm = A.beta[jm];
                    const bool mirror_ok = fabs(bm + A.beta[jj[c]] - WG_PI_HI) <= 1e-14;
                    if (!mirror_ok) raise_status(T.status, WG_DEVERR_GRID);
                    outn[jm] = (ang[c].bad || !mirror_ok) ? make_double2(nan, nan) : make_double2(nr, ni);
                }
                if (cta_live && warp_live) n_elem += (unsigned long long)(L + 1 - l0);
                n_sum += (unsigned long long)(L + 1 - min(lsum[c], L + 1));
            }
        }
    }
    return true;
}

// warp-aggregated counter update (one atomic per warp)
__device__ __forceinline__ void flush_counters(unsigned long long *counters, unsigned long long n_elem,
                                               unsigned long long n_sum) {
    if (!counters) return;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        n_elem += __shfl_down_sync(0xffffffffu, n_elem, off);
        n_sum += __shfl_down_sync(0xffffffffu, n_sum, off);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&counters[0], n_elem);
        atomicAdd(&counters[1], n_sum);
    }
}

}  // namespace wg
