// wg_conv_fp64.cu -- fused l-recursion + weighted l-sum in IEEE double
// (Sec. 4.1 Eq. convdef evaluated with the Sec. 3.2 recursion, Sec. 4.2.2 tables).
//
// Work decomposition
//   A work item = (a group of G consecutive chain columns, a chunk of NT*CPT angles).
//   Columns k are ordered m_sky-major (k = ms*(mb_max+1) + mb), so low k means a low
//   start l0 = max(mb, ms) and a long chain; blockIdx.x walks the items in that
//   order, longest first.  Each thread holds CPT chains (angles j = chunk*NT*CPT +
//   c*NT + tid, c < CPT, so each warp's lanes hold consecutive angles) and keeps its
//   per-angle quantities (cos beta, half-angle logs) in registers across the G columns.
//   For each column the CTA walks l in tiles of TL: it builds the coefficient table
//   (F0, F0*F1, F2) and the weights w_l = conj(b_{l,mb}) a_{l,ms} of the tile in
//   shared memory once, and every chain of the CTA reads them as broadcasts.
//
// Per element (chain, l): y = fma(F0, cos b, -G), d' = fma(y, d, -(F2 d_prev))
// (three FP64 instructions), then, from the first |d| >= 1e-30 on (Sec. 4.2.1),
// C += w_l d (two FP64 FMAs).  The threshold test, the scaled-double bookkeeping
// and the switch to plain doubles (Sec. 3.2) are integer operations on the
// exponent field, so the FP64 pipe -- the scarce unit of this GPU -- only sees the
// five arithmetic instructions.  A warp skips the sum only while none of its
// chains has crossed the threshold.
#pragma once

#include <cuda_runtime.h>

#include "wg_common.cuh"

namespace wg {

template <int TL>
struct SmemFp64 {
    double2 sFG[TL];  // (F0, G)
    double2 sFW[TL];  // (F2, w_re)
    double sWI[TL];   // w_im
};

// One work item: chain columns k in [k_begin, k_end) (m_sky-major order) for the
// angle chunk `chunk` (NT*CPT angles).  Adds the elements evaluated and summed to the
// counters.  Every thread of the CTA must call it (it synchronises the CTA).
template <int NT, int CPT, int TL>
__device__ __forceinline__ void conv_fp64_item(const ConvArgs &A, const Tables &T, int chunk, int k_begin,
                                               int k_end, SmemFp64<TL> &sm, unsigned long long &n_elem,
                                               unsigned long long &n_sum) {
    const int MB1 = A.mb_max + 1;
    const int L = A.l_max;
    const int NB = A.n_beta;
    const int tid = threadIdx.x;
    double2 *sFG = sm.sFG;
    double2 *sFW = sm.sFW;
    double *sWI = sm.sWI;

    int jj[CPT];
    bool valid[CPT];
    Angle ang[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        jj[c] = chunk * NT * CPT + c * NT + tid;
        valid[c] = jj[c] < NB;
        ang[c] = make_angle(valid[c] ? A.beta[jj[c]] : 1.0);
        if (valid[c] && ang[c].bad) raise_status(T.status, WG_DEVERR_BETA);
    }
    const long long eps_bits = __double_as_longlong(WG_EPS_SUM);

    for (int k = k_begin; k < k_end; ++k) {
        const int ms = k / MB1, mb = k - ms * MB1;
        const int l0 = mb > ms ? mb : ms;

        double cur[CPT], prev[CPT], cre[CPT], cim[CPT];
        int nsc[CPT];
        bool plain[CPT], summing[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const Scaled s = seed_value(mb, ms, ang[c], T);
            cur[c] = s.mant;
            nsc[c] = s.n;
            plain[c] = s.plain;
            prev[c] = 0.0;
            cre[c] = 0.0;
            cim[c] = 0.0;
            summing[c] = false;
        }
        bool warp_sum = false;

        for (int ts = l0; ts <= L; ts += TL) {
            __syncthreads();
            for (int i = tid; i < TL; i += NT) {
                const int l = ts + i;
                double f0 = 0.0, g = 0.0, f2 = 0.0, wre = 0.0, wim = 0.0;
                if (l <= L) {
                    if (l < L) lrec_coefficients(l, mb, ms, T, f0, g, f2);
                    const double2 av = reinterpret_cast<const double2 *>(A.a)[(size_t)l * (A.ms_max + 1) + ms];
                    const double2 bv = reinterpret_cast<const double2 *>(A.b)[(size_t)l * MB1 + mb];
                    wre = bv.x * av.x + bv.y * av.y;  // conj(b) * a
                    wim = bv.x * av.y - bv.y * av.x;
                }
                sFG[i] = make_double2(f0, g);
                sFW[i] = make_double2(f2, wre);
                sWI[i] = wim;
            }
            __syncthreads();
            const int nl = min(TL, L + 1 - ts);
            for (int i = 0; i < nl; ++i) {
                const double2 fg = sFG[i];
                const double2 fw = sFW[i];
                const double wim = sWI[i];
                // term l: start summing at the first |d| >= eps (plain values only)
                bool any = false;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    summing[c] = summing[c] || (plain[c] && abs_ge(cur[c], eps_bits));
                    any |= summing[c];
                }
                if (!warp_sum) warp_sum = __any_sync(0xffffffffu, any);
                if (warp_sum) {
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        const double wr = summing[c] ? fw.y : 0.0;
                        const double wi = summing[c] ? wim : 0.0;
                        cre[c] = fma(wr, cur[c], cre[c]);
                        cim[c] = fma(wi, cur[c], cim[c]);
                        n_sum += (summing[c] && valid[c]) ? 1 : 0;
                    }
                }
                if (ts + i < L) {
#pragma unroll
                    for (int c = 0; c < CPT; ++c) {
                        const double y = fma(fg.x, ang[c].cb, -fg.y);
                        const double nx = fma(y, cur[c], -(fw.x * prev[c]));
                        prev[c] = cur[c];
                        cur[c] = nx;
                        if (!plain[c]) scaled_fixup(cur[c], prev[c], nsc[c], plain[c]);
                    }
                }
            }
        }
        double2 *out = reinterpret_cast<double2 *>(A.c_out) + ((size_t)mb * (A.ms_max + 1) + ms) * NB;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            if (valid[c]) {
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                out[jj[c]] = ang[c].bad ? make_double2(nan, nan) : make_double2(cre[c], cim[c]);
                n_elem += (unsigned long long)(L + 1 - l0);
            }
        }
    }
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
