// wg_matrix.cu -- rows of the whole matrix d^l(beta) at one l (the evaluator of Sec. 3.1:
// every d^l_{m m'}, -l <= m' <= l, for 0 <= m <= m_max at a batch of angles).
//
// Sec. 3.1 computes a row with the ratios d_{m m'} / d_{m,m'-1} of the three-term relation
// in m' (Eq. mrec), run downwards from m' = l and anchored at m' = 0 by d_{0 m}.  Sec. 2
// gives the stable direction of Eq. mrec: towards the classical band
//   m^2 + m'^2 - 2 m m' cos beta <= l (l + 1) sin^2 beta       (Eq. classiccond),
// whose centre is m' = m cos beta.  Below the band (m' < m cos beta minus its half-width,
// which happens for m > 0 when sin beta is small) the downward ratios are unstable, so
// here each row is run from BOTH edges towards the centre m* = round(m cos beta):
//   * m' = l, l-1, ..., m*     at beta, from the edge seed d^l_{m l}(beta), and
//   * m' = -l, ..., m* - 1     through d_{m,-k}(beta) = (-1)^{l+m} d_{m,k}(pi - beta), i.e. the
//     same downward run at pi - beta from d^l_{m l}(pi - beta), k = l, ..., 1 - m*.
// Both edge seeds are exact (Eqs. ini1-ini2 in log form, Sec. 3.2), so no anchor or ratio
// is needed; values below 2^-900 are carried as scaled doubles (mantissa, exponent of
// 2^90) exactly as in the l-recursion.  One step (Eq. mrec solved for d_{m,k-1}):
//   d_{k-1} = (2 (k cos x - m) / sin x) d_k / A_k - (C_k / A_k) d_{k+1},
//   A_k = sqrt((l+k)(l-k+1)),  C_k = sqrt((l-k)(l+k+1)),
// with k, 1/A_k and C_k/A_k per k in shared memory: two FMAs and two multiplies per element
// (1/A_k from the P_i table of Sec. 4.2.2, C_k/A_k with one square root per k and CTA).
//
// Work split: a CTA takes one angle, one side and 32 x W consecutive rows m; lane i of a
// warp runs row m0 + i.  All lanes start at k = l and their stops differ by at most
// 32 |cos beta|, so the lanes stay busy, and a single angle fills whole warps.  Each warp
// stages a tile of 32 orders x 32 rows in shared memory and stores it row by row: the
// per-angle layout [j][m][m' + l] then takes 32 consecutive doubles per store.
#include <cuda_runtime.h>

#include <string>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_internal.h"

namespace wg {

struct MatrixArgs {
    int l, m_max, n_beta;
    const double *beta;
    double *out;  // [j][m][m' + l]
    unsigned long long *counters;
};


constexpr int MX_TK = 32;  // orders per tile (= lanes, for the staged transpose)


template <int W>
__global__ void __launch_bounds__(32 * W) dmatrix_kernel(MatrixArgs A, Tables T) {
    const int j = blockIdx.x;
    const int side = blockIdx.z;  // 0: m' = l .. m* at beta; 1: m' = -l .. m*-1 via pi - beta
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int l = A.l;
    const int m0 = (blockIdx.y * W + warp) * 32;  // this warp's first row
    const int m = m0 + lane;
    const bool live = m <= A.m_max;
    const size_t NS = (size_t)(2 * l + 1);
    double *mat = A.out + (size_t)j * (size_t)(A.m_max + 1) * NS;  // this angle's matrix

    __shared__ double sK[MX_TK], sInvA[MX_TK], sCA[MX_TK];
    __shared__ double sStage[W][32][MX_TK + 1];
    __shared__ int sStop[W][32];
    __shared__ Angle sAng;

    if (threadIdx.x == 0) {  // one angle per CTA: its trigonometry once
        sAng = make_angle(A.beta[j]);
        if (side == 0 && blockIdx.y == 0 && sAng.bad) raise_status(T.status, WG_DEVERR_BETA);
    }
    __syncthreads();
    const Angle t = sAng;
    const int mstar = (int)rint((double)m * t.cb);  // centre of the classical band of row m
    Angle x = t;                                    // side 1: the mirrored angle pi - beta
    if (side) {
        x.cb = -t.cb;
        x.lnc = t.lns;
        x.lns = t.lnc;
        x.c_zero = t.s_zero;
        x.s_zero = t.c_zero;
    }
    const int stop = live ? (side ? 1 - mstar : mstar) : l + 1;  // k runs l, l-1, ..., stop
    sStop[warp][lane] = stop;
    const double nan = __longlong_as_double(0x7ff8000000000000LL);
    const bool pole = t.sb == 0.0;  // beta = 0: the identity, no recursion

    Scaled s = seed_value(live ? m : 0, l, x, T);  // d^l_{m l}(x)
    // the sign (-1)^{l+m} of side 1 rides on the seed (the recursion is linear)
    double cur = (side && ((l + m) & 1)) ? -s.mant : s.mant, prev = 0.0;  // d_k, d_{k+1}
    int n = s.n;
    bool plain = s.plain;
    const double s2 = 2.0 / x.sb;
    const double cxs = x.cb * s2, ms = (double)m * s2;

    for (int ts = l; __syncthreads_or(ts >= stop); ts -= MX_TK) {
        if (threadIdx.x < MX_TK) {
            const int kk = ts - threadIdx.x;
            double ia = 0.0, ca = 0.0;
            if (kk > -l && kk <= l) {  // 1/A_k = P_{l+k-1} P_{l-k}, P_i = 1/sqrt(i+1) (Sec. 4.2.2 table)
                ia = T.P[l + kk - 1] * T.P[l - kk];
                ca = sqrt((double)(l - kk) * (double)(l + kk + 1)) * ia;
            }
            sK[threadIdx.x] = (double)kk;
            sInvA[threadIdx.x] = ia;
            sCA[threadIdx.x] = ca;
        }
        __syncthreads();
        // lane: values of row m for k = ts, ts-1, ..., down to its stop, into the stage
        const int kend = max(ts - MX_TK + 1, stop);
        for (int k = ts; k >= kend; --k) {
            const int i = ts - k;
            double v;
            if (t.bad)
                v = nan;
            else if (pole)
                v = (side == 0 && k == m) ? 1.0 : 0.0;
            else
                v = plain ? cur : scaled_store(cur, n);
            sStage[warp][lane][i] = v;
            if (k > stop && !pole) {  // Eq. mrec for d_{k-1}
                const double b = fma(sK[i], cxs, -ms) * sInvA[i];
                const double nx = fma(b, cur, -(sCA[i] * prev));
                prev = cur;
                cur = nx;
                if (!plain) scaled_fixup(cur, prev, n, plain);
            }
        }
        __syncwarp();
        // the warp stores the tile row by row: lane = order k = ts - lane
        const int k = ts - lane;
        const size_t slot = (size_t)(side ? l - k : l + k);
        for (int r = 0; r < 32; ++r) {
            const int mr = m0 + r;
            if (mr > A.m_max) break;
            if (k >= sStop[warp][r] && k >= -l) mat[(size_t)mr * NS + slot] = sStage[warp][r][lane];
        }
        __syncwarp();
    }
    if (A.counters) {
        unsigned long long ne = live ? (unsigned long long)(l - stop + 1) : 0ull;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ne += __shfl_down_sync(0xffffffffu, ne, off);
        if (lane == 0 && ne) atomicAdd(&A.counters[0], ne);
    }
}

static int launch_dmatrix(const MatrixArgs &a, const Tables &t, cudaStream_t s) {
    constexpr int W = 4;
    if (a.n_beta == 0) return 0;
    dim3 grid(a.n_beta, (a.m_max + 1 + 32 * W - 1) / (32 * W), 2);
    dmatrix_kernel<W><<<grid, 32 * W, 0, s>>>(a, t);
    return (int)cudaGetLastError();
}

void set_last_error(const std::string &msg, int code);
int tables_for(int l_max, Tables *t);  // wg_capi.cu

}  // namespace wg

namespace {
int fail(int code, const std::string &msg) {
    wg::set_last_error(msg, code);
    return code;
}
}  // namespace

extern "C" int wigner_d_matrix(int l, int m_max, int n_beta, const double *beta, double *d_out,
                               wg_counter *counters, void *stream) {
    if (l < 0 || l > WG_LMAX) return fail(WG_ERR_ARG, "l must be in [0, WG_LMAX]");
    if (m_max < 0 || m_max > l) return fail(WG_ERR_ARG, "m_max must be in [0, l]");
    if (n_beta < 0) return fail(WG_ERR_ARG, "n_beta must be >= 0");
    if (n_beta == 0) return WG_OK;
    if (!beta || ((uintptr_t)beta & 7)) return fail(WG_ERR_ARG, "beta is NULL or not 8-byte aligned");
    if (!d_out || ((uintptr_t)d_out & 7)) return fail(WG_ERR_ARG, "d_out is NULL or not 8-byte aligned");
    if (counters && ((uintptr_t)counters & 7)) return fail(WG_ERR_ARG, "counters misaligned");
    wg::Tables t;
    int rc = wg::tables_for(l, &t);
    if (rc != WG_OK) return rc;
    wg::MatrixArgs a{l, m_max, n_beta, beta, d_out, counters};
    const int e = wg::launch_dmatrix(a, t, (cudaStream_t)stream);
    if (e != 0) {
        wg::set_last_error(std::string("dmatrix launch: ") + cudaGetErrorString((cudaError_t)e), WG_ERR_CUDA);
        return WG_ERR_CUDA;
    }
    return WG_OK;
}
