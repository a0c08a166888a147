// wg_multi.cu -- the fused sum for several weight columns at once (Sec. 4.1, Eq. convdef
// and its footnote: polarised maps and beams add the sums of the pairs (b^T, s^T),
// (b^G, s^G), (b^C, s^C); a Monte-Carlo run convolves many skies with one beam).
//
//   C^{(k)}_{m_b m_sky}(beta) = sum_l conj(b^{(k)}_{l m_b}) a^{(k)}_{l m_sky} d^l_{m_b m_sky}(beta),  k < n_col
//
// Every column shares the chains d^l, so one recursion (the normalised two-FMA form of
// the FP64 kernels) feeds K column sums: 2 + 2K FP64 FMAs per element instead of 4K
// (WG_FP64), or 2 FMAs plus K float-float sums on the FP32 pipe (WG_FP64S).  Columns go in
// passes of up to KMAX per launch.  A sum over the columns (the polarised total) is one
// column whose weight sum_k conj(b^{(k)}_l) a^{(k)}_l is formed in the tile tables, so it
// costs what a single column does.  The l-sum is a product D[beta x l] W[l x K]; in double
// precision it stays on the FMA pipes (GB300's FP64 tensor rate is far below them).
#include <cuda_runtime.h>

#include <string>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_conv_fp64.cuh"  // dbl_to_ff, flush_counters
#include "wg_internal.h"

namespace wg {

constexpr int KMAX = 4;

struct MultiArgs {
    int l_max, mb_max, ms_max, n_beta;
    const double *beta;
    const double2 *a;  // column k at a + k * sa: [l][ms]
    const double2 *b;  // column k at b + k * sb: [l][mb] (sb = 0: one beam for every column)
    double2 *c;        // column k at c + k * sc: [mb][ms][j]
    size_t sa, sb, sc;
    int k0;     // first column of this pass
    int n_col;  // COMBINE: the number of columns summed into one output
    unsigned long long *counters;
};

template <int TL, int K>
struct SmemMulti {
    double2 sA[TL];          // (F0', G')   (phase 1: (F0, G))
    double2 sWd[K][TL];      // w^{(k)}_l (phase 1), then times sigma_l
    float4 sW[K][TL];        // w^{(k)}_l sigma_l as float-float: (re hi, im hi, re lo, im lo)
    long long sT[TL];        // bit pattern of 1e-30 / sigma_l
    double sF2[TL];          // F2_l
    double sSig[TL + 1];     // sigma_{ts + i}
};

// K separate column sums per pass (COMBINE = false), or one sum of every column's
// product, sum_k conj(b_k) a_k, formed per l in the tile tables (COMBINE = true, K = 1).
template <int NT, int CPT, int TL, bool SUM_FF, int K, bool COMBINE>
__global__ void __launch_bounds__(NT) conv_multi_kernel(MultiArgs A, Tables T, int n_chunks, int group) {
    __shared__ SmemMulti<TL, K> sm;
    const int item = blockIdx.x;
    const int chunk = item % n_chunks;
    const int grp = item / n_chunks;
    const int MB1 = A.mb_max + 1;
    const int ncol = MB1 * (A.ms_max + 1);
    const int k_begin = grp * group;
    const int k_end = min(ncol, k_begin + group);
    const int L = A.l_max;
    const int NB = A.n_beta;
    const int tid = threadIdx.x;
    unsigned long long n_elem = 0, n_sum = 0;

    int jj[CPT];
    bool valid[CPT];
    Angle ang[CPT];
#pragma unroll
    for (int c = 0; c < CPT; ++c) {
        jj[c] = chunk * NT * CPT + (tid >> 5) * (32 * CPT) + c * 32 + (tid & 31);  // a warp: 64 angles in a row
        valid[c] = jj[c] < NB;
        ang[c] = make_angle(valid[c] ? A.beta[jj[c]] : 1.0);
        if (valid[c] && ang[c].bad) raise_status(T.status, WG_DEVERR_BETA);
    }

    for (int k = k_begin; k < k_end; ++k) {
        const int ms = k / MB1, mb = k - ms * MB1;
        const int l0 = mb > ms ? mb : ms;

        double u[CPT], up[CPT], cre[K][CPT], cim[K][CPT];
        float2 ahi[K][CPT], alo[K][CPT];  // float-float (re, im) sums
        int nsc[CPT], lsum[CPT];
        bool plain[CPT], summing[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const Scaled s = seed_value(mb, ms, ang[c], T);
            u[c] = s.mant;  // sigma_{l0} = 1
            nsc[c] = s.n;
            plain[c] = s.plain;
            up[c] = 0.0;
#pragma unroll
            for (int q = 0; q < K; ++q) {
                cre[q][c] = cim[q][c] = 0.0;
                ahi[q][c] = alo[q][c] = make_float2(0.f, 0.f);
            }
            summing[c] = false;
            lsum[c] = L + 1;
        }
        bool warp_sum = false;
        double sig_m1 = 0.0, sig_0 = 1.0;  // thread 0's carry: sigma_{ts-1}, sigma_{ts}

        for (int ts = l0; ts <= L; ts += TL) {
            __syncthreads();
            for (int i = tid; i < TL; i += NT) {  // phase 1: F0, G, F2, the K weights
                const int l = ts + i;
                double f0 = 0.0, g = 0.0, f2 = 0.0;
                if (l < L) lrec_coefficients(l, mb, ms, T, f0, g, f2);
                sm.sA[i] = make_double2(f0, g);
                sm.sF2[i] = f2;
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    double2 w = make_double2(0.0, 0.0);
                    if (l <= L) {
                        const int kb = COMBINE ? 0 : A.k0 + q, ke = COMBINE ? A.n_col : kb + 1;
                        for (int kk = kb; kk < ke; ++kk) {
                            const double2 av = A.a[kk * A.sa + (size_t)l * (A.ms_max + 1) + ms];
                            const double2 bv = A.b[kk * A.sb + (size_t)l * MB1 + mb];
                            w.x += bv.x * av.x + bv.y * av.y;
                            w.y += bv.x * av.y - bv.y * av.x;
                        }
                    }
                    sm.sWd[q][i] = w;
                }
            }
            __syncthreads();
            if (tid == 0) {  // phase 2: sigma_{ts+i}, i = 0..TL (sigma_{l0+1} = 1)
                double sm1 = sig_m1, s0 = sig_0;
                sm.sSig[0] = s0;
                for (int i = 0; i < TL; ++i) {
                    const int l = ts + i;
                    const double nx = (l == l0 || l >= L) ? s0 : sm.sF2[i] * sm1;
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
                sm.sA[i] = fg;
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    double2 w = sm.sWd[q][i];
                    w.x *= sg;
                    w.y *= sg;
                    if (SUM_FF) {
                        float4 wf;
                        dbl_to_ff(w.x, wf.x, wf.z);
                        dbl_to_ff(w.y, wf.y, wf.w);
                        sm.sW[q][i] = wf;
                    } else {
                        sm.sWd[q][i] = w;
                    }
                }
                sm.sT[i] = __double_as_longlong(WG_EPS_SUM / sg);
            }
            __syncthreads();
            const int nl = min(TL, L + 1 - ts);
            for (int i = 0; i < nl; ++i) {
                const double2 fg = sm.sA[i];
                const long long thr = sm.sT[i];
                bool any = false;
#pragma unroll
                for (int c = 0; c < CPT; ++c) {
                    if (!summing[c] && plain[c] && abs_ge(u[c], thr)) {
                        summing[c] = true;
                        lsum[c] = ts + i;
                    }
                    any |= summing[c];
                }
                if (!warp_sum) warp_sum = __any_sync(0xffffffffu, any);
                if (warp_sum) {
                    if (SUM_FF) {
                        ff uu[CPT];
#pragma unroll
                        for (int c = 0; c < CPT; ++c) {
                            uu[c] = split_ff(u[c]);
                            if (!summing[c]) uu[c] = ff{0.f, 0.f};
                        }
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            const float4 w = sm.sW[q][i];
#pragma unroll
                            for (int c = 0; c < CPT; ++c)
                                ff_mac2(ahi[q][c], alo[q][c], make_float2(w.x, w.y), make_float2(w.z, w.w),
                                        uu[c].hi, uu[c].lo);
                        }
                    } else {
#pragma unroll
                        for (int q = 0; q < K; ++q) {
                            const double2 w = sm.sWd[q][i];
#pragma unroll
                            for (int c = 0; c < CPT; ++c) {
                                const double um = summing[c] ? u[c] : 0.0;
                                cre[q][c] = fma(w.x, um, cre[q][c]);
                                cim[q][c] = fma(w.y, um, cim[q][c]);
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
        const size_t col = (size_t)mb * (A.ms_max + 1) + ms;
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            if (valid[c]) {
                const double nan = __longlong_as_double(0x7ff8000000000000LL);
#pragma unroll
                for (int q = 0; q < K; ++q) {
                    double re = cre[q][c], im = cim[q][c];
                    if (SUM_FF) {
                        re = (double)ahi[q][c].x + (double)alo[q][c].x;
                        im = (double)ahi[q][c].y + (double)alo[q][c].y;
                    }
                    A.c[(COMBINE ? 0 : A.k0 + q) * A.sc + col * NB + jj[c]] =
                        ang[c].bad ? make_double2(nan, nan) : make_double2(re, im);
                }
                n_elem += (unsigned long long)(L + 1 - l0);
                n_sum += (unsigned long long)(L + 1 - min(lsum[c], L + 1));
            }
        }
    }
    flush_counters(A.counters, n_elem, n_sum);
}

template <bool SUM_FF, int K, bool COMBINE>
static int launch_multi_t(const MultiArgs &a, const Tables &t, cudaStream_t s) {
    constexpr int NT = 256, CPT = 2, TL = 128, GROUP = 4;
    const int per_chunk = NT * CPT;
    const int n_chunks = (a.n_beta + per_chunk - 1) / per_chunk;
    const int ncol = (a.mb_max + 1) * (a.ms_max + 1);
    const long long items = (long long)n_chunks * ((ncol + GROUP - 1) / GROUP);
    if (items == 0) return 0;
    if (items > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    conv_multi_kernel<NT, CPT, TL, SUM_FF, K, COMBINE><<<(unsigned)items, NT, 0, s>>>(a, t, n_chunks, GROUP);
    return (int)cudaGetLastError();
}

template <bool SUM_FF>
static int launch_multi(const MultiArgs &a, int k, bool combine, const Tables &t, cudaStream_t s) {
    if (combine) return launch_multi_t<SUM_FF, 1, true>(a, t, s);
    switch (k) {
        case 1: return launch_multi_t<SUM_FF, 1, false>(a, t, s);
        case 2: return launch_multi_t<SUM_FF, 2, false>(a, t, s);
        case 3: return launch_multi_t<SUM_FF, 3, false>(a, t, s);
        default: return launch_multi_t<SUM_FF, 4, false>(a, t, s);
    }
}

void set_last_error(const std::string &msg, int code);
int tables_for(int l_max, Tables *t);  // wg_capi.cu

}  // namespace wg

namespace {
int fail(int code, const std::string &msg) {
    wg::set_last_error(msg, code);
    return code;
}
bool al16(const void *p) { return ((uintptr_t)p & 15) == 0; }
}  // namespace

extern "C" int wigner_conv_sum_multi(int l_max, int mb_max, int ms_max, int n_beta, int n_col, const double *beta,
                                     const wg_c64 *a, const wg_c64 *b, int b_shared, int sum_cols, wg_form form,
                                     wg_c64 *c_out, wg_counter *counters, void *stream) {
    if (l_max < 0 || l_max > WG_LMAX) return fail(WG_ERR_ARG, "l_max must be in [0, WG_LMAX]");
    if (mb_max < 0 || mb_max > l_max) return fail(WG_ERR_ARG, "mb_max must be in [0, l_max]");
    if (ms_max < 0 || ms_max > l_max) return fail(WG_ERR_ARG, "ms_max must be in [0, l_max]");
    if (n_beta < 0 || n_col < 0) return fail(WG_ERR_ARG, "n_beta and n_col must be >= 0");
    if (form == WG_FP32X) return fail(WG_ERR_UNSUPPORTED, "several weight columns: FP64 / FP64S only");
    if (form != WG_FP64 && form != WG_FP64S) return fail(WG_ERR_ARG, "unknown form");
    if (n_beta == 0 || (n_col == 0 && !sum_cols)) return WG_OK;
    if (!beta || ((uintptr_t)beta & 7)) return fail(WG_ERR_ARG, "beta is NULL or not 8-byte aligned");
    if (!c_out || !al16(c_out)) return fail(WG_ERR_ARG, "c_out must be non-NULL and 16-byte aligned");
    if (n_col > 0 && (!a || !b || !al16(a) || !al16(b)))
        return fail(WG_ERR_ARG, "a and b must be non-NULL and 16-byte aligned");
    if (counters && ((uintptr_t)counters & 7)) return fail(WG_ERR_ARG, "counters misaligned");
    // many skies with one beam: the tensor-core path (same accuracy class)
    if (!sum_cols && b_shared && n_col >= WG_MULTI_TC_MIN_COLS)
        return wigner_conv_sum_multi_tc(l_max, mb_max, ms_max, n_beta, n_col, beta, a, b, c_out, counters, stream);
    wg::Tables t;
    int rc = wg::tables_for(l_max, &t);
    if (rc != WG_OK) return rc;
    wg::MultiArgs ma{};
    ma.l_max = l_max;
    ma.mb_max = mb_max;
    ma.ms_max = ms_max;
    ma.n_beta = n_beta;
    ma.beta = beta;
    ma.a = (const double2 *)a;
    ma.b = (const double2 *)b;
    ma.c = (double2 *)c_out;
    ma.sa = (size_t)(l_max + 1) * (ms_max + 1);
    ma.sb = b_shared ? 0 : (size_t)(l_max + 1) * (mb_max + 1);
    ma.sc = (size_t)(mb_max + 1) * (ms_max + 1) * n_beta;
    ma.n_col = n_col;
    cudaStream_t s = (cudaStream_t)stream;
    const bool combine = sum_cols != 0;
    const int step = combine ? (n_col > 0 ? n_col : 1) : wg::KMAX;
    for (int k0 = 0; k0 < (n_col > 0 ? n_col : 1); k0 += step) {
        const int k = combine ? 1 : (n_col - k0 < wg::KMAX ? n_col - k0 : wg::KMAX);
        ma.k0 = k0;
        ma.counters = k0 == 0 ? counters : nullptr;  // the chains, counted once
        const int e = form == WG_FP64S ? wg::launch_multi<true>(ma, k, combine, t, s)
                                       : wg::launch_multi<false>(ma, k, combine, t, s);
        if (e != 0) {
            wg::set_last_error(std::string("conv_multi launch: ") + cudaGetErrorString((cudaError_t)e), WG_ERR_CUDA);
            return WG_ERR_CUDA;
        }
    }
    return WG_OK;
}
