// wg_bwd.cu -- adjoints of the fused l-sum and of the d-table (FP64).
//
// Gradients of a real loss L in PyTorch's convention for complex tensors
// (grad z = dL/dRe z + i dL/dIm z), with C_{mb,ms}(beta) = sum_l conj(b_{l,mb}) a_{l,ms} d^l:
//   grad_a[l][ms] = sum_mb b[l][mb] S[l][mb][ms],   S[l][mb][ms] = sum_j G[mb][ms][j] d^l_{mb,ms}(beta_j)
//   grad_b[l][mb] = sum_ms a[l][ms] conj(S[l][mb][ms])
//   grad_beta[j]  = Re sum_{mb,ms} conj(G) sum_l w_l d/dbeta d^l_{mb,ms}(beta_j)
// The beta-derivative uses Eq. mrec's relation between neighbouring m' (Sec. 2):
//   d/dbeta d^l_{m,m'} = ((m' cos b - m)/sin b) d^l_{m,m'} - sqrt((l-m')(l+m'+1)) d^l_{m,m'+1}
// so  sum_l w_l d/dbeta d^l_{mb,ms} = ((ms cos b - mb)/sin b) C_{mb,ms} - E_{mb,ms},
//     E_{mb,ms}(beta) = sum_l w_{l,mb,ms} sqrt((l-ms)(l+ms+1)) d^l_{mb,ms+1}(beta):
// a weighted l-sum over the neighbour chain (mb, ms+1).  The chains are recomputed;
// no d-table is stored.
//
// Kernel layout: as the forward kernel (column group x angle chunk per CTA, CPT chains
// per thread, the normalised two-FMA recursion).  For each column (mb, ms') the CTA
// runs the chains and, in float-float on the FP32 pipe,
//   * accumulates, per chain, E for column (mb, ms'-1) from the weights of that column;
//   * forms S[l] = sum over the CTA's angles of G d^l: each lane sums its CPT chains,
//     a warp reduce-scatter over blocks of 16 l (shuffles) leaves one warp sum per l,
//     and the warps' sums are added in shared memory; with one angle chunk the value
//     is stored, with several it is added atomically into the zeroed workspace.
// Epilogue kernels then form grad_beta (a sum over columns per angle, fixed order)
// and grad_a, grad_b (sums over m_b or m_sky per l).
#include <cuda_runtime.h>

#include "wg_common.cuh"
#include "wg_conv_fp64.cuh"  // dbl_to_ff

namespace wg {

constexpr int LB = 8;  // l-block of the warp reduce-scatter

// (vh, vl)[i], i < LB: the (re, im) float-float values of LB orders in every lane ->
// lane t (t < LB) holds the warp sum of order t in (vh, vl)[0]
__device__ __forceinline__ void warp_reduce_scatter_ff2(float2 (&vh)[LB], float2 (&vl)[LB], int lane) {
#pragma unroll
    for (int off = LB / 2; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int i = 0; i < off; ++i) {
            const float2 sh = up ? vh[i] : vh[i + off], sl = up ? vl[i] : vl[i + off];
            const float2 kh = up ? vh[i + off] : vh[i], kl = up ? vl[i + off] : vl[i];
            const float2 gh = make_float2(__shfl_xor_sync(0xffffffffu, sh.x, off), __shfl_xor_sync(0xffffffffu, sh.y, off));
            const float2 gl = make_float2(__shfl_xor_sync(0xffffffffu, sl.x, off), __shfl_xor_sync(0xffffffffu, sl.y, off));
            vh[i] = kh;
            vl[i] = kl;
            ff_add2(vh[i], vl[i], gh, gl);
        }
    }
#pragma unroll
    for (int off = LB; off < 32; off <<= 1) {
        const float2 gh = make_float2(__shfl_xor_sync(0xffffffffu, vh[0].x, off), __shfl_xor_sync(0xffffffffu, vh[0].y, off));
        const float2 gl = make_float2(__shfl_xor_sync(0xffffffffu, vl[0].x, off), __shfl_xor_sync(0xffffffffu, vl[0].y, off));
        ff_add2(vh[0], vl[0], gh, gl);
    }
}

// Adjoint kernel with the forward kernels' normalised two-FMA recursion
// (u^l = d^l / sigma_l, sigma_{l+1} = F2_l sigma_{l-1}, as in wg_conv_fp64.cuh): the FP64
// pipe runs only the recursion; S = sum_beta G d^l (lane partials, the warp
// reduce-scatter and the warp sums) and the beta term's neighbour sum E accumulate in
// float-float on the FP32 pipe (~48-bit), and S is scaled back by sigma_l in double.
template <int TL>
struct SmemBwd {
    double2 sA[TL];       // (F0', G')  (phase 1: (F0, G))
    double2 sWd[TL];      // E weights (phase 1: w sqrt(...)), then times sigma_l
    float4 sWE[TL];       // E weights as float-float: (re hi, im hi, re lo, im lo)
    long long sThr[TL];   // bit pattern of 1e-30 / sigma_l
    double sF2[TL];
    double sSig[TL + 1];
    float4 sRed[TL / LB][8][LB];  // warp sums of S per l (re hi, lo, im hi, lo), up to 8 warps
};

template <int NT, int CPT, int TL>
__global__ void __launch_bounds__(NT) conv_bwd_kernel(ConvBwdArgs A, Tables T, int n_chunks, int group, int ms_hi,
                                                       int want_s, int atomic_s, double *partial) {
    static_assert(TL % LB == 0, "tile must hold whole l-blocks");
    constexpr int NW = NT / 32;
    static_assert(NW <= 8, "at most 8 warps");
    __shared__ SmemBwd<TL> sm;
    const int item = blockIdx.x;
    const int chunk = item % n_chunks;
    const int grp = item / n_chunks;
    const int MB1 = A.mb_max + 1;
    const int MS1 = A.ms_max + 1;
    const int ncol = MB1 * (ms_hi + 1);
    const int k_begin = grp * group;
    const int k_end = min(ncol, k_begin + group);
    const int L = A.l_max;
    const int NB = A.n_beta;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool want_e = partial != nullptr;

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

    for (int k = k_begin; k < k_end; ++k) {
        const int ms = k / MB1, mb = k - ms * MB1;  // this chain column is (mb, ms)
        const int l0 = mb > ms ? mb : ms;
        const bool do_s = want_s && ms <= A.ms_max;
        const bool do_e = want_e && ms >= 1;

        double u[CPT], up[CPT];
        float2 gh[CPT], gl[CPT], eh[CPT], el[CPT];  // G and E as float-float (re, im) pairs
        int nsc[CPT];
        bool plain[CPT];
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const Scaled s = seed_value(mb, ms, ang[c], T);
            u[c] = s.mant;
            nsc[c] = s.n;
            plain[c] = s.plain;
            up[c] = 0.0;
            eh[c] = el[c] = gh[c] = gl[c] = make_float2(0.f, 0.f);
            if (do_s && valid[c]) {
                const double2 g = reinterpret_cast<const double2 *>(A.grad_c)[((size_t)mb * MS1 + ms) * NB + jj[c]];
                dbl_to_ff(g.x, gh[c].x, gl[c].x);
                dbl_to_ff(g.y, gh[c].y, gl[c].y);
            }
        }
        double sig_m1 = 0.0, sig_0 = 1.0;

        for (int ts = l0; ts <= L; ts += TL) {
            __syncthreads();
            for (int i = tid; i < TL; i += NT) {  // phase 1
                const int l = ts + i;
                double f0 = 0.0, g = 0.0, f2 = 0.0;
                double2 w = make_double2(0.0, 0.0);
                if (l <= L) {
                    if (l < L) lrec_coefficients(l, mb, ms, T, f0, g, f2);
                    if (do_e) {
                        const double2 av = reinterpret_cast<const double2 *>(A.a)[(size_t)l * MS1 + (ms - 1)];
                        const double2 bv = reinterpret_cast<const double2 *>(A.b)[(size_t)l * MB1 + mb];
                        const double sq = sqrt((double)(l - ms + 1) * (double)(l + ms));
                        w = make_double2((bv.x * av.x + bv.y * av.y) * sq, (bv.x * av.y - bv.y * av.x) * sq);
                    }
                }
                sm.sA[i] = make_double2(f0, g);
                sm.sF2[i] = f2;
                sm.sWd[i] = w;
            }
            __syncthreads();
            if (tid == 0) {  // phase 2: sigma
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
            for (int i = tid; i < TL; i += NT) {  // phase 3
                const int l = ts + i;
                const double sg = sm.sSig[i];
                double2 fg = sm.sA[i];
                if (l < L) {
                    const double rho = sg / sm.sSig[i + 1];
                    fg.x *= rho;
                    fg.y *= rho;
                }
                sm.sA[i] = fg;
                const double2 w = sm.sWd[i];
                float4 wf;
                dbl_to_ff(w.x * sg, wf.x, wf.z);
                dbl_to_ff(w.y * sg, wf.y, wf.w);
                sm.sWE[i] = wf;
                sm.sThr[i] = __double_as_longlong(WG_EPS_SUM / sg);
            }
            __syncthreads();
#pragma unroll 1
            for (int blk = 0; blk < TL / LB; ++blk) {
                const int lb = ts + blk * LB;
                if (lb > L) break;  // uniform over the CTA
                float2 sh[LB], sl[LB];  // S of the block's orders: (re, im) float-float
#pragma unroll
                for (int i = 0; i < LB; ++i) {
                    const int l = lb + i;
                    sh[i] = sl[i] = make_float2(0.f, 0.f);
                    if (l <= L) {  // uniform
                        const int ti = blk * LB + i;
                        const float4 we = sm.sWE[ti];
                        const long long thr = sm.sThr[ti];
#pragma unroll
                        for (int c = 0; c < CPT; ++c) {
                            // terms with |d| < 1e-30 are left out, as in the forward sum;
                            // this also keeps split_ff inside its range (|u| >= 2^-100)
                            ff uu = split_ff(u[c]);
                            if (!plain[c] || !abs_ge(u[c], thr)) uu = ff{0.f, 0.f};
                            if (do_s) ff_mac2(sh[i], sl[i], gh[c], gl[c], uu.hi, uu.lo);
                            if (do_e)
                                ff_mac2(eh[c], el[c], make_float2(we.x, we.y), make_float2(we.z, we.w), uu.hi, uu.lo);
                        }
                        if (l < L) {
                            const double2 fg = sm.sA[ti];
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
                if (do_s) {
                    warp_reduce_scatter_ff2(sh, sl, lane);
                    if (lane < LB) sm.sRed[blk][warp][lane] = make_float4(sh[0].x, sl[0].x, sh[0].y, sl[0].y);
                }
            }
            __syncthreads();
            if (do_s) {
                for (int i = tid; i < TL; i += NT) {
                    const int l = ts + i;
                    if (l > L) continue;
                    ff re{0.f, 0.f}, im{0.f, 0.f};
#pragma unroll
                    for (int w = 0; w < NW; ++w) {
                        const float4 v = sm.sRed[i / LB][w][i % LB];
                        re = ff_add(re, ff{v.x, v.y});
                        im = ff_add(im, ff{v.z, v.w});
                    }
                    const double sg = sm.sSig[i];
                    const double vr = ((double)re.hi + (double)re.lo) * sg;
                    const double vi = ((double)im.hi + (double)im.lo) * sg;
                    double *dst = A.S + 2 * (((size_t)l * MB1 + mb) * MS1 + ms);
                    if (atomic_s) {
                        atomicAdd(dst, vr);
                        atomicAdd(dst + 1, vi);
                    } else {
                        dst[0] = vr;
                        dst[1] = vi;
                    }
                }
            }
        }
        if (do_e) {
#pragma unroll
            for (int c = 0; c < CPT; ++c) {
                if (!valid[c]) continue;
                const size_t o = ((size_t)mb * MS1 + (ms - 1)) * NB + jj[c];
                const double2 g = reinterpret_cast<const double2 *>(A.grad_c)[o];
                const double2 cf = reinterpret_cast<const double2 *>(A.c_fwd)[o];
                const double coef = ((double)(ms - 1) * ang[c].cb - (double)mb) / ang[c].sb;
                const double vr = coef * cf.x - ((double)eh[c].x + (double)el[c].x);
                const double vi = coef * cf.y - ((double)eh[c].y + (double)el[c].y);
                partial[o] = g.x * vr + g.y * vi;
            }
        }
    }
}

// grad_beta[j] = sum over columns of partial[col][j] (fixed order); NaN outside (0, pi)
__global__ void reduce_columns_kernel(const double *partial, int ncol, int n_beta, const double *beta,
                                      double *grad_beta, int *status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_beta) return;
    const double b = beta[j];
    if (!(b > 0.0 && b < WG_PI_HI)) {
        grad_beta[j] = __longlong_as_double(0x7ff8000000000000LL);
        if (status) atomicOr(status, WG_DEVERR_BETA);
        return;
    }
    double acc = 0.0;
    for (int c = 0; c < ncol; ++c) acc += partial[(size_t)c * n_beta + j];
    grad_beta[j] = acc;
}

// grad_a[l][ms] = sum_mb b[l][mb] S[l][mb][ms]
__global__ void grad_a_kernel(const double *S, const double *b, int l_max, int mb_max, int ms_max, double *grad_a) {
    const size_t idx = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int MS1 = ms_max + 1, MB1 = mb_max + 1;
    if (idx >= (size_t)(l_max + 1) * MS1) return;
    const int l = (int)(idx / MS1), ms = (int)(idx % MS1);
    double re = 0.0, im = 0.0;
    for (int mb = 0; mb < MB1; ++mb) {
        const double2 bv = reinterpret_cast<const double2 *>(b)[(size_t)l * MB1 + mb];
        const double2 s = reinterpret_cast<const double2 *>(S)[((size_t)l * MB1 + mb) * MS1 + ms];
        re += bv.x * s.x - bv.y * s.y;
        im += bv.x * s.y + bv.y * s.x;
    }
    reinterpret_cast<double2 *>(grad_a)[idx] = make_double2(re, im);
}

// grad_b[l][mb] = sum_ms a[l][ms] conj(S[l][mb][ms]); one CTA per (l, mb)
template <int NT>
__global__ void __launch_bounds__(NT) grad_b_kernel(const double *S, const double *a, int l_max, int mb_max,
                                                    int ms_max, double *grad_b) {
    const int MS1 = ms_max + 1, MB1 = mb_max + 1;
    const int l = blockIdx.x / MB1, mb = blockIdx.x % MB1;
    double re = 0.0, im = 0.0;
    for (int ms = threadIdx.x; ms < MS1; ms += NT) {
        const double2 av = reinterpret_cast<const double2 *>(a)[(size_t)l * MS1 + ms];
        const double2 s = reinterpret_cast<const double2 *>(S)[((size_t)l * MB1 + mb) * MS1 + ms];
        re += av.x * s.x + av.y * s.y;
        im += av.y * s.x - av.x * s.y;
    }
    __shared__ double rr[NT / 32], ri[NT / 32];
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, off);
        im += __shfl_down_sync(0xffffffffu, im, off);
    }
    if ((threadIdx.x & 31) == 0) {
        rr[threadIdx.x >> 5] = re;
        ri[threadIdx.x >> 5] = im;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double tr = 0.0, ti = 0.0;
        for (int w = 0; w < NT / 32; ++w) {
            tr += rr[w];
            ti += ri[w];
        }
        reinterpret_cast<double2 *>(grad_b)[(size_t)l * MB1 + mb] = make_double2(tr, ti);
    }
}

int launch_conv_bwd(const ConvBwdArgs &a, const Tables &t, void *stream_) {
    constexpr int NT = 256, CPT = 2, TL = 128;
    cudaStream_t stream = (cudaStream_t)stream_;
    const int MB1 = a.mb_max + 1, MS1 = a.ms_max + 1;
    const bool want_s = a.grad_a || a.grad_b;
    const bool want_e = a.grad_beta != nullptr;
    const size_t s_bytes = (size_t)(a.l_max + 1) * MB1 * MS1 * 16;
    cudaError_t e;
    if (want_s) {
        e = cudaMemsetAsync(a.S, 0, s_bytes, stream);
        if (e != cudaSuccess) return (int)e;
    }
    if (a.n_beta > 0 && (want_s || want_e)) {
        const int per_chunk = NT * CPT;
        const int n_chunks = (a.n_beta + per_chunk - 1) / per_chunk;
        const int ms_hi = want_e ? a.ms_max + 1 : a.ms_max;
        const int ncol = MB1 * (ms_hi + 1);
        const int group = 4;
        const long long items = (long long)n_chunks * ((ncol + group - 1) / group);
        if (items > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
        conv_bwd_kernel<NT, CPT, TL><<<(unsigned)items, NT, 0, stream>>>(a, t, n_chunks, group, ms_hi,
                                                                           want_s ? 1 : 0, n_chunks > 1 ? 1 : 0,
                                                                           want_e ? a.E : nullptr);
        e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    if (want_e) {
        if (a.n_beta > 0) {
            reduce_columns_kernel<<<(a.n_beta + 255) / 256, 256, 0, stream>>>(a.E, MB1 * MS1, a.n_beta, a.beta,
                                                                              a.grad_beta, t.status);
            e = cudaGetLastError();
            if (e != cudaSuccess) return (int)e;
        }
    }
    if (a.grad_a) {
        const size_t n = (size_t)(a.l_max + 1) * MS1;
        grad_a_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(a.S, a.b, a.l_max, a.mb_max, a.ms_max, a.grad_a);
        e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    if (a.grad_b) {
        grad_b_kernel<128><<<(unsigned)((a.l_max + 1) * MB1), 128, 0, stream>>>(a.S, a.a, a.l_max, a.mb_max, a.ms_max,
                                                                                 a.grad_b);
        e = cudaGetLastError();
        if (e != cudaSuccess) return (int)e;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// d-table adjoint: grad_beta[j] = sum_{mb,ms,l} Gd[mb][ms][l][j] d/dbeta d^l_{mb,ms}(beta_j).
// For chain column (mb, ms'):  coef' sum_l Gd[mb][ms'][l][j] d^l  -  sum_l s_l Gd[mb][ms'-1][l][j] d^l,
// coef' = (ms' cos b - mb)/sin b,  s_l = sqrt((l-ms'+1)(l+ms')); per-(column, angle) partials
// are then summed over columns in a fixed order.
// ---------------------------------------------------------------------------
template <int NT, int TL>
__global__ void __launch_bounds__(NT) dtable_bwd_kernel(DTableBwdArgs A, Tables T, int ms_hi) {
    const int MB1 = A.mb_max + 1, MS1 = A.ms_max + 1;
    const int col = blockIdx.x;  // over MB1 * (ms_hi + 1)
    const int ms = col / MB1, mb = col - ms * MB1;
    const int j = blockIdx.y * NT + threadIdx.x;
    const bool valid = j < A.n_beta;
    const int L = A.l_max;
    const int l0 = mb > ms ? mb : ms;
    const size_t NB = (size_t)A.n_beta;
    const Angle t = make_angle(valid ? A.beta[j] : 1.0);
    const Scaled s = seed_value(mb, ms, t, T);
    double cur = s.mant, prev = 0.0;
    int n = s.n;
    bool plain = s.plain;
    const double *g1 = (ms <= A.ms_max) ? A.grad_d + ((size_t)mb * MS1 + ms) * (size_t)(L + 1) * NB : nullptr;
    const double *g0 = (ms >= 1) ? A.grad_d + ((size_t)mb * MS1 + (ms - 1)) * (size_t)(L + 1) * NB : nullptr;
    double acc1 = 0.0, acc0 = 0.0;
    __shared__ double sF0[TL], sG[TL], sF2[TL], sS[TL];
    for (int ts = l0; ts <= L; ts += TL) {
        __syncthreads();
        for (int i = threadIdx.x; i < TL; i += NT) {
            const int l = ts + i;
            double f0 = 0.0, g = 0.0, f2 = 0.0, sq = 0.0;
            if (l < L) lrec_coefficients(l, mb, ms, T, f0, g, f2);
            if (l <= L && ms >= 1) sq = sqrt((double)(l - ms + 1) * (double)(l + ms));
            sF0[i] = f0;
            sG[i] = g;
            sF2[i] = f2;
            sS[i] = sq;
        }
        __syncthreads();
        const int nl = min(TL, L + 1 - ts);
        for (int i = 0; i < nl; ++i) {
            const int l = ts + i;
            const double dv = plain ? cur : 0.0;
            if (valid) {
                if (g1) acc1 = fma(g1[(size_t)l * NB + j], dv, acc1);
                if (g0) acc0 = fma(g0[(size_t)l * NB + j], sS[i] * dv, acc0);
            }
            if (l < L) {
                const double y = fma(sF0[i], t.cb, -sG[i]);
                const double nx = fma(y, cur, -(sF2[i] * prev));
                prev = cur;
                cur = nx;
                if (!plain) scaled_fixup(cur, prev, n, plain);
            }
        }
    }
    if (valid) {
        const double coef = ((double)ms * t.cb - (double)mb) / t.sb;
        A.partial[(size_t)col * NB + j] = coef * acc1 - acc0;
    }
}

int launch_dtable_bwd(const DTableBwdArgs &a, const Tables &t, void *stream_) {
    constexpr int NT = 64, TL = 128;
    cudaStream_t stream = (cudaStream_t)stream_;
    if (a.n_beta == 0) return 0;
    const int ms_hi = a.ms_max + 1;  // the neighbour column ms_max + 1 (empty when ms_max = l_max)
    const int ncol = (a.mb_max + 1) * (ms_hi + 1);
    dim3 grid(ncol, (a.n_beta + NT - 1) / NT);
    dtable_bwd_kernel<NT, TL><<<grid, NT, 0, stream>>>(a, t, ms_hi);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return (int)e;
    reduce_columns_kernel<<<(a.n_beta + 255) / 256, 256, 0, stream>>>(a.partial, ncol, a.n_beta, a.beta,
                                                                      a.grad_beta, t.status);
    return (int)cudaGetLastError();
}

}  // namespace wg
