// wg_dtable.cu -- the full d-table d^l_{mb,ms}(beta_j) (Sec. 3.2 l-recursion).
//
// One CTA = one chain column (mb, ms) x a chunk of NT angles; one thread = one
// chain (one angle).  The coefficient tables of Sec. 4.2.2 (F0, F0*F1, F2) for an
// l-tile are built once per CTA in shared memory and broadcast to every thread.
// Each step writes d^l for NT consecutive angles, so stores are coalesced along
// beta in the [mb][ms][l][beta] layout.
#include <cuda_runtime.h>

#include "wg_common.cuh"

namespace wg {

// YLM: each d^l is stored times sqrt((2l+1)/(4 pi)): with ms_max = 0 the table is then the
// theta part of the spherical harmonics, Y_l^m(theta, phi) = sqrt((2l+1)/(4 pi)) d^l_{m0}(theta)
// e^{i m phi} (the Condon-Shortley phase comes with d).
template <int NT, int TL, bool YLM = false>
__global__ void __launch_bounds__(NT) dtable_fp64_kernel(DTableArgs A, Tables T) {
    const int col = blockIdx.x;
    const int mb = col / (A.ms_max + 1), ms = col % (A.ms_max + 1);
    const int j = blockIdx.y * NT + threadIdx.x;
    const bool valid = j < A.n_beta;
    const int L = A.l_max;
    const int l0 = mb > ms ? mb : ms;
    const size_t NB = (size_t)A.n_beta;
    double *out = A.d_out + (size_t)col * (size_t)(L + 1) * NB;

    if (valid)
        for (int l = 0; l < l0; ++l) out[(size_t)l * NB + j] = 0.0;

    const Angle t = make_angle(valid ? A.beta[j] : 1.0);
    if (valid && t.bad) raise_status(T.status, WG_DEVERR_BETA);
    const Scaled s = seed_value(mb, ms, t, T);
    double cur = t.bad ? __longlong_as_double(0x7ff8000000000000LL) : s.mant;
    double prev = 0.0;
    int n = t.bad ? 0 : s.n;
    bool plain = t.bad ? true : s.plain;

    __shared__ double sF0[TL], sG[TL], sF2[TL], sN[YLM ? TL : 1];
    for (int ts = l0; ts <= L; ts += TL) {
        __syncthreads();
        for (int i = threadIdx.x; i < TL; i += NT) {
            const int l = ts + i;
            double f0 = 0.0, g = 0.0, f2 = 0.0;
            if (l < L) lrec_coefficients(l, mb, ms, T, f0, g, f2);
            sF0[i] = f0;
            sG[i] = g;
            sF2[i] = f2;
            if (YLM) sN[i] = sqrt((double)(2 * l + 1) * WG_INV_4PI);
        }
        __syncthreads();
        const int nl = min(TL, L + 1 - ts);
        for (int i = 0; i < nl; ++i) {
            const int l = ts + i;
            if (valid) {
                const double v = plain ? cur : scaled_store(cur, n);
                out[(size_t)l * NB + j] = YLM ? v * sN[i] : v;
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
    if (A.counters && threadIdx.x == 0) {
        const int nvalid = min(NT, A.n_beta - (int)blockIdx.y * NT);
        atomicAdd(&A.counters[0], (unsigned long long)nvalid * (unsigned long long)(L + 1 - l0));
    }
}

int launch_dtable_fp64(const DTableArgs &a, const Tables &t, void *stream) {
    constexpr int NT = 64, TL = 128;
    if (a.n_beta == 0) return 0;
    const int ncol = (a.mb_max + 1) * (a.ms_max + 1);
    dim3 grid(ncol, (a.n_beta + NT - 1) / NT);
    dtable_fp64_kernel<NT, TL><<<grid, NT, 0, (cudaStream_t)stream>>>(a, t);
    return (int)cudaGetLastError();
}

// out[m][l][j] = sqrt((2l+1)/(4 pi)) d^l_{m0}(theta_j) (a.ms_max must be 0)
int launch_ylm(const DTableArgs &a, const Tables &t, void *stream) {
    constexpr int NT = 64, TL = 128;
    if (a.n_beta == 0) return 0;
    dim3 grid(a.mb_max + 1, (a.n_beta + NT - 1) / NT);
    dtable_fp64_kernel<NT, TL, true><<<grid, NT, 0, (cudaStream_t)stream>>>(a, t);
    return (int)cudaGetLastError();
}

}  // namespace wg
