// wg_conv_fp64.cu -- launchers of the fused FP64 sum (the per-item device code,
// and its description, are in wg_conv_fp64.cuh).
#include <cuda_runtime.h>

#include "wg_conv_fp64.cuh"

namespace wg {

template <int NT, int CPT, int TL, bool SUM_FF, bool FULL, bool LMIN>
__global__ void __launch_bounds__(NT) conv_fp64_kernel(ConvArgs A, Tables T, int n_chunks, int group,
                                                       const __grid_constant__ WeightMaps wm) {
    __shared__ SmemFp64<TL> sm;
    __shared__ SmemTma<TL> st;
    const int item = blockIdx.x;
    const int chunk = item % n_chunks;
    const int grp = item / n_chunks;
    const int ncol = (A.mb_max + 1) * (A.ms_max + 1);
    const int k_hi = A.k_hi < 0 ? ncol : A.k_hi;
    const int k_begin = A.k_lo + grp * group;
    const int k_end = min(k_hi, k_begin + group);
    if (threadIdx.x == 0) {
        mbar_init(&st.mbar[0], 1);
        mbar_init(&st.mbar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    unsigned ph[2] = {0u, 0u};
    unsigned long long n_elem = 0, n_sum = 0;
    conv_fp64_item<NT, CPT, TL, SUM_FF, true, FULL, LMIN>(A, T, chunk, k_begin, k_end, sm, n_elem, n_sum, &wm, &st,
                                                         ph);
    flush_counters(A.counters, n_elem, n_sum);
}

template <int NT, int CPT, int TL, bool SUM_FF, bool FULL = false, bool LMIN = false>
static int launch_conv_fp64_t(const ConvArgs &a, const Tables &t, void *stream, int group) {
    const int per_chunk = NT * CPT;
    const int n_chunks = (a.n_beta + per_chunk - 1) / per_chunk;
    const int ncol = (a.mb_max + 1) * (a.ms_max + 1);
    const int nk = (a.k_hi < 0 ? ncol : a.k_hi) - a.k_lo;
    const int n_groups = (nk + group - 1) / group;
    const long long items = (long long)n_chunks * n_groups;
    if (items == 0) return 0;
    if (items > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    WeightMaps wm;
    const int e = encode_weight_maps(a.a, a.b, a.l_max, a.mb_max, a.ms_max, TL, &wm);
    if (e != 0) return e;
    conv_fp64_kernel<NT, CPT, TL, SUM_FF, FULL, LMIN>
        <<<(unsigned)items, NT, 0, (cudaStream_t)stream>>>(a, t, n_chunks, group, wm);
    return (int)cudaGetLastError();
}

int launch_conv_fp64s(const ConvArgs &a, const Tables &t, void *stream) {
    return launch_conv_fp64_t<256, 2, 128, true>(a, t, stream, 4);
}

// all-double form: the normalised two-FMA recursion with the sum in FP64 FMAs
int launch_conv_fp64(const ConvArgs &a, const Tables &t, void *stream) {
    return launch_conv_fp64_t<256, 2, 128, false>(a, t, stream, 4);
}

// every sky order (-ms_max..ms_max) for a mirror-symmetric angle grid; a.c_out is
// [mb][ms + ms_max][j]
int launch_conv_fp64_full(const ConvArgs &a, const Tables &t, void *stream, bool sum_ff) {
    return sum_ff ? launch_conv_fp64_t<256, 2, 128, true, true>(a, t, stream, 4)
                  : launch_conv_fp64_t<256, 2, 128, false, true>(a, t, stream, 4);
}

// with the l_min cut of Eq. lmin (a.offset); full: every sky order as above
int launch_conv_fp64_lmin(const ConvArgs &a, const Tables &t, void *stream, bool sum_ff, bool full) {
    if (full)
        return sum_ff ? launch_conv_fp64_t<256, 2, 128, true, true, true>(a, t, stream, 4)
                      : launch_conv_fp64_t<256, 2, 128, false, true, true>(a, t, stream, 4);
    return sum_ff ? launch_conv_fp64_t<256, 2, 128, true, false, true>(a, t, stream, 4)
                  : launch_conv_fp64_t<256, 2, 128, false, false, true>(a, t, stream, 4);
}

}  // namespace wg
