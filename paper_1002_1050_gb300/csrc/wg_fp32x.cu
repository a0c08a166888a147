// wg_fp32x.cu -- launchers of the FP32 form (fused sum and d-table); the per-item
// device code and the precision design are described in wg_fp32x.cuh.
#include <cuda_runtime.h>

#include "../../include/wigner.h"
#include "wg_fp32x.cuh"

namespace wg {

// shared memory in the dynamic segment (a CTA of 256 threads needs more than 48 KB)
template <int NT, int CPT, int TL>
__global__ void __launch_bounds__(NT, 768 / NT) conv_fp32x_kernel(ConvArgs A, Tables T, int n_chunks, int group) {
    extern __shared__ __align__(16) unsigned char fp32x_smem[];
    SmemFp32<NT, CPT, TL> &sm = *reinterpret_cast<SmemFp32<NT, CPT, TL> *>(fp32x_smem);
    const int item = blockIdx.x;
    const int chunk = item % n_chunks;
    const int grp = item / n_chunks;
    const int ncol = (A.mb_max + 1) * (A.ms_max + 1);
    const int k_hi = A.k_hi < 0 ? ncol : A.k_hi;
    const int k_begin = A.k_lo + grp * group;
    const int k_end = min(k_hi, k_begin + group);
    unsigned long long n_elem = 0, n_sum = 0;
    conv_fp32x_item<NT, CPT, TL>(A, T, chunk, k_begin, k_end, sm, n_elem, n_sum);
    flush_counters(A.counters, n_elem, n_sum);
}

// Per-column power-of-two scales of the FP32 form's weights: ea[ms] = e with max over l
// of |a[l][ms]| (re and im) in [2^(e-1), 2^e), eb[mb] likewise for b (0 for a zero
// column), so that the scaled weights stay in float's range whatever the columns'
// magnitudes.  Threads 0..ms_max take a's columns, the next mb_max + 1 threads b's.
__global__ void fp32x_scales_kernel(const double *a, const double *b, int L, int MB, int MS, int *ea, int *eb) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool is_a = t <= MS;
    const int c = is_a ? t : t - (MS + 1);
    if (!is_a && c > MB) return;
    const int stride = is_a ? MS + 1 : MB + 1;
    const double2 *col = reinterpret_cast<const double2 *>(is_a ? a : b) + c;
    int m = 0;
    for (int l = 0; l <= L; ++l) {
        const double2 v = col[(size_t)l * stride];
        m = max(m, max(biased_exp(v.x), biased_exp(v.y)));
    }
    (is_a ? ea : eb)[c] = m == 0 ? 0 : m - 1022;
}

int host_pool(cudaMemPool_t *pool);  // wg_host.cu

template <int NT, int CPT, int TL>
static int launch_conv_fp32x_t(const ConvArgs &a_in, const Tables &t, void *stream, int group) {
    const int per_chunk = NT * CPT;
    const int n_chunks = (a_in.n_beta + per_chunk - 1) / per_chunk;
    const int ncol = (a_in.mb_max + 1) * (a_in.ms_max + 1);
    const int nk = (a_in.k_hi < 0 ? ncol : a_in.k_hi) - a_in.k_lo;
    const long long items = (long long)n_chunks * ((nk + group - 1) / group);
    if (items == 0) return 0;
    if (items > 0x7fffffffLL) return (int)cudaErrorInvalidValue;
    cudaStream_t s = (cudaStream_t)stream;
    // the weight scales, in stream-ordered scratch from the library's pool
    cudaMemPool_t pool;
    if (host_pool(&pool) != WG_OK) return (int)cudaErrorMemoryAllocation;
    ConvArgs a = a_in;
    int *sc = nullptr;
    const int n_sc = a.ms_max + 1 + a.mb_max + 1;
    cudaError_t e = alloc_injected() ? cudaErrorMemoryAllocation
                                     : cudaMallocFromPoolAsync((void **)&sc, (size_t)n_sc * sizeof(int), pool, s);
    if (e != cudaSuccess) return (int)e;
    a.ea = sc;
    a.eb = sc + a.ms_max + 1;
    fp32x_scales_kernel<<<(unsigned)((n_sc + 127) / 128), 128, 0, s>>>(a.a, a.b, a.l_max, a.mb_max, a.ms_max,
                                                                       const_cast<int *>(a.ea), const_cast<int *>(a.eb));
    e = cudaGetLastError();
    constexpr size_t smem = sizeof(SmemFp32<NT, CPT, TL>);
    if (e == cudaSuccess && smem > 48 * 1024)  // an attribute of the current device's function
        e = cudaFuncSetAttribute(conv_fp32x_kernel<NT, CPT, TL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) {
        conv_fp32x_kernel<NT, CPT, TL><<<(unsigned)items, NT, smem, s>>>(a, t, n_chunks, group);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(sc, s);
    return (int)(e != cudaSuccess ? e : ef);
}

int launch_conv_fp32x(const ConvArgs &a, const Tables &t, void *stream) {
    return launch_conv_fp32x_t<256, 4, 240>(a, t, stream, 16);
}

// ---------------------------------------------------------------------------
// d-table, FP32 form (values stored as double)
// ---------------------------------------------------------------------------
// the angles' quantities of the FP32 form, once per launch (one thread per angle)
__global__ void angle32_setup_kernel(const double *beta, int n_beta, Angle32 *ang, int *status) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_beta) return;
    const Angle32 t = make_angle32(beta[j]);
    if (t.bad) raise_status(status, WG_DEVERR_BETA);
    ang[j] = t;
}

// mant 2^(64 n) (times -1 if neg) as a double by integer operations on the float's bits:
// exact while the result is a normal double; below 2^-1022, and for a zero or subnormal
// float, 0
__device__ __forceinline__ double f32_scaled_to_double(float mant, int n, bool neg) {
    const unsigned u = __float_as_uint(mant) ^ (neg ? 0x80000000u : 0u);
    const int e = (int)((u >> 23) & 0xffu);
    const int ed = e - 127 + 1023 + 64 * n;  // the double's biased exponent
    if (e == 0 || ed <= 0) return 0.0;
    return __longlong_as_double((long long)(((unsigned long long)(u & 0x80000000u) << 32) |
                                            ((unsigned long long)ed << 52) |
                                            ((unsigned long long)(u & 0x7fffffu) << 29)));
}

// One CTA per (column, NT angles), one chain per thread; the column's difference-form
// coefficients of each l-tile built once per CTA in shared memory.
template <int NT, int TL>
__global__ void __launch_bounds__(NT) dtable_fp32x_kernel(DTableArgs A, Tables T, const Angle32 *ang) {
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
    const Angle32 t = ang[valid ? j : 0];
    const bool high = t.high;
    const float x2 = t.x2;
    const Seed32 sd = seed32(mb, ms, t, T);
    float cur = (high && (l0 & 1)) ? -sd.mant : sd.mant;
    float aux = cur;
    int n = sd.n;
    __shared__ float4 sT[TL];
    for (int ts = l0; ts <= L; ts += TL) {
        __syncthreads();
        for (int i = threadIdx.x; i < TL; i += NT) {
            const int l = ts + i;
            float4 raw;
            sT[i] = (l <= L) ? diff_coefficients(l, L, mb, ms, T, raw) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
        const int nl = min(TL, L + 1 - ts);
        for (int i = 0; i < nl; ++i) {
            const int l = ts + i;
            if (valid)
                out[(size_t)l * NB + j] = t.bad ? __longlong_as_double(0x7ff8000000000000LL)
                                                : f32_scaled_to_double(cur, n, high && (l & 1));
            const float4 tc = sT[i];
            const float coef = fmaf(tc.x, x2, high ? tc.w : tc.z);
            aux = fmaf(tc.y, aux, coef * cur);
            cur = cur + aux;
            if (n != 0) fixup32(cur, aux, n);
        }
    }
    if (A.counters && threadIdx.x == 0) {
        const int nvalid = min(NT, A.n_beta - (int)blockIdx.y * NT);
        atomicAdd(&A.counters[0], (unsigned long long)nvalid * (unsigned long long)(L + 1 - l0));
    }
}

int launch_dtable_fp32x(const DTableArgs &a, const Tables &t, void *stream) {
    constexpr int NT = 64, TL = 128;
    if (a.n_beta == 0) return 0;
    cudaStream_t s = (cudaStream_t)stream;
    cudaMemPool_t pool;
    if (host_pool(&pool) != WG_OK) return (int)cudaErrorMemoryAllocation;
    Angle32 *ang = nullptr;
    cudaError_t e = alloc_injected() ? cudaErrorMemoryAllocation
                                     : cudaMallocFromPoolAsync((void **)&ang, (size_t)a.n_beta * sizeof(Angle32), pool, s);
    if (e != cudaSuccess) return (int)e;
    angle32_setup_kernel<<<(a.n_beta + 127) / 128, 128, 0, s>>>(a.beta, a.n_beta, ang, t.status);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        const int ncol = (a.mb_max + 1) * (a.ms_max + 1);
        dim3 grid(ncol, (a.n_beta + NT - 1) / NT);
        dtable_fp32x_kernel<NT, TL><<<grid, NT, 0, s>>>(a, t, ang);
        e = cudaGetLastError();
    }
    const cudaError_t ef = cudaFreeAsync(ang, s);
    return (int)(e != cudaSuccess ? e : ef);
}

}  // namespace wg
