// wg_peak.cu -- FMA-pipe throughput microbenchmark.
//
// The recursion and the l-sum are bound by the FP64 (or, in the FP32 form, the FP32)
// FMA pipe, so their roofline denominator is that pipe's throughput.  Each thread
// runs CH independent FMA chains x <- x*a + b for `iters` iterations; a sink value per
// thread keeps the work observable.
#include <cuda_runtime.h>

#include "wg_internal.h"

namespace wg {

template <typename T, int CH>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, double *sink) {
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    const T a = (T)0.9999, b = (T)1e-4;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

int launch_fma_peak(int pipe, int blocks, int threads, int iters, double *sink, void *stream) {
    if (pipe == 0)
        fma_peak_kernel<double, 8><<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, sink);
    else
        fma_peak_kernel<float, 8><<<blocks, threads, 0, (cudaStream_t)stream>>>(iters, sink);
    return (int)cudaGetLastError();
}

}  // namespace wg
