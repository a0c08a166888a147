// wg_peak.cu -- FMA-pipe throughput microbenchmark.
//
// The recursion and the l-sum are bound by the FP64 (or, in the FP32 form, the FP32)
// FMA pipe, so their roofline denominator is that pipe's throughput.  Each thread
// runs CH independent FMA chains x <- x*a + b for `iters` iterations (four per loop
// trip, so the loop's own integer instructions are a small share of the issue slots);
// a sink value per thread keeps the work observable.  The caller picks the chain count
// and the launch shape, so a sweep can find the shape that saturates the pipe.
#include <cuda_runtime.h>

#include "wg_internal.h"

namespace wg {

template <typename T, int CH>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T a, T b, double *sink) {
    T x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
    int i = 0;
    for (; i + 4 <= iters; i += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    }
    for (; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fma(x[c], a, b);
    T s = (T)0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

template <typename T>
static void launch_t(int chains, int blocks, int threads, int iters, double *sink, cudaStream_t s) {
    // a and b are kernel arguments so the compiler cannot fold the chains
    const T a = (T)0.9999, b = (T)1e-4;
    switch (chains) {
        case 1: fma_peak_kernel<T, 1><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
        case 2: fma_peak_kernel<T, 2><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
        case 4: fma_peak_kernel<T, 4><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
        case 16: fma_peak_kernel<T, 16><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
        default: fma_peak_kernel<T, 8><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
    }
}

int launch_fma_peak(int pipe, int chains, int blocks, int threads, int iters, double *sink, void *stream) {
    if (pipe == 0)
        launch_t<double>(chains, blocks, threads, iters, sink, (cudaStream_t)stream);
    else
        launch_t<float>(chains, blocks, threads, iters, sink, (cudaStream_t)stream);
    return (int)cudaGetLastError();
}

}  // namespace wg
