// wg_peak.cu -- FMA-pipe throughput microbenchmark.
//
// The recursion and the l-sum are bound by the FP64 (or, in the FP32 form, the FP32)
// FMA pipe, so their roofline denominator is that pipe's throughput.  Each thread runs
// CH independent chains for `iters` steps (four per loop trip, so the loop's own
// integer instructions are a small share of the issue slots); a sink value per thread
// keeps the work observable.  The caller picks the chain count and the launch shape.
//
//  * FP64: each chain is a three-term recursion x_{n+1} = fma(y, x_n, -x_{n-1}), the
//    operand pattern of the l-recursion's step.  Measured on GB300 this form issues a
//    DFMA every pipe slot (1.253 TFLOP/s of the 1.259 that 2 FMA lanes per SM clock
//    give at 2070 MHz) when every operand is a register; the same chains with a
//    multiplier read from the constant bank (a kernel argument or a literal) stop at
//    1.055 in every launch shape tried -- an operand-source limit, not the pipe's.
//  * FP32: x = fma(x, a, b) per chain, which reaches the pipe's rate.
#include <cuda_runtime.h>

#include "wg_internal.h"

namespace wg {

template <int CH>
__global__ void __launch_bounds__(256) fma_peak_fp64_kernel(int iters, double y0, double *sink) {
    // y must be a register operand: a DFMA that reads a kernel argument or a literal
    // straight from the constant bank issues at ~84 % of the pipe's rate (measured)
    const double y = y0 + 1e-3 * (double)(threadIdx.x & 7);
    double u[CH], up[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) {
        u[c] = 0.5 + 1e-3 * (double)((threadIdx.x + c) & 255);
        up[c] = 0.5 * u[c];
    }
    int i = 0;
    for (; i + 4 <= iters; i += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < CH; ++c) {
                const double nx = fma(y, u[c], -up[c]);
                up[c] = u[c];
                u[c] = nx;
            }
    }
    for (; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CH; ++c) {
            const double nx = fma(y, u[c], -up[c]);
            up[c] = u[c];
            u[c] = nx;
        }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += u[c] + up[c];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <int CH>
__global__ void __launch_bounds__(256) fma_peak_fp32_kernel(int iters, float a, float b, double *sink) {
    float x[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    int i = 0;
    for (; i + 4 <= iters; i += 4) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < CH; ++c) x[c] = fmaf(x[c], a, b);
    }
    for (; i < iters; ++i)
#pragma unroll
        for (int c = 0; c < CH; ++c) x[c] = fmaf(x[c], a, b);
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CH; ++c) s += x[c];
    sink[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

int launch_fma_peak(int pipe, int chains, int blocks, int threads, int iters, double *sink, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    // the coefficients are kernel arguments so the compiler cannot fold the chains; the
    // FP64 chains stay bounded (|y| < 2 makes the recursion oscillate)
    const double y = 1.9;
    const float a = 0.9999f, b = 1e-4f;
    if (pipe == 0) {
        switch (chains) {
            case 1: fma_peak_fp64_kernel<1><<<blocks, threads, 0, s>>>(iters, y, sink); break;
            case 2: fma_peak_fp64_kernel<2><<<blocks, threads, 0, s>>>(iters, y, sink); break;
            case 4: fma_peak_fp64_kernel<4><<<blocks, threads, 0, s>>>(iters, y, sink); break;
            case 16: fma_peak_fp64_kernel<16><<<blocks, threads, 0, s>>>(iters, y, sink); break;
            default: fma_peak_fp64_kernel<8><<<blocks, threads, 0, s>>>(iters, y, sink); break;
        }
    } else {
        switch (chains) {
            case 1: fma_peak_fp32_kernel<1><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
            case 2: fma_peak_fp32_kernel<2><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
            case 4: fma_peak_fp32_kernel<4><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
            case 16: fma_peak_fp32_kernel<16><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
            default: fma_peak_fp32_kernel<8><<<blocks, threads, 0, s>>>(iters, a, b, sink); break;
        }
    }
    return (int)cudaGetLastError();
}

}  // namespace wg
