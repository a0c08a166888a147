// wg_internal.h -- constants and launcher declarations shared inside the library
// (not part of the public C ABI; see include/wigner.h for that).
#pragma once

#include <stdint.h>

// Scaled doubles v = d * S^n with S = 2^90 (Sec. 3.2).  ln S = 90 ln 2 split for
// exact k * LN_S_HI products: LN_S_HI keeps the leading 36 bits, LN_S_LO the rest.
#define WG_LOG2_S 90
#define WG_LN_S_HI 0x1.f310e368e0000p+5      /* 62.38324624951929... (36 bits) */
#define WG_LN_S_LO 0x1.e17863327d069p-31     /* 90 ln 2 - WG_LN_S_HI          */
#define WG_INV_LN_S 0.01602994489876626      /* 1 / (90 ln 2), only to guess k */
// switch to plain doubles once the value is >= 2^-900 (Sec. 3.2): with the mantissa
// kept in [2^-90, 2^90] that is n >= -9
#define WG_PLAIN_MIN_N (-9)
#define WG_PI_HI 3.141592653589793115997963468544185161590576171875 /* the double nearest pi */
#define WG_INV_4PI 0.07957747154594766788 /* 1 / (4 pi), the spherical-harmonic normalisation */
// threshold of Sec. 4.2.1: terms are summed from the first l with |d| >= 1e-30
#define WG_EPS_SUM 1e-30

// device status bits (OR-ed into the status word)
#define WG_DEVERR_BETA 1
#define WG_DEVERR_TIMEOUT 2
#define WG_DEVERR_BOUNDS 4
#define WG_DEVERR_GRID 8     /* a sum over every sky order met an angle grid that is not mirror-symmetric */

// tries of a bounded mbarrier wait before it gives up (each try may also suspend the
// thread for a short hardware-chosen time); a 4 KB tile normally lands within a few
// microseconds
#define WG_WAIT_TRIES_DEFAULT (1 << 20)

namespace wg {

struct Tables;

struct DTableArgs {
    int l_max, mb_max, ms_max, n_beta;
    const double *beta;
    double *d_out;
    unsigned long long *counters;
};

struct ConvArgs {
    int l_max, mb_max, ms_max, n_beta;
    const double *beta;
    const double *a;  // interleaved complex [l][ms]
    const double *b;  // interleaved complex [l][mb]
    double *c_out;    // interleaved complex [mb][ms][j]
    unsigned long long *counters;
    int k_lo = 0, k_hi = -1;  // chain columns k = ms (mb_max + 1) + mb in [k_lo, k_hi); k_hi < 0: all
    double offset = 0.0;      // the l_min cut's offset (kernels built with the cut only)
    int wait_tries = WG_WAIT_TRIES_DEFAULT;  // tries of each TMA wait before it gives up
    // FP32 form only: per-column power-of-two weight scales, a[l][ms] 2^-ea[ms] and
    // b[l][mb] 2^-eb[mb] below 1 in magnitude (null: unscaled)
    const int *ea = nullptr, *eb = nullptr;
};

struct DTableBwdArgs {
    int l_max, mb_max, ms_max, n_beta;
    const double *beta;
    const double *grad_d;
    double *partial;  // [ncol][n_beta] workspace
    double *grad_beta;
};

struct ConvBwdArgs {
    int l_max, mb_max, ms_max, n_beta;
    const double *beta;
    const double *a, *b;      // interleaved complex
    const double *c_fwd;      // interleaved complex [mb][ms][j], may be null
    const double *grad_c;     // interleaved complex [mb][ms][j]
    double *S;                // workspace: interleaved complex [mb][ms][l]
    double *E;                // workspace: interleaved complex [mb][ms][j] (beta term), may be null
    double *grad_a, *grad_b, *grad_beta;
};

// Test hooks set through the C ABI (wigner_debug_*): whether the library's next device
// allocation is to fail as if the device were out of memory (consumes one injected
// failure), and the tries of each TMA wait for the launches that follow.
bool alloc_injected();
int wait_tries();

// launchers (return cudaError_t as int)
int launch_dtable_fp64(const DTableArgs &a, const Tables &t, void *stream);
int launch_dtable_fp32x(const DTableArgs &a, const Tables &t, void *stream);
int launch_conv_fp64(const ConvArgs &a, const Tables &t, void *stream);
int launch_ylm(const DTableArgs &a, const Tables &t, void *stream);
int launch_conv_fp64_lmin(const ConvArgs &a, const Tables &t, void *stream, bool sum_ff, bool full);
int launch_conv_fp64_full(const ConvArgs &a, const Tables &t, void *stream, bool sum_ff);
int launch_conv_fp64s(const ConvArgs &a, const Tables &t, void *stream);
int launch_conv_fp32x(const ConvArgs &a, const Tables &t, void *stream);
int launch_dtable_bwd(const DTableBwdArgs &a, const Tables &t, void *stream);
int launch_conv_bwd(const ConvBwdArgs &a, const Tables &t, void *stream);
int launch_conv_multi_tc(int l_max, int mb_max, int ms_max, int n_beta, int n_col, const double *beta,
                         const double *a, const double *b, double *c_out, unsigned long long *counters,
                         const Tables &T, int wait_tries, void *stream);
int launch_fma_peak(int pipe, int chains, int blocks, int threads, int iters, double *sink, void *stream);

}  // namespace wg
