// wg_capi.cu -- the C ABI of include/wigner.h: argument validation, the per-device
// constant tables of Sec. 4.2.2 (ln n!, P_i, Q_i) built on the host, workspace,
// status word and error reporting.  Kernels live in the other translation units.
#include <cuda_runtime.h>

#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_internal.h"

namespace {

thread_local std::string g_msg;
thread_local int g_code = 0;

int fail(int code, const std::string &msg) {
    g_msg = msg;
    g_code = code;
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    g_msg = std::string(what) + ": " + cudaGetErrorString(e);
    g_code = WG_ERR_CUDA;
    return WG_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// per-device state
// ---------------------------------------------------------------------------
struct DevState {
    int lcap = -1;  // tables valid for l_max <= lcap
    double *tab = nullptr;  // one allocation: lnf_hi, lnf_lo, P, Q (n2 each), R1, R2 (lcap+1 each)
    int *status = nullptr;
    std::vector<void *> retired;  // superseded tables (kept: other streams may still read them)
    // workspace (grown on demand; growth synchronises the device before freeing)
    void *ws = nullptr;
    size_t ws_bytes = 0;
};

std::mutex g_mu;
std::map<int, DevState> g_dev;

// test hooks (wigner_debug_inject_alloc_failures, wigner_debug_set_wait_tries)
std::atomic<int> g_inject_alloc{0};
std::atomic<int> g_wait_tries{WG_WAIT_TRIES_DEFAULT};

// Host-side construction of the constant tables (Sec. 4.2.2 and Sec. 3.2):
//   ln n! for n <= 2 lcap + 1 as a double-double from long double lgamma,
//   P_i = sqrt(1/(i+1)), Q_i = sqrt(i/(i+1)) for i <= 2 lcap + 1,
//   R1_l = 1/(l(l+1)), R2_l = (l+1)/l for 1 <= l <= lcap (0 at l = 0);
// and, for the FP32 form only, E(n) = ln((n-1)!! / n!!) for n <= 2 lcap + 1 as float-float:
//   E(2p) = ln (2p)! - 2 ln p! - 2p ln 2,  E(2p+1) = 2 ln p! + 2p ln 2 - ln (2p+1)!
// ((2p)!! = 2^p p!, (2p+1)!! = (2p+1)! / (2^p p!)).
void build_tables(int lcap, std::vector<double> &h) {
    const size_t n2 = 2 * (size_t)lcap + 2;
    const size_t n1 = (size_t)lcap + 1;
    // doubles: lnf_hi, lnf_lo, P, Q (n2 each), R1, R2 (n1 each); then float2 copies of
    // ln n!, P, Q (n2 each), R1, R2 (n1 each), then E (n2), one float2 per double slot
    h.assign(4 * n2 + 2 * n1 + 3 * n2 + 2 * n1 + n2, 0.0);
    double *lnf_hi = h.data(), *lnf_lo = lnf_hi + n2, *P = lnf_lo + n2, *Q = P + n2;
    double *R1 = Q + n2, *R2 = R1 + n1;
    float *F = reinterpret_cast<float *>(R2 + n1);
    float *lnf_f = F, *P_f = lnf_f + 2 * n2, *Q_f = P_f + 2 * n2, *R1_f = Q_f + 2 * n2, *R2_f = R1_f + 2 * n1;
    float *E_f = R2_f + 2 * n1;
    auto put_ff = [](float *dst, long double v) {
        const float hi = (float)v;
        dst[0] = hi;
        dst[1] = (float)(v - (long double)hi);
    };
    for (size_t i = 0; i < n2; ++i) {
        long double lf = lgammal((long double)i + 1.0L);
        double hi = (double)lf;
        lnf_hi[i] = hi;
        lnf_lo[i] = (double)(lf - (long double)hi);
        const long double p = sqrtl(1.0L / ((long double)i + 1.0L));
        const long double q = sqrtl((long double)i / ((long double)i + 1.0L));
        P[i] = (double)p;
        Q[i] = (double)q;
        put_ff(lnf_f + 2 * i, lf);
        put_ff(P_f + 2 * i, p);
        put_ff(Q_f + 2 * i, q);
    }
    for (size_t l = 1; l < n1; ++l) {
        const long double r1 = 1.0L / ((long double)l * ((long double)l + 1.0L));
        const long double r2 = ((long double)l + 1.0L) / (long double)l;
        R1[l] = (double)r1;
        R2[l] = (double)r2;
        put_ff(R1_f + 2 * l, r1);
        put_ff(R2_f + 2 * l, r2);
    }
    const long double ln2 = 0.693147180559945309417232121458176568L;
    for (size_t n = 0; n < n2; ++n) {
        const long double p = (long double)(n / 2);
        const long double lfp = lgammal(p + 1.0L), lfn = lgammal((long double)n + 1.0L);
        const long double e = (n & 1) ? 2.0L * lfp + 2.0L * p * ln2 - lfn : lfn - 2.0L * lfp - 2.0L * p * ln2;
        put_ff(E_f + 2 * n, e);
    }
}

int check_device(int dev) {
    int major = 0, minor = 0;
    cudaError_t e = cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    e = cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceGetAttribute");
    if (major != 10 || minor != 3)
        return fail(WG_ERR_DEVICE, "this library is built for sm_103a (GB300); device " + std::to_string(dev) +
                                       " is sm_" + std::to_string(major) + std::to_string(minor));
    return WG_OK;
}

// Ensure tables for l_max exist on the current device; fill *t.
int get_tables(int l_max, wg::Tables *t, DevState **out_state = nullptr) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &s = g_dev[dev];
    if (s.status == nullptr) {
        int rc = check_device(dev);
        if (rc != WG_OK) return rc;
        if (wg::alloc_injected()) return fail(WG_ERR_ALLOC, "cudaMalloc(status): injected allocation failure");
        e = cudaMalloc(&s.status, sizeof(int));
        if (e != cudaSuccess) {
            s.status = nullptr;
            return fail(WG_ERR_ALLOC, std::string("cudaMalloc(status): ") + cudaGetErrorString(e));
        }
        e = cudaMemset(s.status, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
        // the memset runs on the legacy stream: finish it before any stream may read the word
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize(status)");
    }
    if (s.lcap < l_max) {
        int lcap = 1024;
        while (lcap < l_max) lcap *= 2;
        if (lcap > WG_LMAX) lcap = WG_LMAX;
        std::vector<double> h;
        build_tables(lcap, h);
        double *d = nullptr;
        if (wg::alloc_injected()) return fail(WG_ERR_ALLOC, "cudaMalloc(tables): injected allocation failure");
        e = cudaMalloc(&d, h.size() * sizeof(double));
        if (e != cudaSuccess) return fail(WG_ERR_ALLOC, std::string("cudaMalloc(tables): ") + cudaGetErrorString(e));
        e = cudaMemcpy(d, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice);
        // a copy from pageable memory may return before its transfer has landed, and a
        // kernel on a non-blocking stream is not ordered after it: wait for the device
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            cudaFree(d);
            return cuda_fail(e, "cudaMemcpy(tables)");
        }
        if (s.tab) s.retired.push_back(s.tab);
        s.tab = d;
        s.lcap = lcap;
    }
    const size_t n2 = 2 * (size_t)s.lcap + 2, n1 = (size_t)s.lcap + 1;
    t->lnf_hi = s.tab;
    t->lnf_lo = s.tab + n2;
    t->P = s.tab + 2 * n2;
    t->Q = s.tab + 3 * n2;
    t->R1 = s.tab + 4 * n2;
    t->R2 = s.tab + 4 * n2 + n1;
    const float2 *F = reinterpret_cast<const float2 *>(s.tab + 4 * n2 + 2 * n1);
    t->lnf_f = F;
    t->P_f = F + n2;
    t->Q_f = F + 2 * n2;
    t->R1_f = F + 3 * n2;
    t->R2_f = F + 3 * n2 + n1;
    t->E_f = F + 3 * n2 + 2 * n1;
    t->lcap = s.lcap;
    t->status = s.status;
    (void)n1;
    if (out_state) *out_state = &s;
    return WG_OK;
}

// Workspace of at least `bytes` on the current device.  Growth synchronises the
// device first, so buffers in use by earlier work on any stream are not freed early.
int get_workspace(size_t bytes, void **ws) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    std::lock_guard<std::mutex> lk(g_mu);
    DevState &s = g_dev[dev];
    if (s.ws_bytes < bytes) {
        e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize(workspace)");
        if (s.ws) cudaFree(s.ws);
        s.ws = nullptr;
        s.ws_bytes = 0;
        size_t want = bytes + bytes / 4;
        if (wg::alloc_injected()) return fail(WG_ERR_ALLOC, "cudaMalloc(workspace): injected allocation failure");
        e = cudaMalloc(&s.ws, want);
        if (e != cudaSuccess) {
            s.ws = nullptr;
            return fail(WG_ERR_ALLOC, std::string("cudaMalloc(workspace): ") + cudaGetErrorString(e));
        }
        s.ws_bytes = want;
    }
    *ws = s.ws;
    return WG_OK;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_orders(int l_max, int mb_max, int ms_max, int n_beta) {
    if (l_max < 0 || l_max > WG_LMAX)
        return fail(WG_ERR_ARG, "l_max must be in [0, " + std::to_string(WG_LMAX) + "]");
    if (mb_max < 0 || mb_max > l_max) return fail(WG_ERR_ARG, "mb_max must be in [0, l_max]");
    if (ms_max < 0 || ms_max > l_max) return fail(WG_ERR_ARG, "ms_max must be in [0, l_max]");
    if (n_beta < 0) return fail(WG_ERR_ARG, "n_beta must be >= 0");
    return WG_OK;
}

int check_ptr(const void *p, size_t align, const char *name) {
    if (p == nullptr) return fail(WG_ERR_ARG, std::string(name) + " is NULL");
    if (!aligned(p, align)) return fail(WG_ERR_ARG, std::string(name) + " is not " + std::to_string(align) + "-byte aligned");
    return WG_OK;
}

#define WG_TRY(x)                     \
    do {                              \
        int rc_ = (x);                \
        if (rc_ != WG_OK) return rc_; \
    } while (0)

int launch_rc(int err, const char *what) {
    if (err == (int)cudaErrorMemoryAllocation)  // a launcher's stream-ordered scratch
        return fail(WG_ERR_ALLOC, std::string(what) + ": " + cudaGetErrorString(cudaErrorMemoryAllocation));
    if (err != 0) return cuda_fail((cudaError_t)err, what);
    return WG_OK;
}

}  // namespace

namespace wg {
void set_last_error(const std::string &msg, int code) {
    g_msg = msg;
    g_code = code;
}
int tables_for(int l_max, Tables *t) { return get_tables(l_max, t); }
bool alloc_injected() {
    int n = g_inject_alloc.load();
    while (n > 0)
        if (g_inject_alloc.compare_exchange_weak(n, n - 1)) return true;
    return false;
}
int wait_tries() { return g_wait_tries.load(); }
}  // namespace wg

extern "C" {

int wigner_version(void) { return 1; }

int wigner_built_arch(void) { return 1003; }

const char *wigner_last_error_message(void) { return g_msg.c_str(); }

int wigner_last_error(void) { return g_code; }

const char *wigner_error_string(int code) {
    switch (code) {
        case WG_OK: return "ok";
        case WG_ERR_ARG: return "invalid argument";
        case WG_ERR_CUDA: return "CUDA runtime error";
        case WG_ERR_ALLOC: return "device allocation failed";
        case WG_ERR_TIMEOUT: return "bounded device wait timed out";
        case WG_ERR_DEVICE: return "unsupported device";
        case WG_ERR_UNSUPPORTED: return "not supported by this library version";
        default: return "unknown error";
    }
}

int wigner_device_status(void *stream) {
    try {
        wg::Tables t;
        WG_TRY(get_tables(0, &t));
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "cudaStreamSynchronize");
        int h = 0;
        e = cudaMemcpy(&h, t.status, sizeof(int), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemcpy(status)");
        e = cudaMemset(t.status, 0, sizeof(int));
        if (e != cudaSuccess) return cuda_fail(e, "cudaMemset(status)");
        if (h & WG_DEVERR_TIMEOUT) return fail(WG_ERR_TIMEOUT, "a bounded device wait gave up");
        if (h & WG_DEVERR_BOUNDS) return fail(WG_ERR_DEVICE, "a device-side bounds check failed");
        if (h & WG_DEVERR_BETA) return fail(WG_ERR_ARG, "an angle was outside [0, pi] (or interior required)");
        if (h & WG_DEVERR_GRID) return fail(WG_ERR_ARG, "the angle grid is not mirror-symmetric (beta[N-1-j] != pi - beta[j])");
        return WG_OK;
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

int wigner_d_table(int l_max, int mb_max, int ms_max, int n_beta, const double *beta, wg_form form,
                   double *d_out, wg_counter *counters, void *stream) {
    try {
        WG_TRY(check_orders(l_max, mb_max, ms_max, n_beta));
        if (form != WG_FP64 && form != WG_FP32X && form != WG_FP64S) return fail(WG_ERR_ARG, "unknown form");
        if (n_beta == 0) return WG_OK;
        WG_TRY(check_ptr(beta, 8, "beta"));
        WG_TRY(check_ptr(d_out, 8, "d_out"));
        if (counters && !aligned(counters, 8)) return fail(WG_ERR_ARG, "counters misaligned");
        wg::Tables t;
        WG_TRY(get_tables(l_max, &t));
        wg::DTableArgs a{l_max, mb_max, ms_max, n_beta, beta, d_out, counters};
        if (form != WG_FP32X) return launch_rc(wg::launch_dtable_fp64(a, t, stream), "dtable_fp64 launch");
        return launch_rc(wg::launch_dtable_fp32x(a, t, stream), "dtable_fp32x launch");
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

int wigner_ylm(int l_max, int m_max, int n_theta, const double *theta, double *out, void *stream) {
    try {
        WG_TRY(check_orders(l_max, m_max, 0, n_theta));
        if (n_theta == 0) return WG_OK;
        WG_TRY(check_ptr(theta, 8, "theta"));
        WG_TRY(check_ptr(out, 8, "out"));
        wg::Tables t;
        WG_TRY(get_tables(l_max, &t));
        wg::DTableArgs a{l_max, m_max, 0, n_theta, theta, out, nullptr};
        return launch_rc(wg::launch_ylm(a, t, stream), "ylm launch");
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

int wigner_d_table_backward(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                            const double *grad_d, double *grad_beta, void *stream) {
    try {
        WG_TRY(check_orders(l_max, mb_max, ms_max, n_beta));
        if (n_beta == 0) return WG_OK;
        WG_TRY(check_ptr(beta, 8, "beta"));
        WG_TRY(check_ptr(grad_d, 8, "grad_d"));
        WG_TRY(check_ptr(grad_beta, 8, "grad_beta"));
        wg::Tables t;
        WG_TRY(get_tables(l_max + 1, &t));
        const size_t ncol = (size_t)(mb_max + 1) * (ms_max + 2);
        void *ws = nullptr;
        WG_TRY(get_workspace(ncol * (size_t)n_beta * sizeof(double), &ws));
        wg::DTableBwdArgs a{l_max, mb_max, ms_max, n_beta, beta, grad_d, (double *)ws, grad_beta};
        return launch_rc(wg::launch_dtable_bwd(a, t, stream), "dtable_bwd launch");
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

int wigner_conv_sum(int l_max, int mb_max, int ms_max, int n_beta, const double *beta, const wg_c64 *a,
                    const wg_c64 *b, wg_form form, wg_c64 *c_out, wg_counter *counters, void *stream) {
    try {
        WG_TRY(check_orders(l_max, mb_max, ms_max, n_beta));
        if (form != WG_FP64 && form != WG_FP32X && form != WG_FP64S) return fail(WG_ERR_ARG, "unknown form");
        if (n_beta == 0) return WG_OK;
        WG_TRY(check_ptr(beta, 8, "beta"));
        WG_TRY(check_ptr(a, 16, "a"));
        WG_TRY(check_ptr(b, 16, "b"));
        WG_TRY(check_ptr(c_out, 16, "c_out"));
        if (counters && !aligned(counters, 8)) return fail(WG_ERR_ARG, "counters misaligned");
        wg::Tables t;
        WG_TRY(get_tables(l_max, &t));
        wg::ConvArgs ca{l_max, mb_max, ms_max, n_beta, beta, (const double *)a, (const double *)b,
                        (double *)c_out, counters};
        ca.wait_tries = wg::wait_tries();
        if (form == WG_FP64) return launch_rc(wg::launch_conv_fp64(ca, t, stream), "conv_fp64 launch");
        if (form == WG_FP64S) return launch_rc(wg::launch_conv_fp64s(ca, t, stream), "conv_fp64s launch");
        return launch_rc(wg::launch_conv_fp32x(ca, t, stream), "conv_fp32x launch");
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

int wigner_conv_sum_full(int l_max, int mb_max, int ms_max, int n_beta, const double *beta, const wg_c64 *a,
                         const wg_c64 *b, wg_form form, wg_c64 *c_out, wg_counter *counters, void *stream) {
    try {
        WG_TRY(check_orders(l_max, mb_max, ms_max, n_beta));
        if (form == WG_FP32X) return fail(WG_ERR_UNSUPPORTED, "the sum over every sky order is FP64 / FP64S only");
        if (form != WG_FP64 && form != WG_FP64S) return fail(WG_ERR_ARG, "unknown form");
        if (n_beta == 0) return WG_OK;
        WG_TRY(check_ptr(beta, 8, "beta"));
        WG_TRY(check_ptr(a, 16, "a"));
        WG_TRY(check_ptr(b, 16, "b"));
        WG_TRY(check_ptr(c_out, 16, "c_out"));
        if (counters && !aligned(counters, 8)) return fail(WG_ERR_ARG, "counters misaligned");
        wg::Tables t;
        WG_TRY(get_tables(l_max, &t));
        wg::ConvArgs ca{l_max, mb_max, ms_max, n_beta, beta, (const double *)a, (const double *)b,
                        (double *)c_out, counters};
        ca.wait_tries = wg::wait_tries();
        return launch_rc(wg::launch_conv_fp64_full(ca, t, stream, form == WG_FP64S), "conv_fp64_full launch");
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

int wigner_conv_sum_lmin(int l_max, int mb_max, int ms_max, int n_beta, const double *beta, const wg_c64 *a,
                         const wg_c64 *b, wg_form form, double offset, int full, wg_c64 *c_out,
                         wg_counter *counters, void *stream) {
    try {
        WG_TRY(check_orders(l_max, mb_max, ms_max, n_beta));
        if (form == WG_FP32X) return fail(WG_ERR_UNSUPPORTED, "the l_min cut is FP64 / FP64S only");
        if (form != WG_FP64 && form != WG_FP64S) return fail(WG_ERR_ARG, "unknown form");
        if (offset != offset) return fail(WG_ERR_ARG, "offset is NaN");
        if (n_beta == 0) return WG_OK;
        WG_TRY(check_ptr(beta, 8, "beta"));
        WG_TRY(check_ptr(a, 16, "a"));
        WG_TRY(check_ptr(b, 16, "b"));
        WG_TRY(check_ptr(c_out, 16, "c_out"));
        if (counters && !aligned(counters, 8)) return fail(WG_ERR_ARG, "counters misaligned");
        wg::Tables t;
        WG_TRY(get_tables(l_max, &t));
        wg::ConvArgs ca{l_max, mb_max, ms_max, n_beta, beta, (const double *)a, (const double *)b,
                        (double *)c_out, counters};
        ca.offset = offset;
        ca.wait_tries = wg::wait_tries();
        return launch_rc(wg::launch_conv_fp64_lmin(ca, t, stream, form == WG_FP64S, full != 0),
                         "conv_fp64_lmin launch");
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

int wigner_conv_sum_backward(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                             const wg_c64 *a, const wg_c64 *b, const wg_c64 *c_fwd, const wg_c64 *grad_c,
                             wg_c64 *grad_a, wg_c64 *grad_b, double *grad_beta, wg_form form, void *stream) {
    try {
        WG_TRY(check_orders(l_max, mb_max, ms_max, n_beta));
        if (form != WG_FP64 && form != WG_FP64S) return fail(WG_ERR_UNSUPPORTED, "the backward pass is FP64 only");
        WG_TRY(check_ptr(a, 16, "a"));
        WG_TRY(check_ptr(b, 16, "b"));
        if (grad_a && !aligned(grad_a, 16)) return fail(WG_ERR_ARG, "grad_a misaligned");
        if (grad_b && !aligned(grad_b, 16)) return fail(WG_ERR_ARG, "grad_b misaligned");
        if (grad_beta && !aligned(grad_beta, 8)) return fail(WG_ERR_ARG, "grad_beta misaligned");
        if (!grad_a && !grad_b && !grad_beta) return WG_OK;
        if (n_beta > 0) {
            WG_TRY(check_ptr(beta, 8, "beta"));
            WG_TRY(check_ptr(grad_c, 16, "grad_c"));
            if (grad_beta) WG_TRY(check_ptr(c_fwd, 16, "c_fwd"));
        }
        wg::Tables t;
        WG_TRY(get_tables(l_max + 1, &t));
        const size_t ncol = (size_t)(mb_max + 1) * (ms_max + 1);
        const size_t s_elems = ncol * (size_t)(l_max + 1) * 2;
        const size_t e_elems = grad_beta ? ncol * (size_t)n_beta * 2 : 0;
        void *ws = nullptr;
        WG_TRY(get_workspace((s_elems + e_elems) * sizeof(double), &ws));
        wg::ConvBwdArgs ba{l_max, mb_max, ms_max, n_beta, beta, (const double *)a, (const double *)b,
                           (const double *)c_fwd, (const double *)grad_c, (double *)ws,
                           grad_beta ? (double *)ws + s_elems : nullptr, (double *)grad_a, (double *)grad_b,
                           grad_beta};
        return launch_rc(wg::launch_conv_bwd(ba, t, stream), "conv_bwd launch");
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

struct wg_plan {
    int device;
    wg_params prm;
};

int wigner_plan_create(wg_plan **plan, const wg_params *prm) {
    try {
        if (!plan || !prm) return fail(WG_ERR_ARG, "plan and params must not be NULL");
        *plan = nullptr;
        WG_TRY(check_orders(prm->l_max_cap, prm->mb_max_cap, prm->ms_max_cap, prm->n_beta_cap));
        wg::Tables t;
        WG_TRY(get_tables(prm->l_max_cap + 1, &t));
        if (prm->reserve_backward) {
            const size_t ncol = (size_t)(prm->mb_max_cap + 1) * (prm->ms_max_cap + 2);
            const size_t conv = ncol * (size_t)(prm->l_max_cap + 1) * 16 + ncol * (size_t)prm->n_beta_cap * 16;
            const size_t dtab = ncol * (size_t)prm->n_beta_cap * sizeof(double);
            void *ws = nullptr;
            WG_TRY(get_workspace(conv > dtab ? conv : dtab, &ws));
        }
        cudaError_t e = cudaDeviceSynchronize();
        if (e != cudaSuccess) return cuda_fail(e, "cudaDeviceSynchronize(plan)");
        wg_plan *p = new (std::nothrow) wg_plan;
        if (!p) return fail(WG_ERR_ALLOC, "host allocation failed");
        cudaGetDevice(&p->device);
        p->prm = *prm;
        *plan = p;
        return WG_OK;
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}

void wigner_plan_destroy(wg_plan *plan) { delete plan; }

int wigner_debug_inject_alloc_failures(int n) {
    if (n < 0) return fail(WG_ERR_ARG, "n must be >= 0");
    g_inject_alloc.store(n);
    return WG_OK;
}

int wigner_debug_set_wait_tries(int tries) {
    if (tries < 0) return fail(WG_ERR_ARG, "tries must be >= 0");
    g_wait_tries.store(tries == 0 ? 0 : tries);
    return WG_OK;
}

int wigner_debug_wait_tries(void) { return g_wait_tries.load(); }

int wigner_fma_peak(int pipe, int chains, int blocks, int threads, int iters, double *sink,
                    unsigned long long *fma_ops, void *stream) {
    if (pipe != 0 && pipe != 1) return fail(WG_ERR_ARG, "pipe must be 0 (FP64) or 1 (FP32)");
    if (chains != 1 && chains != 2 && chains != 4 && chains != 8 && chains != 16)
        return fail(WG_ERR_ARG, "chains must be 1, 2, 4, 8 or 16");
    if (blocks <= 0 || threads <= 0 || threads > 256 || (threads % 32) || iters <= 0)
        return fail(WG_ERR_ARG, "bad launch shape");
    WG_TRY(check_ptr(sink, 8, "sink"));
    if (fma_ops) *fma_ops = (unsigned long long)blocks * threads * (unsigned long long)iters * (unsigned long long)chains;
    return launch_rc(wg::launch_fma_peak(pipe, chains, blocks, threads, iters, sink, stream), "fma_peak launch");
}

}  // extern "C"
