// wg_noalloc.cu -- an allocation-free variant of the fused FP64 l-sum entry point.
//
// Why: wigner_conv_sum keeps its constant tables (ln n!, P_i, Q_i, 1/(l(l+1)), (l+1)/l)
// in device memory that the library allocates with cudaMalloc on first use.  Some
// callers cannot allow that: code that runs while a CUDA graph is being captured, code
// that owns the whole device-memory budget through its own pool, or a real-time loop
// that must never enter the driver's allocator.  wigner_conv_sum_noalloc runs the same
// kernel with its tables in a fixed-size array compiled into this library instead, so
// it never allocates device (or host heap) memory.
//
// The array below holds the tables for l_max <= WG_NOALLOC_LMAX (640 KiB of doubles).
// It is a file-scope __device__ object, so it exists on every GPU that loads this
// library until the process exits.  In host code its name is only a host-side handle:
// the device address is obtained once per device with cudaGetSymbolAddress while that
// device is current, and that address is what the kernel receives.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <string>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_internal.h"

namespace wg {
void set_last_error(const std::string &msg, int code);  // wg_capi.cu: text for wigner_last_error_message
}

namespace {

struct ErrSink {  // g_err = "..." forwards the text to wigner_last_error_message
    int code = WG_ERR_ARG;
    ErrSink &operator=(const std::string &m) {
        wg::set_last_error(m, code);
        return *this;
    }
};
thread_local ErrSink g_err;

constexpr int kLcap = WG_NOALLOC_LMAX;
constexpr size_t kN2 = 2 * (size_t)kLcap + 2;  // ln n!, P_i, Q_i: n, i <= 2 l_max + 1
constexpr size_t kN1 = (size_t)kLcap + 1;      // 1/(l(l+1)), (l+1)/l: l <= l_max
constexpr size_t kWords = 4 * kN2 + 2 * kN1;

static __device__ __align__(256) double g_noalloc_tables[kWords];
// this entry point's own status word (WG_DEVERR_* bits), read and cleared by
// wigner_noalloc_status
static __device__ int g_noalloc_status;

// Host copy of the same tables, built once per process into static storage (no heap).
static double g_host_tables[kWords];
static std::once_flag g_host_once;

constexpr int kMaxDevices = 64;
static double *g_dev_ptr[kMaxDevices];     // device address of g_noalloc_tables, per device
static int *g_status_ptr[kMaxDevices];     // device address of g_noalloc_status, per device
static std::mutex g_mu;
static const int kZero = 0;


// Same definitions as the tables of the allocating path (Sec. 4.2.2 and Sec. 3.2):
// ln n! as hi + lo from long double lgamma; P_i = sqrt(1/(i+1)); Q_i = sqrt(i/(i+1));
// R1_l = 1/(l(l+1)), R2_l = (l+1)/l (both 0 at l = 0).
void fill_host_tables() {
    double *lnf_hi = g_host_tables, *lnf_lo = lnf_hi + kN2, *P = lnf_lo + kN2, *Q = P + kN2;
    double *R1 = Q + kN2, *R2 = R1 + kN1;
    for (size_t i = 0; i < kN2; ++i) {
        const long double lf = lgammal((long double)i + 1.0L);
        const double hi = (double)lf;
        lnf_hi[i] = hi;
        lnf_lo[i] = (double)(lf - (long double)hi);
        P[i] = (double)sqrtl(1.0L / ((long double)i + 1.0L));
        Q[i] = (double)sqrtl((long double)i / ((long double)i + 1.0L));
    }
    R1[0] = 0.0;
    R2[0] = 0.0;
    for (size_t l = 1; l < kN1; ++l) {
        R1[l] = (double)(1.0L / ((long double)l * ((long double)l + 1.0L)));
        R2[l] = (double)(((long double)l + 1.0L) / (long double)l);
    }
}

// Set-up for the current device (first call on that device only): look up the device
// addresses of the array and of the status word, upload the tables, clear the word, and
// wait for the device before publishing the addresses (a copy from pageable memory may
// return before its transfer has landed, and the caller's stream need not be ordered
// after the legacy stream the copies run on).
int device_tables(double **out, int **status) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_err.code = WG_ERR_CUDA;
        g_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return WG_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        g_err.code = WG_ERR_DEVICE;
        g_err = "device ordinal beyond the supported range";
        return WG_ERR_DEVICE;
    }
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_dev_ptr[dev] == nullptr) {
        int major = 0, minor = 0;
        cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
        if (major != 10 || minor != 3) {
            g_err.code = WG_ERR_DEVICE;
            g_err = "this library is built for sm_103a (GB300)";
            return WG_ERR_DEVICE;
        }
        std::call_once(g_host_once, fill_host_tables);
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_noalloc_tables);
        if (e != cudaSuccess || p == nullptr) {
            g_err.code = WG_ERR_CUDA;
            g_err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return WG_ERR_CUDA;
        }
        int *st = nullptr;
        e = cudaGetSymbolAddress((void **)&st, g_noalloc_status);
        if (e != cudaSuccess || st == nullptr) {
            g_err.code = WG_ERR_CUDA;
            g_err = std::string("cudaGetSymbolAddress(status): ") + cudaGetErrorString(e);
            return WG_ERR_CUDA;
        }
        e = cudaMemcpyToSymbol(g_noalloc_tables, g_host_tables, sizeof(g_host_tables), 0, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_noalloc_status, &kZero, sizeof(int), 0, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
        if (e != cudaSuccess) {
            g_err.code = WG_ERR_CUDA;
            g_err = std::string("cudaMemcpyToSymbol: ") + cudaGetErrorString(e);
            return WG_ERR_CUDA;
        }
        g_status_ptr[dev] = st;
        g_dev_ptr[dev] = p;
    }
    *out = g_dev_ptr[dev];
    *status = g_status_ptr[dev];
    return WG_OK;
}

bool is_aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

extern "C" int wigner_conv_sum_noalloc(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                                       const wg_c64 *a, const wg_c64 *b, wg_c64 *c_out, void *stream) {
    g_err.code = WG_ERR_ARG;
    if (l_max < 0 || l_max > kLcap) {
        g_err = "wigner_conv_sum_noalloc: l_max must be in [0, " + std::to_string(kLcap) +
                "] (its tables live in a fixed array); use wigner_conv_sum for larger l_max";
        return WG_ERR_ARG;
    }
    if (mb_max < 0 || mb_max > l_max || ms_max < 0 || ms_max > l_max || n_beta < 0) {
        g_err = "wigner_conv_sum_noalloc: need 0 <= mb_max, ms_max <= l_max and n_beta >= 0";
        return WG_ERR_ARG;
    }
    if (n_beta == 0) return WG_OK;
    if (!beta || !a || !b || !c_out || !is_aligned(beta, 8) || !is_aligned(a, 16) || !is_aligned(b, 16) ||
        !is_aligned(c_out, 16)) {
        g_err = "wigner_conv_sum_noalloc: a NULL or misaligned pointer";
        return WG_ERR_ARG;
    }
    double *tab = nullptr;
    int *status = nullptr;
    int rc = device_tables(&tab, &status);
    if (rc != WG_OK) return rc;
    wg::Tables t;
    t.lnf_hi = tab;
    t.lnf_lo = tab + kN2;
    t.P = tab + 2 * kN2;
    t.Q = tab + 3 * kN2;
    t.R1 = tab + 4 * kN2;
    t.R2 = tab + 4 * kN2 + kN1;
    t.lnf_f = t.P_f = t.Q_f = t.R1_f = t.R2_f = t.E_f = nullptr;  // used only by the FP32 form
    t.lcap = kLcap;
    t.status = status;  // read by wigner_noalloc_status
    wg::ConvArgs ca{l_max, mb_max, ms_max, n_beta, beta, (const double *)a, (const double *)b, (double *)c_out,
                    nullptr};
    ca.wait_tries = wg::wait_tries();
    const int err = wg::launch_conv_fp64(ca, t, stream);
    if (err != 0) {
        g_err.code = WG_ERR_CUDA;
        g_err = std::string("conv_fp64 launch: ") + cudaGetErrorString((cudaError_t)err);
        return WG_ERR_CUDA;
    }
    return WG_OK;
}


// Reads and clears this entry point's status word on the current device, after
// synchronising `stream`.  Allocates nothing: the word is a file-scope device variable
// read and written by symbol copies.
extern "C" int wigner_noalloc_status(void *stream) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        g_err.code = WG_ERR_CUDA;
        g_err = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
        return WG_ERR_CUDA;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        g_err.code = WG_ERR_DEVICE;
        g_err = "device ordinal beyond the supported range";
        return WG_ERR_DEVICE;
    }
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_status_ptr[dev] == nullptr) return WG_OK;  // nothing has run on this device
    }
    e = cudaStreamSynchronize((cudaStream_t)stream);
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&h, g_noalloc_status, sizeof(int), 0, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_noalloc_status, &kZero, sizeof(int), 0, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        g_err.code = WG_ERR_CUDA;
        g_err = std::string("wigner_noalloc_status: ") + cudaGetErrorString(e);
        return WG_ERR_CUDA;
    }
    if (h & WG_DEVERR_TIMEOUT) {
        g_err.code = WG_ERR_TIMEOUT;
        g_err = "wigner_conv_sum_noalloc: a bounded device wait gave up (the abandoned outputs are NaN)";
        return WG_ERR_TIMEOUT;
    }
    if (h & WG_DEVERR_BETA) {
        g_err.code = WG_ERR_ARG;
        g_err = "wigner_conv_sum_noalloc: an angle was outside [0, pi] (its outputs are NaN)";
        return WG_ERR_ARG;
    }
    return WG_OK;
}
