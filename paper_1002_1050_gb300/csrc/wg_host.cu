// wg_host.cu -- the fused sum (Sec. 4.1, Eq. convdef) from and to HOST buffers, with the
// download of C overlapped with the computation.
//
// The inputs go up once on the caller's stream.  The chain columns are then processed
// in NBLK launches over blocks of consecutive sky orders m_sky, cut so that the blocks
// hold about equal work (a column's chains have l_max + 1 - max(m_b, m_sky) elements);
// the output of a block, C[m_b][m_sky range][beta] for every m_b, is one 2-D copy, made
// on a second (library-owned) stream as soon as the block's launch has finished, while
// the next block computes.
// Device buffers come from a library-owned stream-ordered memory pool, so concurrent
// calls on different streams do not share them.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_internal.h"

namespace wg {
void set_last_error(const std::string &msg, int code);
int tables_for(int l_max, Tables *t);  // wg_capi.cu
int host_pool(cudaMemPool_t *pool);
}  // namespace wg

namespace {

// Blocks: one by default -- at ~200 GB/s the download of C (1.2 GB at the L = 4096
// workload) takes ~7 ms against a second of computation, while every extra launch loses
// its tail (measured: four blocks cost ~30 ms more than they hid).  WIGNER_HOST_BLOCKS
// (1..16) sets another count, for workloads with a larger output-to-work ratio.
int n_blocks() {
    const char *v = std::getenv("WIGNER_HOST_BLOCKS");
    const int n = v ? std::atoi(v) : 1;
    return n < 1 ? 1 : (n > 16 ? 16 : n);
}
constexpr int MAX_DEV = 64;

struct HostCallState {
    cudaMemPool_t pool = nullptr;
    cudaStream_t copy = nullptr;
};
std::mutex g_mu;
HostCallState g_state[MAX_DEV];

int fail(int code, const std::string &msg) {
    wg::set_last_error(msg, code);
    return code;
}

int cuda_fail(cudaError_t e, const char *what) {
    return fail(WG_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

int state_for_device(HostCallState **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= MAX_DEV) return fail(WG_ERR_DEVICE, "device index out of range");
    std::lock_guard<std::mutex> lk(g_mu);
    HostCallState &s = g_state[dev];
    if (!s.pool) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&s.pool, &props);
        if (e != cudaSuccess) {
            s.pool = nullptr;
            return cuda_fail(e, "cudaMemPoolCreate");
        }
        unsigned long long keep = ~0ULL;  // keep freed blocks for the next call
        cudaMemPoolSetAttribute(s.pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (!s.copy) {
        e = cudaStreamCreateWithFlags(&s.copy, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            s.copy = nullptr;
            return cuda_fail(e, "cudaStreamCreate(copy)");
        }
    }
    *out = &s;
    return WG_OK;
}

// sky-order boundaries of NBLK blocks of about equal work: block p is ms in [cut[p], cut[p+1])
std::vector<int> block_cuts(int l_max, int mb_max, int ms_max, int NBLK) {
    std::vector<double> w(ms_max + 1);
    double tot = 0.0;
    for (int ms = 0; ms <= ms_max; ++ms) {
        double c = 0.0;
        for (int mb = 0; mb <= mb_max; ++mb) c += (double)(l_max + 1 - std::max(mb, ms));
        w[ms] = c;
        tot += c;
    }
    std::vector<int> cut{0};
    double acc = 0.0;
    for (int ms = 0; ms <= ms_max; ++ms) {
        acc += w[ms];
        if ((int)cut.size() < NBLK && acc >= tot * (double)cut.size() / NBLK && ms < ms_max) cut.push_back(ms + 1);
    }
    cut.push_back(ms_max + 1);
    return cut;
}

}  // namespace

// the library's stream-ordered memory pool of the current device (also used by the
// data cube's scratch spectrum)
int wg::host_pool(cudaMemPool_t *pool) {
    HostCallState *st = nullptr;
    const int rc = state_for_device(&st);
    if (rc == WG_OK) *pool = st->pool;
    return rc;
}

extern "C" int wigner_conv_sum_host(int l_max, int mb_max, int ms_max, int n_beta, const double *beta_host,
                                    const wg_c64 *a_host, const wg_c64 *b_host, wg_form form, wg_c64 *c_host,
                                    void *stream) {
    try {
        if (l_max < 0 || l_max > WG_LMAX) return fail(WG_ERR_ARG, "l_max must be in [0, WG_LMAX]");
        if (mb_max < 0 || mb_max > l_max) return fail(WG_ERR_ARG, "mb_max must be in [0, l_max]");
        if (ms_max < 0 || ms_max > l_max) return fail(WG_ERR_ARG, "ms_max must be in [0, l_max]");
        if (n_beta < 0) return fail(WG_ERR_ARG, "n_beta must be >= 0");
        if (form != WG_FP64 && form != WG_FP32X && form != WG_FP64S) return fail(WG_ERR_ARG, "unknown form");
        if (n_beta == 0) return WG_OK;
        if (!beta_host || !a_host || !b_host || !c_host) return fail(WG_ERR_ARG, "NULL host buffer");
        HostCallState *st = nullptr;
        int rc = state_for_device(&st);
        if (rc != WG_OK) return rc;
        wg::Tables t;
        rc = wg::tables_for(l_max, &t);
        if (rc != WG_OK) return rc;
        cudaStream_t s = (cudaStream_t)stream;
        const size_t MB1 = (size_t)mb_max + 1, MS1 = (size_t)ms_max + 1, L1 = (size_t)l_max + 1, NB = (size_t)n_beta;
        const size_t n_beta_b = NB * 8, n_a = L1 * MS1 * 16, n_b = L1 * MB1 * 16, n_c = MB1 * MS1 * NB * 16;
        void *d_beta = nullptr, *d_a = nullptr, *d_b = nullptr, *d_c = nullptr;
        // buffers go back to the pool in stream order on every exit
        auto release = [&] {
            for (void *p : {d_c, d_b, d_a, d_beta})
                if (p) cudaFreeAsync(p, s);
        };
        cudaError_t e = wg::alloc_injected() ? cudaErrorMemoryAllocation
                                             : cudaMallocFromPoolAsync(&d_beta, n_beta_b, st->pool, s);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&d_a, n_a, st->pool, s);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&d_b, n_b, st->pool, s);
        if (e == cudaSuccess) e = cudaMallocFromPoolAsync(&d_c, n_c, st->pool, s);
        if (e != cudaSuccess) {
            release();
            return fail(WG_ERR_ALLOC, std::string("device buffers: ") + cudaGetErrorString(e));
        }
        e = cudaMemcpyAsync(d_beta, beta_host, n_beta_b, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_a, a_host, n_a, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(d_b, b_host, n_b, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(e, "upload");
        }

        const std::vector<int> cut = block_cuts(l_max, mb_max, ms_max, n_blocks());
        std::vector<cudaEvent_t> evs;
        for (size_t p = 0; p + 1 < cut.size() && e == cudaSuccess; ++p) {
            const int ms_a = cut[p], ms_b = cut[p + 1];
            if (ms_b <= ms_a) continue;
            wg::ConvArgs ca{l_max, mb_max, ms_max, n_beta, (const double *)d_beta, (const double *)d_a,
                            (const double *)d_b, (double *)d_c, nullptr};
            ca.k_lo = ms_a * (int)MB1;
            ca.k_hi = ms_b * (int)MB1;
            int le = form == WG_FP64 ? wg::launch_conv_fp64(ca, t, s)
                                     : (form == WG_FP64S ? wg::launch_conv_fp64s(ca, t, s) : wg::launch_conv_fp32x(ca, t, s));
            if (le != 0) {
                e = (cudaError_t)le;
                break;
            }
            cudaEvent_t ev;
            e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e != cudaSuccess) break;
            evs.push_back(ev);
            e = cudaEventRecord(ev, s);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st->copy, ev, 0);
            // C[mb][ms_a .. ms_b)[:] for every mb: MB1 rows of (ms_b - ms_a) NB complex values
            const size_t off = (size_t)ms_a * NB * 16, pitch = MS1 * NB * 16;
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync((char *)c_host + off, pitch, (const char *)d_c + off, pitch,
                                      (size_t)(ms_b - ms_a) * NB * 16, MB1, cudaMemcpyDeviceToHost, st->copy);
        }
        // the caller's stream waits for the downloads issued so far (also after an error,
        // so that the buffers are released only once nothing reads them)
        cudaEvent_t done;
        cudaError_t e2 = cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
        if (e2 == cudaSuccess) {
            evs.push_back(done);
            e2 = cudaEventRecord(done, st->copy);
        }
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, done, 0);
        if (e2 != cudaSuccess) cudaStreamSynchronize(st->copy);
        for (cudaEvent_t ev : evs) cudaEventDestroy(ev);
        release();
        if (e != cudaSuccess) return cuda_fail(e, "conv launch / download");
        if (e2 != cudaSuccess) return cuda_fail(e2, "download join");
        return WG_OK;
    } catch (const std::bad_alloc &) {
        return fail(WG_ERR_ALLOC, "host allocation failed");
    }
}
