// wg_tma.cuh -- staging the l-ordered weights of a chain column into shared memory
// with the Tensor Memory Accelerator (cp.async.bulk.tensor), completion tracked by an
// mbarrier.
//
// The sky a[l][m_sky] and the beam b[l][m_b] are row-major complex128 arrays.  Seen as
// 2-D float64 tensors of (rows l_max + 1) x (2 (ms_max + 1)) and (l_max + 1) x
// (2 (mb_max + 1)), the weights of column (m_b, m_sky) for an l-tile are the boxes
// {2 doubles, TL rows} at x = 2 m_sky and x = 2 m_b, y = the tile's first l: one
// 16-byte element per row, gathered by the TMA unit into TL consecutive double2 of
// shared memory (rows past l_max are filled with zeros).  The innermost coordinate
// x = 2 m is even, so x times 8 bytes is a multiple of 16, as tiled copies require;
// the row pitches 16 (ms_max + 1) and 16 (mb_max + 1) bytes are multiples of 16 and
// the base pointers are checked to be 16-byte aligned on the host.
#pragma once

#include <cuda.h>  // CUtensorMap (the type only; maps are encoded through the runtime's driver entry point)
#include <cuda_runtime.h>

#include "wg_internal.h"

namespace wg {

struct WeightMaps {
    CUtensorMap a;  // the sky, box {2, TL}
    CUtensorMap b;  // the beam, box {2, TL}
};

// tries of mbarrier.try_wait before a wait gives up by default; the waits of a tile
// take their limit from the launch (ConvArgs::wait_tries), the drain of copies already
// issued after a wait gave up always uses this one
constexpr int TMA_WAIT_ITERS = WG_WAIT_TRIES_DEFAULT;

__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// makes initialised mbarriers visible to the asynchronous (TMA) proxy
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

// orders this thread's earlier shared-memory accesses before later TMA writes
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int x, int y,
                                            unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// wall-clock bound of every mbarrier wait, in nanoseconds: a failed try may suspend the
// thread for a hardware-chosen time, so a count of tries alone does not bound the time a
// wait for a phase that never completes takes
constexpr unsigned long long WG_WAIT_NS = 2000000000ull;

__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Bounded wait for the completion of the mbarrier phase of the given parity; false if
// it has not completed after `tries` tries or WG_WAIT_NS nanoseconds (tries <= 0: gives
// up at once).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int tries = TMA_WAIT_ITERS) {
    if (tries <= 0) return false;
    const unsigned long long t0 = globaltimer_ns();
    for (int it = 0; it < tries; ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity)
            : "memory");
        if (done) return true;
        if (globaltimer_ns() - t0 > WG_WAIT_NS) return false;
    }
    return false;
}

// The two weight boxes of one l-tile of column (mb, ms) into (dst_a, dst_b), completing
// on `bar` (one thread; the destination buffers must no longer be read).
template <int TL>
__device__ __forceinline__ void tma_weights(const WeightMaps *wm, int mb, int ms, int ts, double2 *dst_a,
                                            double2 *dst_b, unsigned long long *bar) {
    fence_proxy_async();
    mbar_arrive_expect_tx(bar, 2u * TL * 16u);
    tma_load_2d(dst_a, &wm->a, 2 * ms, ts, bar);
    tma_load_2d(dst_b, &wm->b, 2 * mb, ts, bar);
}

// host: encode the two maps for an l-tile of TL rows (0 or a cudaError_t)
int encode_weight_maps(const double *a, const double *b, int l_max, int mb_max, int ms_max, int tl, WeightMaps *out);

}  // namespace wg
