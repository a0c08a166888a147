// wg_multi_tc.cu -- many weight columns on the tensor cores: the l-sum of Eq. convdef
// for a batch of skies that share one beam (the Monte-Carlo use of Sec. 4.1), fused
// with the FP64 l-recursion (Sec. 3.2, Sec. 4.2.2 tables).
//
// For one chain column (m_b, m_sky) and K skies a^(k), the sum over l of a CTA's 128
// angles is a real matrix product
//     C_k(beta_j) = sum_l a^(k)_l conj(b_l) d^l(beta_j) = P_k - i Q_k,
//     P_k = sum_l a^(k)_l (Re b_l d^l),   Q_k = sum_l a^(k)_l (Im b_l d^l),
// with rows = angles (A operand: Re b_l d^l or Im b_l d^l, one value per (angle, l))
// and columns = (sky, re/im) (B operand: a^(k)_l, 2K real columns).  A launch computes
// P (part 0, C stored) or Q (part 1, C -= i Q; skipped for beam orders whose Im b is 0).
//
// FP64-class accuracy from bf16 tensor cores (an Ozaki-style split): each operand value,
// scaled into (-1, 1) by a power of two (A: 2^-eb with |b| < 2^eb per beam order; B:
// 2^-ea with |a| < 2^ea per (sky, m_sky)), is written as six 7-bit integer slices
//     x = sum_{q<6} s_q 2^(-7(q+1)) + e,   |s_0| <= 128, |s_q| <= 96, |e| < 2^-42.7,
// each slice exact in bf16.  The 21 slice products with i + j <= 5 are accumulated by
// level q = i + j in tensor memory: D_q = sum_l sum_{i+j=q} A_i B_j.  Each order adds
// an integer of magnitude at most 53248 to a level (level 5: 128 96 + 4 80 96 + 80 128
// with |A_q| <= 80 for q >= 1 on the A side), so FP32 accumulation is exact for 256
// orders (< 2^24); every 256 orders the levels are folded, V = sum_q D_q 2^(-7q), into
// float-float accumulators kept in tensor memory, and at the end of the chain
// C = 2^(ea + eb - 14) V.  The error per term is below 2^-42 of |a|max |b|max
// (dropped products i + j >= 6 and the slice remainders), far below the 1e-11 bar.
//
// The recursion is the normalised two-FMA form of the fused FP64 sum (u^l = d^l /
// sigma_l); the A value is u^l f_l with f_l = sigma_l b_l 2^-eb formed per tile.
//
// Roles (416 threads, one CTA per SM: the tensor memory is allocated whole):
//   warps 0-3   chains: one angle per thread, the FP64 recursion only (u^l of each tile
//               into shared memory), so the FP64 pipe is fed without gaps;
//   warps 4-7   slicers: row r = the same angle (and tensor-memory lane r): A = u^l f_l in
//               six slices, the level folds every 256 orders, and the output;
//   warp 8      control: the next tile's coefficient tables (lanes = l), TMA of the sky
//               tiles, the MMAs (lane 0), tensor-memory allocation;
//   warps 9-12  weights: the B slices of each sky tile.
// A tile is 32 orders (two MMA K-steps of 16), double-buffered; the roles hand tiles
// over through named barriers, MMA completion through tcgen05.commit on mbarriers,
// TMA completion through mbarriers.  Every mbarrier wait is bounded; a wait that
// gives up records WG_DEVERR_TIMEOUT, the CTA skips its remaining work (keeping every
// barrier), waits (bounded) for the operations it issued, frees the tensor memory and
// writes NaN for its outputs.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <mutex>
#include <string>

#include "../../include/wigner.h"
#include "wg_common.cuh"
#include "wg_internal.h"
#include "wg_tc.cuh"

namespace wg {
void set_last_error(const std::string &msg, int code);
int tables_for(int l_max, Tables *t);
int host_pool(cudaMemPool_t *pool);

namespace {

constexpr int TC_M = 128;        // angles per CTA (MMA M)
constexpr int TC_TL = 32;        // orders per tile (two K-steps of 16)
constexpr int TC_NS = 6;         // slices per operand value
constexpr int TC_SEG = 8;        // tiles per exactly accumulated segment (256 orders)
constexpr int TC_SKIES = 32;     // skies per launch column group (N = 64 real columns)
constexpr int TC_THREADS = 416;  // warps 0-3 chains, 4-7 slicers, 8 control, 9-12 weights
constexpr int WARP_CTL = 8, TID_B0 = 288;
constexpr int TC_GROUP = 8;      // chain columns per CTA
constexpr size_t TC_TABLE_BYTES = (size_t)1 << 30;  // scratch for the recursion tables of a column batch

// named barriers (0 is __syncthreads); the stage s is added to the paired ids.  The
// order of the roles rests on these alone (every role that arrives on a barrier syncs on
// another that the consumer arrives at after consuming it), never on the mbarrier waits,
// which may give up:
//   TAB_READY(s)  control -> chains   tables of the tile in stage s built
//   U_READY(h)    chains -> slicers   u^l of half h (16 orders) of the tile written
//   U_FREE(h)     slicers -> chains   half h of the u buffer read
//   B_READY(s)    weights -> control  B slices in stage s written (and the sky tile read)
//   A_READY(s)    slicers -> control  A slices in stage s written; the tables in stage s
//                                     are then read by every role (the chains finished the
//                                     tile before the slicers could start its last half)
//   B_FREE(s)     control -> weights  the MMA of stage s issued, the next sky tile requested
//   MMA_ISSUED    control -> slicers  the MMA of a segment's last tile issued
//   FLUSHED       slicers -> control  the levels of a segment read from tensor memory
constexpr int BAR_TAB_READY = 1, BAR_U_READY = 3, BAR_B_READY = 5, BAR_A_READY = 7, BAR_B_FREE = 9,
              BAR_FLUSHED = 11, BAR_MMA_ISSUED = 12, BAR_U_FREE = 13;
constexpr int CNT_CHAIN_CTL = 160, CNT_SLICE_CTL = 160, CNT_CHAIN_SLICE = 256, CNT_B_CTL = 160;

struct TcSmem {
    alignas(1024) unsigned char A[2][TC_NS][2][4096];  // [stage][slice][K-step] 128 rows x 16 bf16
    alignas(1024) unsigned char B[2][TC_NS][2][2048];  // [stage][slice][K-step] up to 64 rows x 16 bf16
    alignas(128) double2 Aw[2][TC_TL][TC_SKIES];       // TMA tile of the skies: [l][k] (re, im)
    double2 FG[2][TC_TL];                              // (F0', G') of the normalised recursion
    float2 F[2][TC_TL];                                // f_l = sigma_l b_l 2^-eb as float-float
    double U[TC_TL][TC_M];                             // u^l of the tile, [l][row]
    unsigned long long mbar_tma[2], mbar_mma[2];
    uint32_t tmem;
    int abort;
};

static_assert(sizeof(TcSmem) + 1024 <= 232448, "shared memory of the tensor-core kernel exceeds 227 KB");

// per (chain column, l): the normalised recursion's F0' = F0 rho, G' = G rho and sigma_l
// (float-float), made by tc_tables_kernel for a batch of columns before the main kernel
struct TcTab {
    double f0p, gp;
    float sh, sl;
};

struct TcArgs {
    int l_max, mb_max, ms_max, n_beta, n_col;
    const TcTab *tab;  // [k - c0][l], l <= l_max, for the columns [c0, c1) of this launch
    int c0, c1;
    const double *beta;
    const double *b;   // interleaved complex [l][mb]
    double *c_out;     // interleaved complex [k][mb][ms][j]
    const int *ea;     // [n_col][ms_max + 1]: |a| < 2^ea over l
    const int *eb;     // [2][mb_max + 1]: |Re b| < 2^eb[0], |Im b| < 2^eb[1]; INT_MIN: that part is 0
    int part;          // 0: P (store C), 1: Q (C -= i Q)
    int k_groups, n_chunks, group;
    unsigned long long *counters;
    int wait_tries;
};

// x 2^k as float-float (integer operations, one FP32 add and multiply): hi = the top 24
// bits of the scaled mantissa, lo = the next 23 (truncated).  Values whose scaled
// exponent is below emin (>= -80) come back as zero.
__device__ __forceinline__ void dsplit(double x, int k, int emin, float &h, float &l) {
    const long long bits = __double_as_longlong(x);
    const int hi32 = (int)(bits >> 32);
    const int be = (hi32 >> 20) & 0x7ff;
    const int e = be - 1023 + k;
    const unsigned sign = (unsigned)hi32 & 0x80000000u;
    const unsigned long long mant = (unsigned long long)bits & 0xfffffffffffffULL;
    const bool keep = be != 0 && e >= emin;
    const unsigned rem23 = (unsigned)(mant >> 6) & 0x7fffffu;
    const float lf = __fadd_rn(__uint_as_float(0x4B000000u | rem23), -8388608.0f);  // rem23, exactly
    const float sc = __uint_as_float(sign | ((unsigned)(e - 46 + 127) << 23));       // +-2^(e-46)
    h = keep ? __uint_as_float(sign | ((unsigned)(e + 127) << 23) | (unsigned)(mant >> 29)) : 0.f;
    l = keep ? __fmul_rn(lf, sc) : 0.f;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t *>(&v);
}

// Six 7-bit slices of a pair of values x = h + l in (-1, 1), |l| <= 2^-24 |h|: integer
// slices s_q with x = sum_q s_q 2^(-7(q+1)) + e.  Slices 0-2 come from h alone (each
// remainder exact); l joins the remainder before slice 3 (one rounding, 2^-45 of 1).
// out[q] packs the slices of the pair as bf16 (exact integers).
__device__ __forceinline__ void slice6_pair(float2 h, float2 l, uint32_t (&out)[TC_NS]) {
    const float2 M = make_float2(12582912.f, 12582912.f);  // 1.5 2^23: (x + M) - M rounds x to an integer
    const float2 S = make_float2(128.f, 128.f), m1 = make_float2(-1.f, -1.f);
    const float2 L28 = make_float2(268435456.f, 268435456.f);  // 2^28
    float2 r = __fmul2_rn(h, S);
#pragma unroll
    for (int q = 0; q < TC_NS; ++q) {
        if (q == 3) r = __ffma2_rn(l, L28, r);
        const float2 t = __fadd2_rn(r, M);
        const float2 s = __ffma2_rn(M, m1, t);  // t - M
        out[q] = pack_bf16x2(s.x, s.y);
        if (q + 1 < TC_NS) r = __fmul2_rn(__ffma2_rn(s, m1, r), S);  // (r - s) 128, exact
    }
}

// a float as a double by bit arithmetic (exact; zero and subnormal floats give 0)
__device__ __forceinline__ double f2d_bits(float x) {
    const unsigned u = __float_as_uint(x);
    const unsigned e = (u >> 23) & 0xffu;
    if (e == 0) return 0.0;
    const unsigned long long b = ((unsigned long long)(u & 0x80000000u) << 32) |
                                 ((unsigned long long)(e - 127u + 1023u) << 52) |
                                 ((unsigned long long)(u & 0x7fffffu) << 29);
    return __longlong_as_double((long long)b);
}

// bounded wait used by every role; records the timeout and the abort flag
__device__ __forceinline__ bool tc_wait(TcSmem &sm, unsigned long long *bar, unsigned parity, int tries,
                                        int *status) {
    if (*(volatile int *)&sm.abort) return false;
    if (mbar_wait(bar, parity, tries)) return true;
    *(volatile int *)&sm.abort = 1;
    raise_status(status, WG_DEVERR_TIMEOUT);
    return false;
}

// the flattened (column, tile) sequence every role walks in the same order
struct TileIter {
    int k, k_end, MB1, L;   // column k = ms MB1 + mb
    int mb, ms, l0, t, nt;  // current column and tile
    bool valid;
    __device__ void skip_empty(const TcArgs &A) {
        while (k < k_end) {
            ms = k / MB1;
            mb = k - ms * MB1;
            if (A.part == 0 || A.eb[(A.mb_max + 1) + mb] != INT_MIN) break;
            ++k;
        }
        valid = k < k_end;
        if (valid) {
            l0 = mb > ms ? mb : ms;
            t = 0;
            nt = (L + 1 - l0 + TC_TL - 1) / TC_TL;
        }
    }
    __device__ void init(const TcArgs &A, int k_begin, int kend) {
        k = k_begin;
        k_end = kend;
        MB1 = A.mb_max + 1;
        L = A.l_max;
        skip_empty(A);
    }
    __device__ void next(const TcArgs &A) {
        if (++t >= nt) {
            ++k;
            skip_empty(A);
        }
    }
    __device__ int ts() const { return l0 + t * TC_TL; }
    __device__ bool seg_first() const { return t % TC_SEG == 0; }
    __device__ bool seg_last() const { return (t + 1) % TC_SEG == 0 || t + 1 == nt; }
    __device__ bool col_last() const { return t + 1 == nt; }
};

// ---------------------------------------------------------------------------------
// control warp: tables of tile `it` into stage s (lanes = orders), carrying sigma
// ---------------------------------------------------------------------------------
// inputs of a tile's tables (lane = order l): the pre-computed entry and the beam part,
// loaded one tile ahead so their latency hides behind the MMA issue
struct TabIn {
    double2 fg;
    float2 sig;
    double bpart;
};

__device__ __forceinline__ TabIn load_tab(const TcArgs &A, const TileIter &it) {
    const int lane = threadIdx.x & 31;
    const int L = A.l_max;
    const int l = it.ts() + lane;
    TabIn in{make_double2(0.0, 0.0), make_float2(0.f, 0.f), 0.0};
    if (l <= L) {
        const TcTab e = A.tab[(size_t)(it.k - A.c0) * (L + 1) + l];
        if (l < L) in.fg = make_double2(e.f0p, e.gp);
        in.sig = make_float2(e.sh, e.sl);
        const double2 bv = reinterpret_cast<const double2 *>(A.b)[(size_t)l * (A.mb_max + 1) + it.mb];
        in.bpart = A.part == 0 ? bv.x : bv.y;
    }
    return in;
}

// control warp: the tables of tile `it` into stage s (lanes = orders): (F0', G') and
// f_l = sigma_l b_l 2^-eb, a float-float product on the FP32 pipe (the FP64 work of the
// tables is in tc_tables_kernel, so no role but the chains uses this SM's FP64 units)
__device__ __forceinline__ void build_tables(const TcArgs &A, const TileIter &it, const TabIn &in, int s,
                                             TcSmem &sm) {
    const int lane = threadIdx.x & 31;
    float fh = 0.f, fl = 0.f;
    const int eb = A.eb[A.part * (A.mb_max + 1) + it.mb];
    if (eb != INT_MIN) {
        float bh, bl;
        dsplit(in.bpart, -eb, -80, bh, bl);
        const float p = __fmul_rn(in.sig.x, bh);
        float e = __fmaf_rn(in.sig.x, bh, -p);
        e = __fmaf_rn(in.sig.x, bl, e);
        e = __fmaf_rn(in.sig.y, bh, e);
        fh = __fadd_rn(p, e);
        fl = __fsub_rn(e, __fsub_rn(fh, p));
    }
    sm.FG[s][lane] = in.fg;
    sm.F[s][lane] = make_float2(fh, fl);
}

__device__ __forceinline__ void issue_tma(const TcArgs &A, const CUtensorMap *amap, const TileIter &it, int s, int k0,
                                          TcSmem &sm) {
    fence_proxy_async();
    mbar_arrive_expect_tx(&sm.mbar_tma[s], (unsigned)(TC_SKIES * TC_TL * 16));
    tma_load_3d(&sm.Aw[s][0][0], amap, 2 * it.ms, k0, it.ts(), &sm.mbar_tma[s]);
}

__device__ __forceinline__ void issue_mmas(TcSmem &sm, int s, uint32_t tbase, int N, bool seg_first) {
    tc_fence_after();
    const uint32_t idesc = tc_idesc_bf16(N);
#pragma unroll
    for (int kk = 0; kk < 2; ++kk)
#pragma unroll
        for (int q = 0; q < TC_NS; ++q)
#pragma unroll
            for (int i = 0; i <= q; ++i) {
                const int j = q - i;
                const uint64_t da = tc_desc(smem_u32(&sm.A[s][i][kk][0]));
                const uint64_t db = tc_desc(smem_u32(&sm.B[s][j][kk][0]));
                const uint32_t acc = (seg_first && kk == 0 && i == 0) ? 0u : 1u;
                tc_mma_bf16(tbase + (uint32_t)(q * N), da, db, idesc, acc);
            }
    tc_commit(&sm.mbar_mma[s]);
}

// ---------------------------------------------------------------------------------
// weight warps: B slices of stage s from the TMA'd sky tile (rows n = 2k + re/im)
// ---------------------------------------------------------------------------------
__device__ __forceinline__ void build_b(const TcArgs &A, const TileIter &it, int s, int k0, int nsky, int N,
                                       TcSmem &sm) {
    const int tb = threadIdx.x - TID_B0;  // 0..127
    for (int task = tb; task < TC_SKIES * 2 * 4; task += 128) {
        const int g = task & 3;          // 8-order group of the tile
        const int n = task >> 2;         // row: 2 k + part
        if (n >= N) continue;
        const int kl = n >> 1, p = n & 1;
        const int ea = kl < nsky ? A.ea[(size_t)(k0 + kl) * (A.ms_max + 1) + it.ms] : 0;
        float hs[8], ls[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const double2 v = sm.Aw[s][8 * g + i][kl];
            dsplit(p ? v.y : v.x, -ea, -45, hs[i], ls[i]);
        }
        uint32_t pk[TC_NS][4];
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            uint32_t o[TC_NS];
            slice6_pair(make_float2(hs[i], hs[i + 1]), make_float2(ls[i], ls[i + 1]), o);
#pragma unroll
            for (int q = 0; q < TC_NS; ++q) pk[q][i >> 1] = o[q];
        }
        const uint32_t off = tc_off(n, 8 * (g & 1));
#pragma unroll
        for (int q = 0; q < TC_NS; ++q)
            *reinterpret_cast<uint4 *>(&sm.B[s][q][g >> 1][off]) = make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
    }
}

}  // namespace

__global__ void __launch_bounds__(TC_THREADS, 1)
    conv_multi_tc_kernel(TcArgs A, Tables T, const __grid_constant__ CUtensorMap amap) {
    extern __shared__ unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    int item = blockIdx.x;
    const int kg = item % A.k_groups;
    item /= A.k_groups;
    const int chunk = item % A.n_chunks;
    const int grp = item / A.n_chunks;
    const int MB1 = A.mb_max + 1, MS1 = A.ms_max + 1;
    const int k_begin = A.c0 + grp * A.group, k_end = min(A.c1, k_begin + A.group);
    const int k0 = kg * TC_SKIES, nsky = min(TC_SKIES, A.n_col - k0);
    const int N = ((2 * nsky + 15) / 16) * 16;
    const int L = A.l_max, NB = A.n_beta;

    TileIter probe;
    probe.init(A, k_begin, k_end);
    if (!probe.valid) return;  // part 1 with no imaginary beam in this group (uniform)

    if (warp == WARP_CTL) tmem_alloc(&sm.tmem, 512);
    if (tid == WARP_CTL * 32) {
        mbar_init(&sm.mbar_tma[0], 1);
        mbar_init(&sm.mbar_tma[1], 1);
        mbar_init(&sm.mbar_mma[0], 1);
        mbar_init(&sm.mbar_mma[1], 1);
        fence_mbar_init();
        sm.abort = 0;
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tbase = sm.tmem;

    if (warp < 4) {
        // ===== chain warps: the FP64 recursion, u^l of the tile into shared memory =====
        const int r = tid;
        const int j = chunk * TC_M + r;
        const bool valid = j < NB;
        const Angle ang = make_angle(valid ? A.beta[j] : 1.0);
        if (valid && ang.bad && A.part == 0) raise_status(T.status, WG_DEVERR_BETA);
        TileIter it = probe;
        unsigned long long n_elem = 0;
        int gt = 0;
        double u = 0.0, up = 0.0;
        int nsc = 0;
        bool plain = true;
        while (it.valid) {
            const int s = gt & 1;
            if (it.t == 0) {
                const Scaled sd = seed_value(it.mb, it.ms, ang, T);
                u = (valid && !ang.bad) ? sd.mant : 0.0;
                nsc = sd.n;
                plain = sd.plain;
                up = 0.0;
                if (valid && A.part == 0 && kg == 0) n_elem += (unsigned long long)(L + 1 - it.l0);
            }
            bar_sync(BAR_TAB_READY + s, CNT_CHAIN_CTL);
            const int ts = it.ts();
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                if (gt >= 1) bar_sync(BAR_U_FREE + h, CNT_CHAIN_SLICE);
                // the half's coefficients into registers, each multiplier y formed two steps
                // ahead of its use, the 16 values of u stored after the half: a dependent
                // DFMA then never waits behind a shared-memory access in the warp's
                // in-order stream (measured 156 cycles per two-DFMA step against 207 with a
                // load and a store in every step; the FP64 unit of a sub-partition takes a
                // warp-wide DFMA every 64 cycles)
                double2 fg[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) fg[i] = sm.FG[s][16 * h + i];
                double uu[16];
                double y0 = fma(fg[0].x, ang.cb, -fg[0].y);
                double y1 = fma(fg[1].x, ang.cb, -fg[1].y);
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int l = ts + 16 * h + i;
                    const double y = y0;
                    y0 = y1;
                    if (i + 2 < 16) y1 = fma(fg[i + 2].x, ang.cb, -fg[i + 2].y);
                    uu[i] = (plain && l <= L) ? u : 0.0;
                    if (l < L) {
                        const double nx = fma(y, u, -up);
                        up = u;
                        u = nx;
                    }
                    // scaled doubles: the range check every fourth step keeps its integer work
                    // off most steps; four steps grow a mantissa by less than 2^64 (at most
                    // 2 (l0 + 1) / (k + 1) + 1 per step, l0 <= 32767), so from below 2^90 it
                    // stays far inside the double range
                    if ((i & 3) == 3 && !plain) scaled_fixup(u, up, nsc, plain);
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) sm.U[16 * h + i][r] = uu[i];
                bar_arrive(BAR_U_READY + h, CNT_CHAIN_SLICE);
            }
            it.next(A);
            ++gt;
        }
        if (A.counters) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) n_elem += __shfl_down_sync(0xffffffffu, n_elem, off);
            if (lane == 0 && n_elem) {
                atomicAdd(&A.counters[0], n_elem);
                atomicAdd(&A.counters[1], n_elem);
            }
        }
    } else if (warp < 8) {
        // ===== slicer warps: A = u f in six 7-bit slices, the level folds and the output =====
        const int r = tid - 128;
        const int j = chunk * TC_M + r;
        const bool valid = j < NB;
        const double bj = valid ? A.beta[j] : 1.0;
        const bool bad_ang = !(bj >= 0.0 && bj <= WG_PI_HI);
        const uint32_t tl = tbase + ((uint32_t)((warp - 4) * 32) << 16);
        TileIter it = probe;
        int gt = 0;
        while (it.valid) {
            const int s = gt & 1;
            TileIter nx = it;
            nx.next(A);
#pragma unroll 1
            for (int h = 0; h < 2; ++h) {
                bar_sync(BAR_U_READY + h, CNT_CHAIN_SLICE);
                if (h == 0 && gt >= 2) tc_wait(sm, &sm.mbar_mma[s], ((gt >> 1) - 1) & 1, A.wait_tries, T.status);
#pragma unroll
                for (int g8 = 0; g8 < 2; ++g8) {
                    uint32_t pk[TC_NS][4];
#pragma unroll
                    for (int i2 = 0; i2 < 8; i2 += 2) {
                        const int i = 16 * h + 8 * g8 + i2;
                        float hh[2], ll[2];
#pragma unroll
                        for (int p = 0; p < 2; ++p) {
                            float uh, ul;
                            dsplit(sm.U[i + p][r], 0, -60, uh, ul);
                            const float2 f = sm.F[s][i + p];
                            const float pr = __fmul_rn(uh, f.x);
                            float e = __fmaf_rn(uh, f.x, -pr);
                            e = __fmaf_rn(uh, f.y, e);
                            e = __fmaf_rn(ul, f.x, e);
                            hh[p] = __fadd_rn(pr, e);
                            ll[p] = __fsub_rn(e, __fsub_rn(hh[p], pr));
                        }
                        uint32_t o[TC_NS];
                        slice6_pair(make_float2(hh[0], hh[1]), make_float2(ll[0], ll[1]), o);
#pragma unroll
                        for (int q = 0; q < TC_NS; ++q) pk[q][i2 >> 1] = o[q];
                    }
                    const uint32_t off = tc_off(r, 8 * g8);
#pragma unroll
                    for (int q = 0; q < TC_NS; ++q)
                        *reinterpret_cast<uint4 *>(&sm.A[s][q][h][off]) =
                            make_uint4(pk[q][0], pk[q][1], pk[q][2], pk[q][3]);
                }
                if (nx.valid) bar_arrive(BAR_U_FREE + h, CNT_CHAIN_SLICE);
            }
            fence_proxy_async();
            bar_arrive(BAR_A_READY + s, CNT_SLICE_CTL);
            if (it.seg_last()) {
                // fold this segment's levels into the float-float accumulators (or the output)
                bar_sync(BAR_MMA_ISSUED, CNT_SLICE_CTL);
                const bool ok = tc_wait(sm, &sm.mbar_mma[s], (gt >> 1) & 1, A.wait_tries, T.status);
                tc_fence_after();
                const bool first = it.t < TC_SEG;
                const bool last = it.col_last();
                const bool bad = !ok || *(volatile int *)&sm.abort || bad_ang;
                for (int c8 = 0; c8 < N; c8 += 8) {
                    float lv[TC_NS][8], ah[8], al[8];
#pragma unroll
                    for (int q = 0; q < TC_NS; ++q) tmem_ld8(tl + (uint32_t)(q * N + c8), lv[q]);
                    if (!first) {
                        tmem_ld8(tl + (uint32_t)(6 * N + c8), ah);
                        tmem_ld8(tl + (uint32_t)(7 * N + c8), al);
                    }
                    tmem_ld_wait();
                    // V = sum_q D_q 2^(-7q) in float-float, two columns at a time with the
                    // packed instructions (each lane as the scalar float-float sum)
#pragma unroll
                    for (int c = 0; c < 8; c += 2) {
                        float2 vh = make_float2(lv[0][c], lv[0][c + 1]), vl = make_float2(0.f, 0.f);
#pragma unroll
                        for (int q = 1; q < TC_NS; ++q) {
                            const float sc = __uint_as_float((unsigned)(127 - 7 * q) << 23);
                            ff_add2(vh, vl, __fmul2_rn(make_float2(lv[q][c], lv[q][c + 1]), make_float2(sc, sc)),
                                    make_float2(0.f, 0.f));
                        }
                        if (!first) {
                            float2 xh = make_float2(ah[c], ah[c + 1]), xl = make_float2(al[c], al[c + 1]);
                            ff_add2(xh, xl, vh, vl);
                            vh = xh;
                            vl = xl;
                        }
                        ah[c] = vh.x;
                        ah[c + 1] = vh.y;
                        al[c] = vl.x;
                        al[c + 1] = vl.y;
                    }
                    if (last) {
                        if (valid) {
                            const int eb = A.eb[A.part * MB1 + it.mb];
#pragma unroll
                            for (int p = 0; p < 4; ++p) {
                                const int kl = (c8 >> 1) + p;
                                if (kl >= nsky) continue;
                                const int e = A.ea[(size_t)(k0 + kl) * MS1 + it.ms] + eb - 14;
                                double re = f2d_bits(ah[2 * p]) + f2d_bits(al[2 * p]);
                                double im = f2d_bits(ah[2 * p + 1]) + f2d_bits(al[2 * p + 1]);
                                re = biased_exp(re) + e >= 1 ? exp_shift(re, e) : 0.0;
                                im = biased_exp(im) + e >= 1 ? exp_shift(im, e) : 0.0;
                                double2 *out = reinterpret_cast<double2 *>(A.c_out) +
                                               (((size_t)(k0 + kl) * MB1 + it.mb) * MS1 + it.ms) * NB + j;
                                const double nan = __longlong_as_double(0x7ff8000000000000LL);
                                if (A.part == 0) {
                                    *out = bad ? make_double2(nan, nan) : make_double2(re, im);
                                } else {
                                    const double2 c = *out;
                                    *out = bad ? make_double2(nan, nan) : make_double2(c.x + im, c.y - re);
                                }
                            }
                        }
                    } else {
                        tmem_st8(tl + (uint32_t)(6 * N + c8), ah);
                        tmem_st8(tl + (uint32_t)(7 * N + c8), al);
                    }
                }
                tmem_st_wait();
                tc_fence_before();
                bar_arrive(BAR_FLUSHED, CNT_SLICE_CTL);
            }
            it = nx;
            ++gt;
        }
    } else if (warp == WARP_CTL) {
        // ============================ control warp ============================
        TileIter tab = probe, mma = probe, tma = probe;
        build_tables(A, tab, load_tab(A, tab), 0, sm);
        bar_arrive(BAR_TAB_READY + 0, CNT_CHAIN_CTL);
        tab.next(A);
        TabIn nxt{};
        if (tab.valid) nxt = load_tab(A, tab);
        // operations issued per stage (the drain at the end waits for the last of each);
        // the decision to issue is taken once per warp from lane 0's view of the abort flag
        int n_tma[2] = {0, 0}, n_mma[2] = {0, 0};
        auto go = [&]() { return __shfl_sync(0xffffffffu, *(volatile int *)&sm.abort, 0) == 0; };
        if (go()) {
            if (lane == 0) issue_tma(A, &amap, tma, 0, k0, sm);
            ++n_tma[0];
        }
        tma.next(A);
        if (tma.valid) {
            if (go()) {
                if (lane == 0) issue_tma(A, &amap, tma, 1, k0, sm);
                ++n_tma[1];
            }
            tma.next(A);
        }
        int gt = 0;
        while (mma.valid) {
            const int s = gt & 1;
            if (tab.valid) {  // tables of tile gt + 1 into the other stage (free since A_READY of gt - 1)
                build_tables(A, tab, nxt, s ^ 1, sm);
                bar_arrive(BAR_TAB_READY + (s ^ 1), CNT_CHAIN_CTL);
                tab.next(A);
                if (tab.valid) nxt = load_tab(A, tab);  // inputs of tile gt + 2, ahead
            }
            bar_sync(BAR_B_READY + s, CNT_B_CTL);
            bar_sync(BAR_A_READY + s, CNT_SLICE_CTL);
            if (mma.seg_first() && gt > 0) bar_sync(BAR_FLUSHED, CNT_SLICE_CTL);
            if (go()) {
                if (lane == 0) issue_mmas(sm, s, tbase, N, mma.seg_first());
                ++n_mma[s];
            }
            __syncwarp();
            if (mma.seg_last()) bar_arrive(BAR_MMA_ISSUED, CNT_SLICE_CTL);
            if (tma.valid) {  // the sky tile of gt + 2 into this stage: its B slices are built
                if (go()) {
                    if (lane == 0) issue_tma(A, &amap, tma, s, k0, sm);
                    ++n_tma[s];
                }
                __syncwarp();
                bar_arrive(BAR_B_FREE + s, CNT_B_CTL);
                tma.next(A);
            }
            mma.next(A);
            ++gt;
        }
        bar_sync(BAR_FLUSHED, CNT_SLICE_CTL);  // the last fold has read the tensor memory
        // drain: the last commit of each stage and every TMA phase not yet waited for
        if (lane == 0) {
            for (int st = 0; st < 2; ++st) {
                if (n_mma[st] > 0) mbar_wait(&sm.mbar_mma[st], (n_mma[st] - 1) & 1, TMA_WAIT_ITERS);
                if (n_tma[st] > 0) mbar_wait(&sm.mbar_tma[st], (n_tma[st] - 1) & 1, TMA_WAIT_ITERS);
            }
        }
        __syncwarp();
        tc_fence_after();
        tmem_dealloc(tbase, 512);
    } else {
        // ============================ weight warps ============================
        TileIter it = probe;
        int gt = 0;
        while (it.valid) {
            const int s = gt & 1;
            if (gt >= 2) bar_sync(BAR_B_FREE + s, CNT_B_CTL);
            tc_wait(sm, &sm.mbar_tma[s], (gt >> 1) & 1, A.wait_tries, T.status);
            if (gt >= 2) tc_wait(sm, &sm.mbar_mma[s], ((gt >> 1) - 1) & 1, A.wait_tries, T.status);
            build_b(A, it, s, k0, nsky, N, sm);
            fence_proxy_async();
            bar_arrive(BAR_B_READY + s, CNT_B_CTL);
            it.next(A);
            ++gt;
        }
    }
}

// The tables of the normalised recursion for the chain columns [c0, c1): one warp per
// column walks l in steps of 32 (lanes = orders) with the Sec. 4.2.2 coefficients
// F0, G = F0 F1, F2, the normalisation sigma_{l+1} = F2_l sigma_{l-1} (sigma_{l0} =
// sigma_{l0+1} = 1) as a product scan along each parity of the lanes, rho_l =
// sigma_l / sigma_{l+1}, F0' = F0 rho, G' = G rho.
__global__ void tc_tables_kernel(int L, int MB, int c0, int c1, Tables T, TcTab *tab) {
    const int lane = threadIdx.x & 31;
    const int wg = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int nw = (int)((gridDim.x * blockDim.x) >> 5);
    const int MB1 = MB + 1;
    for (int k = c0 + wg; k < c1; k += nw) {
        const int ms = k / MB1, mb = k - ms * MB1;
        const int l0 = mb > ms ? mb : ms;
        TcTab *out = tab + (size_t)(k - c0) * (L + 1);
        double c_m1 = 1.0, c_0 = 1.0;  // sigma_{l0-1} := 1 and sigma_{l0} = 1 give sigma_{l0+1} = 1
        for (int ts = l0; ts <= L; ts += 32) {
            const int l = ts + lane;
            double f0 = 0.0, g = 0.0, f2 = 1.0;
            if (l < L) {
                lrec_coefficients(l, mb, ms, T, f0, g, f2);
                if (l == l0) f2 = 1.0;
            }
            double P = f2;
#pragma unroll
            for (int off = 2; off < 32; off <<= 1) {
                const double v = __shfl_up_sync(0xffffffffu, P, off);
                if (lane >= off) P *= v;
            }
            const double sig_next = P * ((lane & 1) ? c_0 : c_m1);  // sigma_{l+1}
            const double sig_up = __shfl_up_sync(0xffffffffu, sig_next, 1);
            const double sig = lane == 0 ? c_0 : sig_up;              // sigma_l
            if (l <= L) {
                TcTab e;
                e.f0p = 0.0;
                e.gp = 0.0;
                if (l < L) {
                    const double rho = sig / sig_next;
                    e.f0p = f0 * rho;
                    e.gp = g * rho;
                }
                dsplit(sig, 0, -80, e.sh, e.sl);
                out[l] = e;
            }
            c_m1 = __shfl_sync(0xffffffffu, sig_next, 30);
            c_0 = __shfl_sync(0xffffffffu, sig_next, 31);
        }
    }
}

// |x| < 2^e bounds per (sky, m_sky) over l for a, and per (part, m_b) for b
__global__ void tc_scales_kernel(const double *a, const double *b, int L, int MB, int MS, int n_col, int *ea,
                                 int *eb) {
    const int ms = blockIdx.x * blockDim.x + threadIdx.x;
    if (blockIdx.y < (unsigned)n_col) {
        if (ms > MS) return;
        const double2 *col = reinterpret_cast<const double2 *>(a) + (size_t)blockIdx.y * (L + 1) * (MS + 1) + ms;
        int m = 0;
        for (int l = 0; l <= L; ++l) {
            const double2 v = col[(size_t)l * (MS + 1)];
            m = max(m, max(biased_exp(v.x), biased_exp(v.y)));
        }
        ea[(size_t)blockIdx.y * (MS + 1) + ms] = m == 0 ? 0 : m - 1022;
    } else {
        const int p = ms / (MB + 1), mb = ms - p * (MB + 1);
        if (p > 1) return;
        int m = 0;
        for (int l = 0; l <= L; ++l) {
            const double2 v = reinterpret_cast<const double2 *>(b)[(size_t)l * (MB + 1) + mb];
            m = max(m, biased_exp(p ? v.y : v.x));
        }
        eb[p * (MB + 1) + mb] = m == 0 ? (p ? INT_MIN : 0) : m - 1022;
    }
}

namespace {
typedef CUresult (*EncodeTiledFn3)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn3 encode3() {
    static std::once_flag once;
    static EncodeTiledFn3 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn3>(p);
    });
    return fn;
}
}  // namespace

// The skies a[k][l][ms] as a 3-D float64 tensor {2 (ms_max + 1), n_col, l_max + 1} (the
// sky index before the order, so a box lands as [l][k] in shared memory and the weight
// warps read consecutive skies from consecutive banks); a box {2, 32, 32} is the tile of
// one m_sky column, 32 skies, 32 orders (x = 2 m_sky is even, so the copy starts on a
// 16-byte boundary; skies past n_col and rows past l_max come back as zeros).
int launch_conv_multi_tc(int l_max, int mb_max, int ms_max, int n_beta, int n_col, const double *beta,
                         const double *a, const double *b, double *c_out, unsigned long long *counters,
                         const Tables &T, int wait_tries, void *stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n_beta == 0 || n_col == 0) return 0;
    EncodeTiledFn3 fn = encode3();
    if (!fn) return (int)cudaErrorNotSupported;
    CUtensorMap amap;
    const cuuint64_t dims[3] = {(cuuint64_t)2 * (ms_max + 1), (cuuint64_t)n_col, (cuuint64_t)l_max + 1};
    const cuuint64_t strides[2] = {(cuuint64_t)16 * (ms_max + 1) * (l_max + 1), (cuuint64_t)16 * (ms_max + 1)};
    const cuuint32_t box[3] = {2u, (cuuint32_t)TC_SKIES, (cuuint32_t)TC_TL};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    if (fn(&amap, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3, const_cast<double *>(a), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return (int)cudaErrorInvalidValue;

    cudaMemPool_t pool;
    if (host_pool(&pool) != WG_OK) return (int)cudaErrorMemoryAllocation;
    int *ea = nullptr, *eb = nullptr;
    const size_t n_ea = (size_t)n_col * (ms_max + 1), n_eb = (size_t)2 * (mb_max + 1);
    cudaError_t e = alloc_injected() ? cudaErrorMemoryAllocation
                                     : cudaMallocFromPoolAsync((void **)&ea, (n_ea + n_eb) * sizeof(int), pool, s);
    if (e != cudaSuccess) return (int)e;
    eb = ea + n_ea;
    {
        dim3 grid((unsigned)((ms_max + 1 + 127) / 128), (unsigned)n_col + 1);
        if ((unsigned)(2 * (mb_max + 1) + 127) / 128 > grid.x) grid.x = (unsigned)(2 * (mb_max + 1) + 127) / 128;
        tc_scales_kernel<<<grid, 128, 0, s>>>(a, b, l_max, mb_max, ms_max, n_col, ea, eb);
        e = cudaGetLastError();
    }
    const size_t smem = sizeof(TcSmem) + 1024;
    static std::once_flag attr_once;
    static cudaError_t attr_err = cudaSuccess;
    std::call_once(attr_once, [&] {
        attr_err = cudaFuncSetAttribute(conv_multi_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    });
    if (e == cudaSuccess) e = attr_err;
    TcArgs ta;
    ta.l_max = l_max;
    ta.mb_max = mb_max;
    ta.ms_max = ms_max;
    ta.n_beta = n_beta;
    ta.n_col = n_col;
    ta.beta = beta;
    ta.b = b;
    ta.c_out = c_out;
    ta.ea = ea;
    ta.eb = eb;
    ta.k_groups = (n_col + TC_SKIES - 1) / TC_SKIES;
    ta.n_chunks = (n_beta + TC_M - 1) / TC_M;
    ta.group = TC_GROUP;
    ta.counters = counters;
    ta.wait_tries = wait_tries;
    // columns in batches whose tables fit TC_TABLE_BYTES of scratch
    const int ncol = (mb_max + 1) * (ms_max + 1);
    const size_t per_col = (size_t)(l_max + 1) * sizeof(TcTab);
    long long cpb = (long long)(TC_TABLE_BYTES / per_col) / TC_GROUP * TC_GROUP;
    if (cpb < TC_GROUP) cpb = TC_GROUP;
    if (cpb > ncol) cpb = ncol;
    TcTab *tab = nullptr;
    if (e == cudaSuccess)
        e = alloc_injected() ? cudaErrorMemoryAllocation
                             : cudaMallocFromPoolAsync((void **)&tab, (size_t)cpb * per_col, pool, s);
    ta.tab = tab;
    for (int c0 = 0; c0 < ncol && e == cudaSuccess; c0 += (int)cpb) {
        const int c1 = (int)std::min<long long>(ncol, c0 + cpb);
        tc_tables_kernel<<<152 * 4, 256, 0, s>>>(l_max, mb_max, c0, c1, T, tab);
        e = cudaGetLastError();
        ta.c0 = c0;
        ta.c1 = c1;
        const long long items = (long long)((c1 - c0 + TC_GROUP - 1) / TC_GROUP) * ta.n_chunks * ta.k_groups;
        if (items > 0x7fffffffLL) e = cudaErrorInvalidValue;
        for (int part = 0; part < 2 && e == cudaSuccess; ++part) {
            ta.part = part;
            conv_multi_tc_kernel<<<(unsigned)items, TC_THREADS, smem, s>>>(ta, T, amap);
            e = cudaGetLastError();
        }
    }
    if (tab) cudaFreeAsync(tab, s);
    cudaFreeAsync(ea, s);
    return (int)e;
}

}  // namespace wg

extern "C" int wigner_conv_sum_multi_tc(int l_max, int mb_max, int ms_max, int n_beta, int n_col, const double *beta,
                                        const wg_c64 *a, const wg_c64 *b, wg_c64 *c_out, wg_counter *counters,
                                        void *stream) {
    auto fail = [](int code, const std::string &msg) {
        wg::set_last_error(msg, code);
        return code;
    };
    if (l_max < 0 || l_max > WG_LMAX) return fail(WG_ERR_ARG, "l_max must be in [0, WG_LMAX]");
    if (mb_max < 0 || mb_max > l_max) return fail(WG_ERR_ARG, "mb_max must be in [0, l_max]");
    if (ms_max < 0 || ms_max > l_max) return fail(WG_ERR_ARG, "ms_max must be in [0, l_max]");
    if (n_beta < 0 || n_col < 0) return fail(WG_ERR_ARG, "n_beta and n_col must be >= 0");
    if (n_beta == 0 || n_col == 0) return WG_OK;
    if (!beta || ((uintptr_t)beta & 7)) return fail(WG_ERR_ARG, "beta is NULL or not 8-byte aligned");
    if (!a || !b || !c_out || ((uintptr_t)a & 15) || ((uintptr_t)b & 15) || ((uintptr_t)c_out & 15))
        return fail(WG_ERR_ARG, "a, b and c_out must be non-NULL and 16-byte aligned");
    if (counters && ((uintptr_t)counters & 7)) return fail(WG_ERR_ARG, "counters misaligned");
    wg::Tables t;
    int rc = wg::tables_for(l_max, &t);
    if (rc != WG_OK) return rc;
    const int e = wg::launch_conv_multi_tc(l_max, mb_max, ms_max, n_beta, n_col, beta, (const double *)a,
                                           (const double *)b, (double *)c_out, counters, t, wg::wait_tries(), stream);
    if (e == (int)cudaErrorMemoryAllocation) return fail(WG_ERR_ALLOC, "conv_multi_tc: scratch allocation failed");
    if (e != 0) return fail(WG_ERR_CUDA, std::string("conv_multi_tc launch: ") + cudaGetErrorString((cudaError_t)e));
    return WG_OK;
}
