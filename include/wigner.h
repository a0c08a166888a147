/*
 * wigner.h -- C ABI of the GB300 (sm_103a) library for reduced Wigner matrices
 * d^l_{m_b m_sky}(beta) and the beam-convolution l-sum of Prezeau & Reinecke,
 * "Algorithm for the evaluation of reduced Wigner matrices".
 *
 * What is computed
 *   d^l_{m m'}(beta) = <l m| exp(-i beta J_y) |l m'>            (Sec. 2, Eq. reducedwignerdef)
 *   by the stable l-recursion (Sec. 2, Eq. lrec; Sec. 4.2.2 table form)
 *       d^{l+1} = F0_l (cos beta - F1_l) d^l - F2_l d^{l-1}
 *   started at l0 = max(m_b, m_sky) from the log-space seeds of Eqs. ini1-ini2 and
 *   logstart (Sec. 3.2), carried in scaled doubles v = d * 2^(90 n) until the value
 *   reaches 2^-900 and in plain doubles after that (Sec. 3.2); and the l-sum
 *       C_{m_b m_sky}(beta) = sum_{l=l0}^{l_max} conj(b_{l m_b}) a_{l m_sky} d^l_{m_b m_sky}(beta)
 *   of Sec. 4.1, Eq. convdef, fused with the recursion so the d-table is never stored.
 *   Terms are summed from the first l at which |d| >= 1e-30 (Sec. 4.2.1); smaller
 *   terms change C by less than 1e-30 * sum |w|.
 *
 * Conventions (all calls)
 *   - Orders: 0 <= m_b <= mb_max <= l_max, 0 <= m_sky <= ms_max <= l_max; l_max <= WG_LMAX.
 *     Only non-negative orders are computed, except by wigner_conv_sum_full (every sky
 *     order) and wigner_d_matrix (every m').
 *   - Angles: beta[j] in [0, pi], float64, device memory, n_beta >= 0 entries.
 *     beta = 0 and beta = pi are exact: d(0) = delta_{m m'}, d(pi) = (-1)^(l-m') delta_{m,-m'}.
 *     An angle outside [0, pi] (or NaN) makes the affected outputs NaN and records
 *     WG_ERR_ARG in the device status word (see wigner_device_status); the call
 *     itself cannot see device data and returns WG_OK.
 *   - Complex numbers are wg_c64 {re, im}, layout-compatible with complex128 /
 *     torch.complex128.  All arrays are dense, row-major, C-contiguous.
 *   - Every pointer argument is a DEVICE pointer on the current CUDA device unless
 *     noted; the caller owns every buffer it passes.  The library owns only its
 *     per-device constant tables (ln n!, square-root tables) and a status word,
 *     created on the first call on a device (this first call allocates and
 *     copies, so make it before any stream capture).
 *   - Execution is asynchronous and stream-ordered on `stream` (a cudaStream_t;
 *     NULL = legacy default stream).  Calls never throw; they return WG_OK (0) or
 *     a negative WG_ERR_* code after validating their arguments on the host.
 *   - Precision forms: WG_FP64 runs everything in IEEE double.  WG_FP64S ("split
 *     pipe") runs the recursion in IEEE double with two FMAs per step (the chain is
 *     carried normalised by a product of the F2 coefficients) and the weighted sum in
 *     float-float (~48-bit) arithmetic on the FP32 pipe; its C agrees with WG_FP64 to
 *     ~1e-13 (fused sums only; the d-table and adjoints treat it as WG_FP64).
 *     WG_FP32X runs the recursion body in float with an int32 exponent carry: away
 *     from the poles (sin beta >= max(0.1, 1.2e-5 l_max)) the chain normalised by a
 *     product of the F2 coefficients (two FMAs per step), near the poles a difference
 *     form of the recursion that keeps float accuracy there; seeds and coefficients in
 *     float-float, compensated float sums.  Its error is stated per workload (relative
 *     L2 ~4e-6 on C at l_max = 8192; tests bind 2e-4 on d and 1e-4 on C).
 *   - No kernel waits on another CTA or a flag.  The FP64 fused sums stage their
 *     weights by TMA and wait on an mbarrier with a bounded number of tries; a wait
 *     that gives up records WG_ERR_TIMEOUT in the device status word.
 */
#ifndef WIGNER_GB300_H
#define WIGNER_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define WG_LMAX 32767 /* largest supported l_max */

typedef struct {
    double re, im;
} wg_c64;

typedef enum { WG_FP64 = 0, WG_FP32X = 1, WG_FP64S = 2 } wg_form;

enum {
    WG_OK = 0,
    WG_ERR_ARG = -1,         /* invalid argument (sizes, orders, null or misaligned pointer) */
    WG_ERR_CUDA = -2,        /* a CUDA runtime call failed (message in wigner_last_error_message) */
    WG_ERR_ALLOC = -3,       /* device allocation of the library's tables failed */
    WG_ERR_TIMEOUT = -4,     /* a bounded device-side wait gave up (reported by wigner_device_status) */
    WG_ERR_DEVICE = -5,      /* no usable sm_103 device / kernel image */
    WG_ERR_UNSUPPORTED = -6  /* valid request this library version does not implement */
};

/* Optional counters filled by some calls (device pointer, may be NULL):
 *   [0] elements  -- (chain, l) elements evaluated, l0 <= l <= l_max
 *   [1] summed    -- elements whose term entered the sum (from the first |d| >= 1e-30 on)
 * The library ADDS to the counters (atomically); the caller zeroes them. */
typedef unsigned long long wg_counter;

/* ---------------------------------------------------------------------------
 * wigner_d_table -- the full table (Sec. 3.2 l-recursion, Eqs. lrec, ini1-ini2, logstart).
 *   d_out[mb][ms][l][j] = d^l_{mb,ms}(beta_j),  shape (mb_max+1, ms_max+1, l_max+1, n_beta),
 *   float64, 8-byte aligned; entries with l < max(mb, ms) are written as 0 (every element
 *   of d_out is written).
 *   form: WG_FP64 (WG_FP64S is taken as WG_FP64) or WG_FP32X (the stored values are double
 *   in both cases).
 *   counters: optional, see above.
 *   Per call the library takes stream-ordered scratch from its own memory pool (the FP64
 *   form: 56 B per angle, 24 B per column and order, 24 B per column) and returns it on
 *   the same stream.  An angle outside [0, pi] makes its entries NaN and sets the device
 *   status (wigner_device_status returns WG_ERR_ARG).
 * Errors: WG_ERR_ARG for bad orders/sizes/pointers; WG_ERR_ALLOC when the scratch cannot
 * be allocated; WG_ERR_CUDA on launch failure.
 * ------------------------------------------------------------------------- */
int wigner_d_table(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                   wg_form form, double *d_out, wg_counter *counters, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_d_table_backward -- adjoint of wigner_d_table with respect to beta.
 *   grad_beta[j] = sum_{mb,ms,l} grad_d[mb][ms][l][j] * d/dbeta d^l_{mb,ms}(beta_j)
 *   using Eq. mrec's derivative relation
 *     d/dbeta d^l_{m m'} = ((m' cos b - m)/sin b) d^l_{m m'} - sqrt((l-m')(l+m'+1)) d^l_{m,m'+1}
 *   on recomputed chains (the table is not read).  grad_d has d_out's shape and layout.
 *   grad_beta is OVERWRITTEN (float64[n_beta]).  Angles must be interior (0 < beta < pi);
 *   at the endpoints the result is NaN and WG_ERR_ARG is recorded in the status word.
 *   Uses library workspace of (mb_max+1)(ms_max+1) n_beta doubles (grown on demand).
 * ------------------------------------------------------------------------- */
int wigner_d_table_backward(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                            const double *grad_d, double *grad_beta, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum -- fused recursion + weighted l-sum (Sec. 4.1 Eq. convdef, Sec. 4.2).
 *   a: sky coefficients a[l][ms], wg_c64, shape (l_max+1, ms_max+1), 16-byte aligned.
 *   b: beam coefficients b[l][mb], wg_c64, shape (l_max+1, mb_max+1), 16-byte aligned.
 *   c_out[mb][ms][j] = sum_{l >= max(mb,ms)} conj(b[l][mb]) a[l][ms] d^l_{mb,ms}(beta_j),
 *   wg_c64, shape (mb_max+1, ms_max+1, n_beta), overwritten.
 *   form: WG_FP64, WG_FP64S or WG_FP32X.  counters: optional.
 *   In the FP64 forms the l-ordered weights reach shared memory by TMA, so a and b must
 *   also have row pitches that are multiples of 16 bytes (always true for wg_c64 rows).
 * ------------------------------------------------------------------------- */
int wigner_conv_sum(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                    const wg_c64 *a, const wg_c64 *b, wg_form form, wg_c64 *c_out,
                    wg_counter *counters, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum_host -- wigner_conv_sum (Sec. 4.1 Eq. convdef) on HOST buffers.
 *   beta_host, a_host, b_host, c_host: host memory with the layouts of wigner_conv_sum;
 *   page-locked (cudaHostAlloc / pinned) memory lets the copies overlap the computation,
 *   pageable memory works but is copied synchronously.
 *   The inputs are uploaded on `stream`, the sum runs, and C is downloaded on a
 *   library-owned stream that `stream` then waits for.  The columns can be computed in
 *   blocks of sky orders whose downloads overlap the next block's computation; at the
 *   measured ~200 GB/s host link one block is fastest for the workloads here, and the
 *   environment variable WIGNER_HOST_BLOCKS (1..16) sets another count.  On return all
 *   work is enqueued and `stream` waits for the downloads: synchronise `stream` before
 *   reading c_host.  The host buffers must stay valid until then.
 *   Device buffers come from a library-owned stream-ordered pool (allocated on first use,
 *   kept for later calls), so calls on different streams may run concurrently.
 *   Errors: as wigner_conv_sum (NULL host buffers: WG_ERR_ARG; no room: WG_ERR_ALLOC).
 * ------------------------------------------------------------------------- */
int wigner_conv_sum_host(int l_max, int mb_max, int ms_max, int n_beta, const double *beta_host,
                         const wg_c64 *a_host, const wg_c64 *b_host, wg_form form, wg_c64 *c_host,
                         void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum_full -- the sum of Eq. convdef over EVERY sky order, -ms_max <= m_sky
 * <= ms_max (the C_{m_b m_sky}(beta) of the conviqt data cube, Sec. 4.1 Eq. conviqt),
 * for a real sky field, s_{l,-m} = (-1)^m conj(s_{l m}) (Sec. 4.2 symmetries), so a
 * holds only m_sky >= 0 as in wigner_conv_sum.
 *   The angle grid must be mirror-symmetric: beta[N-1-j] = pi - beta[j] (to ~10 ulp),
 *   as Gauss-Legendre and equispaced grids are.  Each chain (m_b, m_sky >= 0) at
 *   beta[j] then also yields the order -m_sky at pi - beta[j] by the appendix identity
 *   d^l_{m,-m'}(pi - beta) = (-1)^{l+m} d^l_{m m'}(beta) (the corrected sign): a second
 *   weighted sum over the same recursion (Sec. 4.2, "use of symmetries").  A grid that
 *   is not mirror-symmetric makes the negative orders NaN and records WG_ERR_ARG in
 *   the device status word.
 *   c_out[mb][ms + ms_max][j], wg_c64, shape (mb_max+1, 2 ms_max+1, n_beta), overwritten;
 *   C_{-m_b,-m_sky} = conj(C_{m_b m_sky}) gives the negative beam orders.
 *   form: WG_FP64 or WG_FP64S (WG_FP32X: WG_ERR_UNSUPPORTED).  counters: optional (per
 *   chain, as wigner_conv_sum).
 * ------------------------------------------------------------------------- */
int wigner_conv_sum_full(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                         const wg_c64 *a, const wg_c64 *b, wg_form form, wg_c64 *c_out,
                         wg_counter *counters, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_data_cube -- the conviqt data cube of Sec. 4.1, Eq. conviqt:
 *   cube[j][p][q] = sum_{m_b=-mb_max}^{mb_max} sum_{m_sky=-ms_max}^{ms_max}
 *                   e^{-i m_b alpha_p} e^{-i m_sky gamma_q} C_{m_b m_sky}(beta_j),
 *   alpha_p = 2 pi p / n_alpha, gamma_q = 2 pi q / n_gamma,
 *   from c_full = the output of wigner_conv_sum_full (m_b >= 0; the negative beam orders
 *   follow from C_{-m_b,-m_sky} = conj(C_{m_b m_sky}), Sec. 4.2).  For real sky and beam
 *   fields the cube is real: float64, shape (n_beta, n_alpha, n_gamma), overwritten.
 *   n_alpha >= 2 mb_max + 1 and n_gamma >= 2 ms_max + 1 (no aliasing); sizes with small
 *   prime factors transform fastest.  A kernel of the library scatters C into the
 *   Hermitian half spectrum (through the library's stream-ordered pool: n_beta n_alpha
 *   (n_gamma/2+1) complex values of scratch); cuFFT (libcufft.so.12, loaded at the first
 *   call; WG_ERR_UNSUPPORTED if it cannot be) runs the batched 2-D complex-to-real
 *   transforms.  cuFFT plans are kept per (device, n_alpha, n_gamma, n_beta) for the
 *   process, with the workspace cuFFT allocates for them.
 *   Errors: WG_ERR_ARG (orders, sizes, NULL or misaligned pointers), WG_ERR_ALLOC,
 *   WG_ERR_CUDA (launch or cuFFT failure), WG_ERR_UNSUPPORTED.
 * ------------------------------------------------------------------------- */
int wigner_data_cube(int mb_max, int ms_max, int n_beta, const wg_c64 *c_full, int n_alpha, int n_gamma,
                     double *cube, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_d_matrix -- rows of the whole matrix d^l(beta) at one l (the evaluator of
 * Sec. 3.1): d_out[j][m][m' + l] = d^l_{m m'}(beta_j) for 0 <= m <= m_max, -l <= m' <= l;
 * float64, shape (n_beta, m_max+1, 2l+1) (one matrix per angle), 8-byte aligned,
 * overwritten.  The rows m < 0 follow from d_{-m,-m'} = (-1)^{m-m'} d_{m m'}.
 *   Each row runs the three-term relation in m' (Eq. mrec) in its stable direction
 *   (Sec. 2, Eq. classiccond): from m' = l down to m* = round(m cos beta), the centre of
 *   the classical band, and from m' = -l up to m* - 1 (as the same run at pi - beta),
 *   both from the exact edge seeds d^l_{m,+-l} of Eqs. ini1-ini2 in scaled doubles
 *   (Sec. 3.2).  This replaces the paper's ratios anchored at m' = 0, which lose accuracy
 *   below the band when m > 0 and sin beta is small.  beta = 0 gives the identity.
 *   One warp runs 32 consecutive rows of one angle, so a single angle fills the GPU
 *   once m_max is in the thousands.
 *   counters: optional, [0] += (m_max+1)(2l+1) n_beta.
 *   Errors: WG_ERR_ARG (l outside [0, WG_LMAX], m_max outside [0, l], pointers).
 * ------------------------------------------------------------------------- */
int wigner_d_matrix(int l, int m_max, int n_beta, const double *beta, double *d_out,
                    wg_counter *counters, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_ylm -- the polar part of the spherical harmonics (Sec. 2: d^l_{m0} with the
 * normalisation of Y_l^m): out[m][l][j] = sqrt((2l+1)/(4 pi)) d^l_{m 0}(theta_j), so that
 * Y_l^m(theta, phi) = out[m][l][j] e^{i m phi} (Condon-Shortley phase); zero for l < m.
 *   float64, shape (m_max+1, l_max+1, n_theta), overwritten; 0 <= m_max <= l_max.
 *   Computed by the l-recursion of wigner_d_table (m_sky = 0) with the normalisation
 *   applied as each value is stored.  Errors: as wigner_d_table.
 * ------------------------------------------------------------------------- */
int wigner_ylm(int l_max, int m_max, int n_theta, const double *theta, double *out, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum_lmin -- the sum of Eq. convdef with the l_min cut of Sec. 4.2.1
 * (Eq. lmin, its approximate line): each chain (m_b, m_sky, beta_j) sums from
 *   l_min = (sqrt(m_sky^2 + m_b^2 - 2 m_sky m_b cos beta_j) - offset) / sin beta_j
 * (and from the first |d| >= 1e-30, as wigner_conv_sum); the terms below lie in the
 * non-classical region, so the error falls steeply as offset grows (offset >= m_b + m_sky
 * cuts nothing).  At beta = 0 (d = delta) a chain with m_b != m_sky is cut whole.  Chains
 * cut whole are not computed: a CTA whose chains are all cut skips the column, a warp
 * whose chains are all cut skips its steps, and their C is 0.
 *   full = 0: the layout and inputs of wigner_conv_sum; full != 0: of wigner_conv_sum_full
 *   (every sky order on a mirror-symmetric grid; the mirrored chain has the same l_min).
 *   offset: any value but NaN (WG_ERR_ARG); the paper uses offset >= l_max / 20.
 *   l_min is computed in double with each operation rounded once; an angle whose l_min
 *   lies within rounding of an integer may place the cut one order either way.
 *   form: WG_FP64 or WG_FP64S (WG_FP32X: WG_ERR_UNSUPPORTED).  counters: [0] counts the
 *   elements of the chains whose warp ran the recursion.  Errors: as wigner_conv_sum.
 * ------------------------------------------------------------------------- */
int wigner_conv_sum_lmin(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                         const wg_c64 *a, const wg_c64 *b, wg_form form, double offset, int full,
                         wg_c64 *c_out, wg_counter *counters, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum_multi -- the sum of Eq. convdef for n_col weight columns at once:
 *   c_out[k][mb][ms][j] = sum_l conj(b_k[l][mb]) a[k][l][ms] d^l_{mb,ms}(beta_j),  0 <= k < n_col.
 *   Polarised convolution (the footnote of Sec. 4.1) adds the sums of the pairs
 *   (b^T, s^T), (b^G, s^G), (b^C, s^C); a Monte-Carlo run convolves many skies with one
 *   beam.  Every column needs the same d^l, so the recursion runs once per pass of up to
 *   four columns: 2 + 2K FP64 FMAs per element and K columns (WG_FP64), against 4K for K
 *   separate wigner_conv_sum calls.  The weights are read with plain loads.
 *   a: wg_c64, shape (n_col, l_max+1, ms_max+1), 16-byte aligned.
 *   b: wg_c64, shape (l_max+1, mb_max+1) if b_shared != 0 (one beam for every column),
 *      else (n_col, l_max+1, mb_max+1); 16-byte aligned.
 *   sum_cols = 0: c_out[k] holds column k, shape (n_col, mb_max+1, ms_max+1, n_beta);
 *      ceil(n_col / 4) launches, or, with b_shared and n_col >= WG_MULTI_TC_MIN_COLS, the
 *      tensor-core path of wigner_conv_sum_multi_tc.
 *   sum_cols != 0: c_out holds sum_k of the columns (the polarised total), shape
 *      (mb_max+1, ms_max+1, n_beta); the weight sum_k conj(b_k) a_k is formed per l inside
 *      the kernel, so this costs one column's work; one launch (n_col = 0 gives zeros).
 *   c_out is overwritten.
 *   form: WG_FP64 or WG_FP64S (WG_FP32X: WG_ERR_UNSUPPORTED).  counters: optional; the
 *   element counts are those of one column (the chains are shared).
 *   No allocation.  Errors: as wigner_conv_sum.
 * ------------------------------------------------------------------------- */
int wigner_conv_sum_multi(int l_max, int mb_max, int ms_max, int n_beta, int n_col, const double *beta,
                          const wg_c64 *a, const wg_c64 *b, int b_shared, int sum_cols, wg_form form,
                          wg_c64 *c_out, wg_counter *counters, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum_multi_tc -- the separate-column sum of wigner_conv_sum_multi for many
 * skies that share one beam (the Monte-Carlo use of Sec. 4.1), on the tensor cores.
 * wigner_conv_sum_multi routes here when sum_cols == 0, b_shared != 0 and
 * n_col >= WG_MULTI_TC_MIN_COLS (either FP64 form).
 *   c_out[k][mb][ms][j] = sum_l conj(b[l][mb]) a[k][l][ms] d^l_{mb,ms}(beta_j), 0 <= k < n_col.
 *   Per chain column and 128 angles the l-sum is a real matrix product, rows = angles
 *   (Re b_l d^l, and Im b_l d^l for beam orders whose Im b is not 0), columns = the 2 n_col
 *   real and imaginary parts of the skies.  Each operand value is scaled into (-1, 1) by a
 *   power of two and split exactly into six 7-bit bf16 slices; tcgen05.mma accumulates the
 *   21 slice products of the leading levels in tensor memory (exact in FP32 for 256 orders),
 *   folded every 256 orders into float-float accumulators.  Error per term below 2^-42
 *   of max|a| max|b|: the FP64 path's 1e-11 bar holds (tests/ check it).  The recursion
 *   is the FP64 two-FMA recursion of wigner_conv_sum; it runs once per 32 skies.
 *   a: wg_c64 (n_col, l_max+1, ms_max+1); b: wg_c64 (l_max+1, mb_max+1); both 16-byte
 *   aligned with the layouts of wigner_conv_sum_multi.  c_out overwritten.
 *   Scratch: n_col (ms_max+1) + 2 (mb_max+1) ints from the library's stream-ordered pool
 *   (the per-column power-of-two scales), released in stream order.
 *   counters: [0] and [1] += the elements of the chains (counted once).
 *   Errors: WG_ERR_ARG (sizes, NULL or misaligned pointers), WG_ERR_ALLOC, WG_ERR_CUDA;
 *   a bounded wait that gives up: WG_ERR_TIMEOUT in the status word, outputs NaN.
 * ------------------------------------------------------------------------- */
#define WG_MULTI_TC_MIN_COLS 8
int wigner_conv_sum_multi_tc(int l_max, int mb_max, int ms_max, int n_beta, int n_col, const double *beta,
                             const wg_c64 *a, const wg_c64 *b, wg_c64 *c_out, wg_counter *counters, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum_backward -- adjoint of wigner_conv_sum for a real loss L, in
 * PyTorch's convention for complex tensors (grad = dL/dRe + i dL/dIm):
 *   grad_a[l][ms]  = sum_mb b[l][mb] S[l][mb][ms],      S = sum_j grad_c[mb][ms][j] d^l(beta_j)
 *   grad_b[l][mb]  = sum_ms a[l][ms] conj(S[l][mb][ms])
 *   grad_beta[j]   = Re sum_{mb,ms} conj(grad_c) sum_l w_l d/dbeta d^l(beta_j)
 * with d/dbeta d^l from Eq. mrec's relation (the m_sky+1 neighbour chain), chains
 * recomputed (no stored table).  c_fwd is the forward result for the same inputs
 * (used by the beta term); it may be NULL when grad_beta is NULL.
 * grad_a, grad_b, grad_beta may each be NULL (not computed) and are OVERWRITTEN.
 * Shapes as in wigner_conv_sum.  FP64 only (form argument reserved: pass WG_FP64).
 * Uses library workspace of (l_max+1)(mb_max+1)(ms_max+1) complex values.
 * ------------------------------------------------------------------------- */
int wigner_conv_sum_backward(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                             const wg_c64 *a, const wg_c64 *b, const wg_c64 *c_fwd,
                             const wg_c64 *grad_c, wg_c64 *grad_a, wg_c64 *grad_b,
                             double *grad_beta, wg_form form, void *stream);

/* ---------------------------------------------------------------------------
 * Batched uneven instances in one persistent launch.  The chains of different angles
 * are independent (Sec. 4.1 distributes angle subsets over tasks for this reason), so
 * whole fused sums of different l_max, mb_max, n_beta and form can share one launch.
 * Each instance is one wigner_conv_sum problem (same layouts, device pointers inside);
 * the plan splits every instance into work items (instance, angle chunk, group of chain
 * columns) sorted longest first, and a persistent kernel (one CTA per resident slot)
 * pulls them from an atomic counter; no CTA ever waits for another.
 *
 * wigner_batch_plan_create: inst is a HOST array of n descriptors (copied).  The plan
 *   owns device copies of the descriptors and the work list and allocates them here.
 *   autotune != 0 times the compiled (threads, chains per thread, l-tile) variants on a
 *   sample of the plan's own items and keeps the fastest -- this RUNS kernels that write
 *   the instances' outputs on `stream` and synchronises it; the choice is cached per
 *   process, and in the JSON file named by the environment variable WIGNER_TUNE_CACHE
 *   if set (key: GPU name + a hash of the instance shapes and forms).
 * wigner_batch_run: runs every instance (outputs overwritten).  use_graph != 0 captures
 *   the run (counter reset + persistent kernel) into a CUDA graph on the first call and
 *   replays it afterwards; the graph keeps the pointers given at plan creation, so the
 *   instances' buffers must stay allocated (their contents may change between runs).
 * wigner_batch_plan_destroy: synchronises the last stream the plan ran on, then frees.
 * wigner_batch_plan_info: chosen variant, number of work items, persistent grid size.
 * wigner_conv_sum_batched: create (no autotune) + run + destroy; blocks until done.
 * Errors: WG_ERR_ARG names the first bad instance; WG_ERR_ALLOC / WG_ERR_CUDA.
 * ------------------------------------------------------------------------- */
typedef struct {
    int l_max, mb_max, ms_max, n_beta;
    wg_form form;
    const double *beta;
    const wg_c64 *a, *b;
    wg_c64 *c_out;
} wg_instance;

typedef struct wg_batch_plan wg_batch_plan;

int wigner_batch_plan_create(wg_batch_plan **plan, int n, const wg_instance *inst, int autotune,
                             void *stream);
int wigner_batch_run(wg_batch_plan *plan, int use_graph, void *stream);
void wigner_batch_plan_destroy(wg_batch_plan *plan);
int wigner_batch_plan_info(const wg_batch_plan *plan, int *variant, int *n_items, int *grid);
int wigner_conv_sum_batched(int n, const wg_instance *inst, void *stream);

/* ---------------------------------------------------------------------------
 * wigner_conv_sum_noalloc -- wigner_conv_sum (form WG_FP64, no counters) that never
 * allocates memory.  The paper has no counterpart: this entry point exists for callers
 * that cannot let a library call cudaMalloc -- code running while a CUDA graph is being
 * captured, applications that hand all device memory to their own pool allocator, and
 * real-time loops that must not enter the driver's allocator.  wigner_conv_sum keeps
 * its constant tables in device memory it allocates on first use; this variant runs the
 * same kernel with those tables in a fixed array of WG_NOALLOC_LMAX-sized tables
 * (about 640 KiB) compiled into the library, which every GPU that loads the library
 * holds until the process exits.
 *   Arguments, layouts and results as wigner_conv_sum.  l_max > WG_NOALLOC_LMAX is
 *   rejected with WG_ERR_ARG (use wigner_conv_sum for larger problems).
 *   Set-up: the first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress, with that device current) and fills it with a synchronous
 *   host-to-device copy (no allocation).  Make that first call before any stream
 *   capture, and do not overlap it with another call of this entry point on the same
 *   device: until it returns, the array is being written.  Later calls only read the
 *   array (its contents never change after set-up), so they may overlap one another.
 *   The set-up also clears this entry point's own status word (a file-scope device
 *   variable, like the tables) and waits for the device before the first launch, so the
 *   first call may be made on any stream, blocking or not.
 *   Device-side conditions go to that status word, which wigner_noalloc_status reads
 *   and clears (never wigner_device_status, whose word is allocated): an angle outside
 *   [0, pi] (its outputs NaN; WG_ERR_ARG) and a bounded TMA wait that gave up (the
 *   abandoned outputs NaN; WG_ERR_TIMEOUT).  The word is shared by every call on the
 *   device and keeps its bits until read.
 *   Calls no cudaMalloc, cudaFree or other allocating routine, on the host heap either.
 * ------------------------------------------------------------------------- */
#define WG_NOALLOC_LMAX 8192
int wigner_conv_sum_noalloc(int l_max, int mb_max, int ms_max, int n_beta, const double *beta,
                            const wg_c64 *a, const wg_c64 *b, wg_c64 *c_out, void *stream);

/* wigner_noalloc_status -- synchronises `stream`, then returns and clears the status word
 * of wigner_conv_sum_noalloc on the current device: WG_OK, WG_ERR_TIMEOUT (a bounded wait
 * gave up) or WG_ERR_ARG (an angle outside [0, pi]); WG_OK if the entry point has not run
 * on this device.  Allocates nothing (symbol copies of one int). */
int wigner_noalloc_status(void *stream);

/* ---------------------------------------------------------------------------
 * Plans: reserve the library's device state up front.
 * wigner_plan_create makes the constant tables (ln n!, P_i, Q_i, ...) for every
 * l_max <= prm->l_max_cap exist on the current device and, with
 * prm->reserve_backward != 0, the adjoints' workspace for problems up to
 * (l_max_cap, mb_max_cap, ms_max_cap, n_beta_cap).  Calls within those caps then
 * allocate nothing, so they may be captured into a CUDA graph.  This call allocates and
 * synchronises the device; make it before any capture.  The tables and workspace are
 * per-device library state shared by all calls; wigner_plan_destroy releases only the
 * plan handle (the state lives until the process exits).
 * Errors: WG_ERR_ARG (NULL plan or params, caps out of range), WG_ERR_ALLOC, WG_ERR_CUDA.
 * ------------------------------------------------------------------------- */
typedef struct {
    int l_max_cap, mb_max_cap, ms_max_cap, n_beta_cap;
    int reserve_backward;
} wg_params;

typedef struct wg_plan wg_plan;

int wigner_plan_create(wg_plan **plan, const wg_params *prm);
void wigner_plan_destroy(wg_plan *plan);

/* ---------------------------------------------------------------------------
 * Status and diagnostics
 * ------------------------------------------------------------------------- */
/* Synchronises `stream`, returns and clears the device status word of the current
 * device: WG_OK, WG_ERR_ARG (an angle out of range) or WG_ERR_TIMEOUT (a bounded
 * wait gave up). */
int wigner_device_status(void *stream);
const char *wigner_error_string(int code);
/* Text of the last host-side failure on this thread (empty if none). */
const char *wigner_last_error_message(void);
/* Code of the last failing call on this thread (WG_OK if none has failed). */
int wigner_last_error(void);
/* Library version and the compute capability it was built for (e.g. 1003 = sm_103). */
int wigner_version(void);
int wigner_built_arch(void);

/* ---------------------------------------------------------------------------
 * FMA-pipe microbenchmark (measures the roofline denominators of the path).
 *   pipe = 0: FP64 FMA, 1: FP32 FMA.  Runs `iters` steps of `chains` (1, 2, 4, 8 or 16)
 *   independent chains per thread on blocks x threads (threads <= 256, a multiple of
 *   32): FP64 chains are three-term recursions x' = fma(y, x, -x_prev), the operand
 *   pattern of the l-recursion, with every operand in a register (a DFMA that reads a
 *   constant-bank operand does not reach the FP64 pipe's rate on GB300), FP32 chains
 *   x = fma(x, a, b).  Writes a sink value
 *   per thread to sink (device, blocks*threads doubles) so the work cannot be elided.
 *   Returns the number of FMA lane-operations performed in *fma_ops (host).
 * ------------------------------------------------------------------------- */
int wigner_fma_peak(int pipe, int chains, int blocks, int threads, int iters, double *sink,
                    unsigned long long *fma_ops, void *stream);

/* ---------------------------------------------------------------------------
 * Test hooks for the failure paths (host side only; nothing here makes a GPU fault).
 * wigner_debug_inject_alloc_failures: the library's next n device allocations (tables,
 *   status word, adjoint workspace, batch plans, host-call buffers) fail as if the
 *   device were out of memory, without calling the allocator: the call that needed the
 *   memory returns WG_ERR_ALLOC and allocates nothing; n = 0 clears.  Process-wide.
 * wigner_debug_set_wait_tries: the number of tries of each bounded mbarrier wait (the
 *   TMA weight pipeline of the FP64 fused sums) in launches made from now on; default
 *   2^20, 0 makes every such wait give up at once.  A wait that gives up records
 *   WG_ERR_TIMEOUT in the status word (wigner_device_status, or wigner_noalloc_status
 *   for wigner_conv_sum_noalloc), waits with the default limit for the copies it has
 *   already issued, and writes NaN to the outputs its CTA abandons.  Process-wide.
 * wigner_debug_wait_tries: the current value.
 * Errors: WG_ERR_ARG for a negative argument.
 * ------------------------------------------------------------------------- */
int wigner_debug_inject_alloc_failures(int n);
int wigner_debug_set_wait_tries(int tries);
int wigner_debug_wait_tries(void);

#ifdef __cplusplus
}
#endif
#endif /* WIGNER_GB300_H */
