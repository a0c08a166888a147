// wg_cube.cu -- the conviqt data cube (Sec. 4.1, Eq. conviqt):
//
//   c(alpha_p, beta_j, gamma_q) = sum_{m_b=-M}^{M} sum_{m_sky=-S}^{S} e^{-i m_b alpha_p} e^{-i m_sky gamma_q}
//                                 C_{m_b m_sky}(beta_j),   alpha_p = 2 pi p / N_a, gamma_q = 2 pi q / N_g,
//
// from the C of every sky order (wigner_conv_sum_full: m_b >= 0, -S <= m_sky <= S; the
// negative beam orders follow from C_{-m_b,-m_sky} = conj(C_{m_b m_sky}), Sec. 4.2).
// With that symmetry c is real, and c = sum conj(C_{m_b m_sky}) e^{+i(m_b alpha + m_sky gamma)}:
// a complex-to-real inverse 2-D DFT of Z[m_b mod N_a][m_sky] = conj(C_{m_b m_sky}) over
// the half spectrum 0 <= m_sky <= N_g / 2.  Our kernel scatters C into Z (a transpose
// through shared memory: C has beta innermost, Z m_sky innermost); cuFFT runs the
// batched 2-D Z2D transform (one per angle), loaded at run time so that the rest of the
// library does not depend on it.
#include <cuda_runtime.h>
#include <cufft.h>  // types only; the functions are looked up with dlsym
#include <dlfcn.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "../../include/wigner.h"
#include "wg_internal.h"

namespace wg {
void set_last_error(const std::string &msg, int code);
int host_pool(cudaMemPool_t *pool);  // wg_host.cu
}  // namespace wg

namespace {

int fail(int code, const std::string &msg) {
    wg::set_last_error(msg, code);
    return code;
}

// ---- cuFFT, looked up once ----
typedef cufftResult (*PlanManyFn)(cufftHandle *, int, int *, int *, int, int, int *, int, int, cufftType, int);
typedef cufftResult (*SetStreamFn)(cufftHandle, cudaStream_t);
typedef cufftResult (*ExecZ2DFn)(cufftHandle, cufftDoubleComplex *, cufftDoubleReal *);
struct CufftApi {
    PlanManyFn plan_many = nullptr;
    SetStreamFn set_stream = nullptr;
    ExecZ2DFn exec_z2d = nullptr;
    bool ok = false;
};

const CufftApi &cufft() {
    static std::once_flag once;
    static CufftApi api;
    std::call_once(once, [] {
        void *h = dlopen("libcufft.so.12", RTLD_NOW | RTLD_LOCAL);
        if (!h) h = dlopen("/usr/local/cuda/lib64/libcufft.so.12", RTLD_NOW | RTLD_LOCAL);
        if (!h) h = dlopen("libcufft.so", RTLD_NOW | RTLD_LOCAL);
        if (!h) return;
        api.plan_many = (PlanManyFn)dlsym(h, "cufftPlanMany");
        api.set_stream = (SetStreamFn)dlsym(h, "cufftSetStream");
        api.exec_z2d = (ExecZ2DFn)dlsym(h, "cufftExecZ2D");
        api.ok = api.plan_many && api.set_stream && api.exec_z2d;
    });
    return api;
}

// plans per (device, N_a, N_g, batch), kept for the process
std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, cufftHandle> g_plans;

constexpr int TB = 32;  // transpose tile (beta x m_sky)

// Z[j][p][k] = conj(C_{m_b, k}(beta_j)) for p = m_b mod N_a, |m_b| <= M, 0 <= k <= S, with
// C_{-m_b, k} = conj(C_{m_b, -k}); every other entry of Z is zero (written here too).
// grid: (ceil(NH / TB), ceil(NB / TB), N_a), NH = N_g / 2 + 1; block TB x 8.
__global__ void __launch_bounds__(TB * 8) cube_scatter_kernel(const double2 *__restrict__ C, int mb_max,
                                                              int ms_max, int n_beta, int n_a, int nh,
                                                              double2 *__restrict__ Z) {
    __shared__ double2 tile[TB][TB + 1];
    const int p = blockIdx.z;
    // the beam order stored at row p, and where it comes from
    const int mb = (p <= mb_max) ? p : p - n_a;  // p in [N_a - M, N_a) holds m_b = p - N_a < 0
    const bool have = (mb >= -mb_max && mb <= mb_max);
    const int k0 = blockIdx.x * TB, j0 = blockIdx.y * TB;
    const int S = ms_max, NS = 2 * ms_max + 1;
    // read: threads along beta (innermost in C)
    for (int r = threadIdx.y; r < TB; r += blockDim.y) {
        const int k = k0 + r, j = j0 + threadIdx.x;
        double2 v = make_double2(0.0, 0.0);
        if (have && k <= S && j < n_beta) {
            if (mb >= 0) {  // conj(C_{m_b, k})
                const double2 c = C[((size_t)mb * NS + (S + k)) * n_beta + j];
                v = make_double2(c.x, -c.y);
            } else {  // conj(C_{m_b, k}) = C_{-m_b, -k}
                v = C[((size_t)(-mb) * NS + (S - k)) * n_beta + j];
            }
        }
        tile[r][threadIdx.x] = v;
    }
    __syncthreads();
    // write: threads along m_sky (innermost in Z)
    for (int r = threadIdx.y; r < TB; r += blockDim.y) {
        const int j = j0 + r, k = k0 + threadIdx.x;
        if (j < n_beta && k < nh) Z[((size_t)j * n_a + p) * nh + k] = tile[threadIdx.x][r];
    }
}

}  // namespace

namespace wg {
int cube_launch(const double2 *C, int mb_max, int ms_max, int n_beta, int n_a, int n_g, double *cube,
                cudaStream_t s);
}

int wg::cube_launch(const double2 *C, int mb_max, int ms_max, int n_beta, int n_a, int n_g, double *cube,
                    cudaStream_t s) {
    const CufftApi &api = cufft();
    if (!api.ok) return fail(WG_ERR_UNSUPPORTED, "cuFFT (libcufft.so.12) could not be loaded");
    int dev = 0;
    cudaGetDevice(&dev);
    cufftHandle plan;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto key = std::make_tuple(dev, n_a, n_g, n_beta);
        auto it = g_plans.find(key);
        if (it == g_plans.end()) {
            int n[2] = {n_a, n_g};
            if (api.plan_many(&plan, 2, n, nullptr, 1, 0, nullptr, 1, 0, CUFFT_Z2D, n_beta) != CUFFT_SUCCESS)
                return fail(WG_ERR_CUDA, "cufftPlanMany failed");
            g_plans[key] = plan;
        } else {
            plan = it->second;
        }
    }
    const int nh = n_g / 2 + 1;
    cudaMemPool_t pool;
    int rc = wg::host_pool(&pool);
    if (rc != WG_OK) return rc;
    void *z = nullptr;
    cudaError_t e = cudaMallocFromPoolAsync(&z, (size_t)n_beta * n_a * nh * sizeof(double2), pool, s);
    if (e != cudaSuccess) return fail(WG_ERR_ALLOC, std::string("cube spectrum: ") + cudaGetErrorString(e));
    dim3 grid((nh + TB - 1) / TB, (n_beta + TB - 1) / TB, n_a);
    cube_scatter_kernel<<<grid, dim3(TB, 8), 0, s>>>(C, mb_max, ms_max, n_beta, n_a, nh, (double2 *)z);
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        cufftResult r;
        {
            std::lock_guard<std::mutex> lk(g_mu);  // a plan is bound to one stream at a time
            r = api.set_stream(plan, s);
            if (r == CUFFT_SUCCESS) r = api.exec_z2d(plan, (cufftDoubleComplex *)z, cube);
        }
        if (r != CUFFT_SUCCESS) {
            cudaFreeAsync(z, s);
            return fail(WG_ERR_CUDA, "cufftExecZ2D failed");
        }
    }
    cudaFreeAsync(z, s);
    if (e != cudaSuccess) return fail(WG_ERR_CUDA, std::string("cube scatter launch: ") + cudaGetErrorString(e));
    return WG_OK;
}

extern "C" int wigner_data_cube(int mb_max, int ms_max, int n_beta, const wg_c64 *c_full, int n_alpha,
                                int n_gamma, double *cube, void *stream) {
    if (mb_max < 0 || ms_max < 0 || ms_max > WG_LMAX || mb_max > ms_max || n_beta < 0)
        return fail(WG_ERR_ARG, "orders out of range (0 <= mb_max <= ms_max <= WG_LMAX)");
    if (n_alpha < 2 * mb_max + 1 || n_gamma < 2 * ms_max + 1)
        return fail(WG_ERR_ARG, "n_alpha >= 2 mb_max + 1 and n_gamma >= 2 ms_max + 1 are needed (no aliasing)");
    if (n_alpha > (1 << 20) || n_gamma > (1 << 22)) return fail(WG_ERR_ARG, "n_alpha or n_gamma too large");
    if (n_beta == 0) return WG_OK;
    if (!c_full || ((uintptr_t)c_full & 15)) return fail(WG_ERR_ARG, "c_full is NULL or not 16-byte aligned");
    if (!cube || ((uintptr_t)cube & 7)) return fail(WG_ERR_ARG, "cube is NULL or not 8-byte aligned");
    return wg::cube_launch((const double2 *)c_full, mb_max, ms_max, n_beta, n_alpha, n_gamma, cube,
                           (cudaStream_t)stream);
}
