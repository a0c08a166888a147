// wg_batch.cu -- many uneven fused sums in one persistent launch.
//
// The chains of every (beta, m_b, m_sky) triple are independent (Sec. 4.1: the paper
// distributes beta subsets over MPI tasks for the same reason), so instances of
// different l_max, mb_max, n_beta and precision form can share one launch.  The plan
// splits every instance into work items (instance, chunk of angles, group of chain
// columns), sorts them by estimated cost, longest first, and a persistent kernel -- one
// CTA per resident slot -- pulls items from an atomic counter (no inter-CTA waits) and
// runs the FP64 or FP32-form item code of the single-instance kernels.  An autotuner
// times the compiled (chains per thread, l-tile) variants on a sample of the plan's own
// items; a run can be captured once into a CUDA graph and replayed.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/wigner.h"
#include "wg_conv_fp64.cuh"
#include "wg_fp32x.cuh"
#include "wg_internal.h"

namespace wg {
void set_last_error(const std::string &msg, int code);
int tables_for(int l_max, Tables *t);  // wg_capi.cu

struct BatchInst {
    ConvArgs args;
    int form;
};

template <int NT, int CPT64, int TL64, int CPT32, int TL32>
__global__ void __launch_bounds__(NT) batch_kernel(const BatchInst *__restrict__ insts, const int4 *__restrict__ items,
                                                   int n_items, int *counter, Tables T) {
    __shared__ union {
        SmemFp64<TL64> f64;
        SmemFp32<NT, CPT32, TL32> f32;
    } sm;
    __shared__ int s_item;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(counter, 1);
        __syncthreads();
        const int it = s_item;
        __syncthreads();  // every thread has read s_item before it is overwritten
        if (it >= n_items) break;
        const int4 w = items[it];
        const ConvArgs a = insts[w.x].args;
        const int form = insts[w.x].form;
        unsigned long long ne = 0, ns = 0;
        if (form == WG_FP64)
            conv_fp64_item<NT, CPT64, TL64, false>(a, T, w.y, w.z, w.w, sm.f64, ne, ns);
        else if (form == WG_FP64S)
            conv_fp64_item<NT, CPT64, TL64, true>(a, T, w.y, w.z, w.w, sm.f64, ne, ns);
        else
            conv_fp32x_item<NT, CPT32, TL32>(a, T, w.y, w.z, w.w, sm.f32, ne, ns);
    }
}

// compiled variants: (threads, FP64 chains/thread, FP64 l-tile, FP32 chains/thread, FP32 l-tile)
struct Variant {
    int nt, cpt64, tl64, cpt32, tl32;
    const void *fn;
};

static const Variant kVariants[] = {
    {128, 2, 128, 4, 64, (const void *)batch_kernel<128, 2, 128, 4, 64>},
    {128, 1, 128, 2, 64, (const void *)batch_kernel<128, 1, 128, 2, 64>},
    {128, 2, 64, 4, 128, (const void *)batch_kernel<128, 2, 64, 4, 128>},
    {256, 1, 128, 2, 64, (const void *)batch_kernel<256, 1, 128, 2, 64>},
};
static const int kNumVariants = (int)(sizeof(kVariants) / sizeof(kVariants[0]));

static cudaError_t launch_variant(int v, int grid, const BatchInst *insts, const int4 *items, int n_items,
                                  int *counter, const Tables &T, cudaStream_t s) {
    switch (v) {
        case 0: batch_kernel<128, 2, 128, 4, 64><<<grid, 128, 0, s>>>(insts, items, n_items, counter, T); break;
        case 1: batch_kernel<128, 1, 128, 2, 64><<<grid, 128, 0, s>>>(insts, items, n_items, counter, T); break;
        case 2: batch_kernel<128, 2, 64, 4, 128><<<grid, 128, 0, s>>>(insts, items, n_items, counter, T); break;
        default: batch_kernel<256, 1, 128, 2, 64><<<grid, 256, 0, s>>>(insts, items, n_items, counter, T); break;
    }
    return cudaGetLastError();
}

}  // namespace wg

struct wg_batch_plan {
    int device = 0;
    int variant = 0;
    int grid = 0;
    std::vector<wg_instance> inst;
    wg::Tables tables{};
    wg::BatchInst *d_insts = nullptr;
    int4 *d_items = nullptr;
    int n_items = 0;
    int *d_counter = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    cudaStream_t last_stream = nullptr;
};

namespace {

using wg::kNumVariants;
using wg::kVariants;

struct Item {
    int inst, chunk, k_begin, k_end;
    double cost;
};

// relative cost of an element in each form (measured: the split-pipe FP64 form runs
// ~1.5x and the FP32 form ~6x faster per element than the all-double form)
double form_weight(int form) { return form == WG_FP64 ? 1.0 : (form == WG_FP64S ? 1.0 / 1.5 : 1.0 / 6.0); }

void build_items(const std::vector<wg_instance> &inst, const wg::Variant &v, std::vector<Item> &out) {
    out.clear();
    const double target = 3.0e7;  // element-steps per work item (weighted)
    for (int i = 0; i < (int)inst.size(); ++i) {
        const wg_instance &I = inst[i];
        if (I.n_beta == 0) continue;
        const int cpt = I.form == WG_FP32X ? v.cpt32 : v.cpt64;
        const int per_chunk = v.nt * cpt;
        const int n_chunks = (I.n_beta + per_chunk - 1) / per_chunk;
        const int MB1 = I.mb_max + 1;
        const int ncol = MB1 * (I.ms_max + 1);
        const double w = form_weight(I.form);
        // chain length of column k (m_sky-major: ms = k / MB1, mb = k % MB1)
        auto len = [&](int k) { return (double)(I.l_max + 1 - std::max(k % MB1, k / MB1)); };
        int k = 0;
        while (k < ncol) {
            const int kb = k;
            double c = 0.0;
            while (k < ncol && (k == kb || c * per_chunk * w < target) && k - kb < 64) {
                c += len(k);
                ++k;
            }
            for (int ch = 0; ch < n_chunks; ++ch) {
                const int nb = std::min(per_chunk, I.n_beta - ch * per_chunk);
                out.push_back(Item{i, ch, kb, k, c * nb * w});
            }
        }
    }
    std::stable_sort(out.begin(), out.end(), [](const Item &a, const Item &b) { return a.cost > b.cost; });
}

int upload_items(wg_batch_plan *p, const std::vector<Item> &items) {
    if (p->d_items) cudaFree(p->d_items);
    p->d_items = nullptr;
    p->n_items = (int)items.size();
    if (items.empty()) return WG_OK;
    std::vector<int4> h(items.size());
    for (size_t i = 0; i < items.size(); ++i)
        h[i] = make_int4(items[i].inst, items[i].chunk, items[i].k_begin, items[i].k_end);
    cudaError_t e = wg::alloc_injected() ? cudaErrorMemoryAllocation : cudaMalloc(&p->d_items, h.size() * sizeof(int4));
    if (e != cudaSuccess) {
        p->d_items = nullptr;
        wg::set_last_error(std::string("cudaMalloc(batch items): ") + cudaGetErrorString(e), WG_ERR_ALLOC);
        return WG_ERR_ALLOC;
    }
    e = cudaMemcpy(p->d_items, h.data(), h.size() * sizeof(int4), cudaMemcpyHostToDevice);
    // from pageable memory the copy may return before it has landed, and the plan runs
    // on the caller's stream, which need not be ordered after the legacy stream
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        wg::set_last_error(std::string("cudaMemcpy(batch items): ") + cudaGetErrorString(e), WG_ERR_CUDA);
        return WG_ERR_CUDA;
    }
    return WG_OK;
}

int grid_for(int variant) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kVariants[variant].fn, kVariants[variant].nt, 0);
    return std::max(1, sms * std::max(1, per_sm));
}

int run_once(wg_batch_plan *p, cudaStream_t s) {
    if (p->n_items == 0) return WG_OK;
    cudaError_t e = cudaMemsetAsync(p->d_counter, 0, sizeof(int), s);
    if (e == cudaSuccess)
        e = wg::launch_variant(p->variant, p->grid, p->d_insts, p->d_items, p->n_items, p->d_counter, p->tables, s);
    if (e != cudaSuccess) {
        wg::set_last_error(std::string("batch launch: ") + cudaGetErrorString(e), WG_ERR_CUDA);
        return WG_ERR_CUDA;
    }
    return WG_OK;
}

// ---- tuning cache: in-process map, optionally persisted as a JSON object in $WIGNER_TUNE_CACHE
std::mutex g_tune_mu;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string tune_key(const std::vector<wg_instance> &inst) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceProp prop;
    cudaGetDeviceProperties(&prop, dev);
    // signature: GPU name + per instance (form, l_max bucket, mb_max, n_beta bucket)
    std::string k = prop.name;
    unsigned long long h = 1469598103934665603ull;
    for (const wg_instance &I : inst) {
        const long long vals[4] = {(long long)I.form, (long long)(I.l_max / 512), (long long)I.mb_max,
                                   (long long)(I.n_beta / 256)};
        for (long long x : vals) {
            h ^= (unsigned long long)x + 0x9e3779b97f4a7c15ull;
            h *= 1099511628211ull;
        }
    }
    char buf[40];
    snprintf(buf, sizeof(buf), "|%zu|%016llx", inst.size(), h);
    return k + buf;
}

void tune_load() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = getenv("WIGNER_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "r");
    if (!f) return;
    std::string s;
    char buf[4096];
    size_t n;
    while ((n = fread(buf, 1, sizeof(buf), f)) > 0) s.append(buf, n);
    fclose(f);
    // entries "key": variant
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        size_t colon = s.find(':', end);
        if (colon == std::string::npos) break;
        g_tune[key] = atoi(s.c_str() + colon + 1);
        pos = s.find_first_of(",}", colon);
        if (pos == std::string::npos) break;
    }
}

void tune_store() {
    const char *path = getenv("WIGNER_TUNE_CACHE");
    if (!path) return;
    FILE *f = fopen(path, "w");
    if (!f) return;
    fprintf(f, "{\n");
    size_t i = 0;
    for (const auto &kv : g_tune) fprintf(f, "  \"%s\": %d%s\n", kv.first.c_str(), kv.second, ++i < g_tune.size() ? "," : "");
    fprintf(f, "}\n");
    fclose(f);
}

// Time each compiled variant on a sample of its own work items (about 1/16 of the
// batch's weighted cost, spread over the sorted list) and keep the fastest.
int autotune(wg_batch_plan *p, cudaStream_t s) {
    double best_rate = -1.0;
    int best = 0;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int v = 0; v < kNumVariants; ++v) {
        std::vector<Item> items, sample;
        build_items(p->inst, kVariants[v], items);
        double total = 0.0;
        for (const Item &it : items) total += it.cost;
        const size_t stride = std::max<size_t>(1, items.size() / std::max<size_t>(1, items.size() / 16));
        double scost = 0.0;
        for (size_t i = 0; i < items.size(); i += stride) {
            sample.push_back(items[i]);
            scost += items[i].cost;
        }
        p->variant = v;
        p->grid = grid_for(v);
        int rc = upload_items(p, sample);
        if (rc != WG_OK) return rc;
        rc = run_once(p, s);  // warm-up
        if (rc != WG_OK) return rc;
        cudaEventRecord(e0, s);
        rc = run_once(p, s);
        if (rc != WG_OK) return rc;
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        const double rate = scost / std::max(1e-3, (double)ms);
        if (rate > best_rate) {
            best_rate = rate;
            best = v;
        }
        (void)total;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->variant = best;
    return WG_OK;
}

int validate(const wg_instance &I, int idx) {
    auto bad = [&](const char *what) {
        wg::set_last_error("instance " + std::to_string(idx) + ": " + what, WG_ERR_ARG);
        return WG_ERR_ARG;
    };
    if (I.l_max < 0 || I.l_max > WG_LMAX) return bad("l_max out of range");
    if (I.mb_max < 0 || I.mb_max > I.l_max || I.ms_max < 0 || I.ms_max > I.l_max) return bad("orders out of range");
    if (I.n_beta < 0) return bad("n_beta < 0");
    if (I.form != WG_FP64 && I.form != WG_FP32X && I.form != WG_FP64S) return bad("unknown form");
    if (I.n_beta == 0) return WG_OK;
    if (!I.beta || ((uintptr_t)I.beta % 8)) return bad("beta NULL or misaligned");
    if (!I.a || ((uintptr_t)I.a % 16)) return bad("a NULL or misaligned");
    if (!I.b || ((uintptr_t)I.b % 16)) return bad("b NULL or misaligned");
    if (!I.c_out || ((uintptr_t)I.c_out % 16)) return bad("c_out NULL or misaligned");
    return WG_OK;
}

void free_plan(wg_batch_plan *p) {
    if (!p) return;
    if (p->graph_exec) cudaGraphExecDestroy(p->graph_exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    if (p->d_items) cudaFree(p->d_items);
    if (p->d_insts) cudaFree(p->d_insts);
    if (p->d_counter) cudaFree(p->d_counter);
    delete p;
}

}  // namespace

extern "C" {

int wigner_batch_plan_create(wg_batch_plan **plan, int n, const wg_instance *inst, int autotune_flag, void *stream) {
    if (!plan) {
        wg::set_last_error("plan is NULL", WG_ERR_ARG);
        return WG_ERR_ARG;
    }
    *plan = nullptr;
    if (n < 0 || (n > 0 && !inst)) {
        wg::set_last_error("bad instance list", WG_ERR_ARG);
        return WG_ERR_ARG;
    }
    int max_l = 0;
    for (int i = 0; i < n; ++i) {
        const int rc = validate(inst[i], i);
        if (rc != WG_OK) return rc;
        max_l = std::max(max_l, inst[i].l_max);
    }
    wg_batch_plan *p = new (std::nothrow) wg_batch_plan();
    if (!p) return WG_ERR_ALLOC;
    cudaGetDevice(&p->device);
    p->inst.assign(inst, inst + n);
    int rc = wg::tables_for(max_l, &p->tables);
    if (rc != WG_OK) {
        free_plan(p);
        return rc;
    }
    std::vector<wg::BatchInst> h(n);
    for (int i = 0; i < n; ++i) {
        const wg_instance &I = inst[i];
        h[i].args = wg::ConvArgs{I.l_max, I.mb_max, I.ms_max, I.n_beta, I.beta, (const double *)I.a,
                                 (const double *)I.b, (double *)I.c_out, nullptr};
        h[i].form = (int)I.form;
    }
    cudaError_t e = wg::alloc_injected() ? cudaErrorMemoryAllocation : cudaMalloc(&p->d_counter, sizeof(int));
    if (e == cudaSuccess && n > 0) e = cudaMalloc(&p->d_insts, n * sizeof(wg::BatchInst));
    if (e != cudaSuccess) {
        wg::set_last_error(std::string("cudaMalloc(batch plan): ") + cudaGetErrorString(e), WG_ERR_ALLOC);
        free_plan(p);
        return WG_ERR_ALLOC;
    }
    if (n > 0) {
        e = cudaMemcpy(p->d_insts, h.data(), n * sizeof(wg::BatchInst), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();  // see upload_items
        if (e != cudaSuccess) {
            wg::set_last_error(std::string("cudaMemcpy(batch plan): ") + cudaGetErrorString(e), WG_ERR_CUDA);
            free_plan(p);
            return WG_ERR_CUDA;
        }
    }
    cudaStream_t s = (cudaStream_t)stream;
    int variant = 0;
    bool tuned = false;
    if (autotune_flag && n > 0) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        tune_load();
        const std::string key = tune_key(p->inst);
        auto it = g_tune.find(key);
        if (it != g_tune.end() && it->second >= 0 && it->second < kNumVariants) {
            variant = it->second;
            tuned = true;
        } else {
            rc = autotune(p, s);
            if (rc != WG_OK) {
                free_plan(p);
                return rc;
            }
            variant = p->variant;
            g_tune[key] = variant;
            tune_store();
            tuned = true;
        }
    }
    (void)tuned;
    p->variant = variant;
    p->grid = grid_for(variant);
    std::vector<Item> items;
    build_items(p->inst, kVariants[variant], items);
    rc = upload_items(p, items);
    if (rc != WG_OK) {
        free_plan(p);
        return rc;
    }
    *plan = p;
    return WG_OK;
}

int wigner_batch_run(wg_batch_plan *p, int use_graph, void *stream) {
    if (!p) {
        wg::set_last_error("plan is NULL", WG_ERR_ARG);
        return WG_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    p->last_stream = s;
    if (!use_graph) return run_once(p, s);
    if (!p->graph_exec) {
        cudaStream_t cs;
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            wg::set_last_error(std::string("cudaStreamCreate: ") + cudaGetErrorString(e), WG_ERR_CUDA);
            return WG_ERR_CUDA;
        }
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        int rc = WG_OK;
        if (e == cudaSuccess) rc = run_once(p, cs);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cs, &g);
        cudaStreamDestroy(cs);
        if (e != cudaSuccess || e2 != cudaSuccess || rc != WG_OK || !g) {
            if (g) cudaGraphDestroy(g);
            wg::set_last_error(std::string("graph capture failed: ") + cudaGetErrorString(e != cudaSuccess ? e : e2),
                               WG_ERR_CUDA);
            return rc != WG_OK ? rc : WG_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&p->graph_exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            p->graph_exec = nullptr;
            wg::set_last_error(std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e), WG_ERR_CUDA);
            return WG_ERR_CUDA;
        }
        p->graph = g;
    }
    cudaError_t e = cudaGraphLaunch(p->graph_exec, s);
    if (e != cudaSuccess) {
        wg::set_last_error(std::string("cudaGraphLaunch: ") + cudaGetErrorString(e), WG_ERR_CUDA);
        return WG_ERR_CUDA;
    }
    return WG_OK;
}

void wigner_batch_plan_destroy(wg_batch_plan *p) {
    if (!p) return;
    cudaStreamSynchronize(p->last_stream);
    free_plan(p);
}

int wigner_batch_plan_info(const wg_batch_plan *p, int *variant, int *n_items, int *grid) {
    if (!p) return WG_ERR_ARG;
    if (variant) *variant = p->variant;
    if (n_items) *n_items = p->n_items;
    if (grid) *grid = p->grid;
    return WG_OK;
}

int wigner_conv_sum_batched(int n, const wg_instance *inst, void *stream) {
    wg_batch_plan *p = nullptr;
    int rc = wigner_batch_plan_create(&p, n, inst, 0, stream);
    if (rc != WG_OK) return rc;
    rc = wigner_batch_run(p, 0, stream);
    wigner_batch_plan_destroy(p);  // synchronises the stream
    return rc;
}

}  // extern "C"
