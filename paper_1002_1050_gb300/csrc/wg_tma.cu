// wg_tma.cu -- host side of the weight staging: tensor-map encoding through the
// runtime's driver entry point (no link against the driver library).
#include <cuda.h>
#include <cuda_runtime.h>

#include <mutex>

#include "wg_tma.cuh"

namespace wg {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    });
    return fn;
}

// a row-major complex128 array [rows][cols] as a 2-D float64 tensor, box {2, tl}
int encode_one(CUtensorMap *map, const double *base, int rows, int cols, int tl) {
    EncodeTiledFn fn = encode_fn();
    if (!fn) return (int)cudaErrorNotSupported;
    const cuuint64_t dims[2] = {(cuuint64_t)2 * (cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)16 * (cuuint64_t)cols};
    const cuuint32_t box[2] = {2u, (cuuint32_t)tl};
    const cuuint32_t estr[2] = {1u, 1u};
    const CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<double *>(base), dims, strides, box, estr,
                          CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : (int)cudaErrorInvalidValue;
}

}  // namespace

int encode_weight_maps(const double *a, const double *b, int l_max, int mb_max, int ms_max, int tl, WeightMaps *out) {
    if (tl < 1 || tl > 256) return (int)cudaErrorInvalidValue;
    int e = encode_one(&out->a, a, l_max + 1, ms_max + 1, tl);
    if (e == 0) e = encode_one(&out->b, b, l_max + 1, mb_max + 1, tl);
    return e;
}

}  // namespace wg
