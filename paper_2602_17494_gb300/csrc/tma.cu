// Host side of the TMA tensor maps: cuTensorMapEncodeTiled is a driver API
// call, reached through the runtime's entry-point lookup so that the library
// does not link libcuda directly.
#include "tma.cuh"
#include "tvs_internal.cuh"

#include <mutex>

namespace tvs {

namespace {
using EncodeFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                              const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                              CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeFn encoder() {
    static EncodeFn fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    });
    return fn;
}
}  // namespace

bool make_tensor_map(CUtensorMap* map, const void* base, int storage, int rows, int cols, int pitch, long plane,
                     int planes, int box_x, int box_y) {
    EncodeFn enc = encoder();
    if (!enc) return false;
    CUtensorMapDataType dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    if (storage == TVS_BF16) dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    else if (storage == TVS_F16) dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16;
    else if (storage == TVS_S16) dt = CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const size_t es = storage_bytes(storage);
    const cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
    const cuuint64_t strides[2] = {(cuuint64_t)pitch * es, (cuuint64_t)plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, (cuuint32_t)planes};
    const cuuint32_t estr[3] = {1u, 1u, 1u};
    const CUresult r = enc(map, dt, planes > 1 ? 3u : 2u, const_cast<void*>(base), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace tvs
