// tvs_project_noalloc: the divergence-free projection for callers that cannot
// allocate device memory.
//
// Some callers cannot call cudaMalloc or hand the library a workspace: code
// that runs under a memory pool they do not control, or inside a host callback
// or plug-in where allocating is not allowed.  This entry point takes only the
// input and output arrays.  Its scratch (the DCT tables and one plane of
// transform data) lives in one file-scope device array of fixed size, which
// every GPU that loads the library holds until the process exits.
#include "launchers.h"

#include <cstdio>

namespace tvs {
namespace {

constexpr size_t kNoAllocBytes = size_t(5) << 20;   // 5 MiB
constexpr int kNoAllocMaxSide = 1025;                  // grids up to 1025 x 1025 points (images up to 1024^2)

__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

size_t noalloc_need(int rows, int cols) {
    Carver cv(nullptr);
    PoissonPlans pp;
    carve_poisson(cv, pp, rows, cols);
    cv.take<float>((size_t)rows * cols);
    return cv.used();
}

}  // namespace
}  // namespace tvs

using namespace tvs;

extern "C" tvs_status tvs_project_noalloc(const float* in, float* out, int rows, int cols, cudaStream_t stream) {
    if (!in || !out || rows < 3 || cols < 3) return TVS_ERR_ARG;
    if (rows > kNoAllocMaxSide || cols > kNoAllocMaxSide || noalloc_need(rows, cols) > kNoAllocBytes) {
        set_error_text("tvs_project_noalloc: grid larger than 1025 x 1025 points, the most its fixed 5 MiB "
                       "scratch holds");
        return TVS_ERR_UNSUPPORTED;
    }
    // Host code only knows a host-side stand-in for the array, so every call
    // looks up its device address on the current device.  The lookup is a
    // host-side query (the first one on a device loads the library's device
    // code there); doing it on every call keeps the address right after the
    // caller resets the device or its context, where a cached one would be stale.
    void* base = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
    if (e != cudaSuccess) {
        set_error("cudaGetSymbolAddress(g_noalloc_scratch)", e);
        return TVS_ERR_CUDA;
    }
    Carver cv(base);
    PoissonPlans pp;
    carve_poisson(cv, pp, rows, cols);
    float* S = cv.take<float>((size_t)rows * cols);
    // Every scratch word read below is written first in this call (tables,
    // then all rows of S), so nothing from an earlier call needs clearing.
    const long plane = (long)rows * cols;
    if ((e = build_poisson(pp, stream)) != cudaSuccess) {
        set_error("tvs_project_noalloc: tables", e);
        return TVS_ERR_CUDA;
    }
    RowSrcArgs sa{in, plane, cols};
    if ((e = poisson_solve(S, rows, cols, cols, pp, RowSource::DivField, sa, stream)) != cudaSuccess) {
        set_error("tvs_project_noalloc: poisson", e);
        return TVS_ERR_CUDA;
    }
    if ((e = launch_grad_sub(in, cols, plane, S, cols, rows, cols, 1.0f, out, cols, plane, stream)) != cudaSuccess) {
        set_error("tvs_project_noalloc: gradient", e);
        return TVS_ERR_CUDA;
    }
    return TVS_OK;
}
