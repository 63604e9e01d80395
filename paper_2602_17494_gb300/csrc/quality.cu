// Image quality measures of Section 5.3 on the device: PSNR and the
// single-window MSSIM of a reconstruction d against a ground truth gt
// (intensities in [0, 1], so the largest pixel value is 1).  One pass of
// per-thread compensated FP32 sums of d, gt, d^2, gt^2, d gt and (d - gt)^2,
// reduced in FP64 across threads and blocks; the host forms the ratios.
#include "drivers.h"

namespace tvs {

// slots (4 and 5 are max slots of the shared reduction and stay unused)
enum { kQd = 0, kQg = 1, kQdd = 2, kQgg = 3, kQdg = 6, kQee = 7 };
constexpr int kQThreads = 256;

__global__ void __launch_bounds__(kQThreads)
quality_kernel(const float* __restrict__ d, const float* __restrict__ gt, long n, double* __restrict__ partial) {
    KSum s[6];
    for (long i = (long)blockIdx.x * kQThreads + threadIdx.x; i < n; i += (long)gridDim.x * kQThreads) {
        const float a = __ldg(&d[i]), b = __ldg(&gt[i]);
        s[0].add(a);
        s[1].add(b);
        s[2].add(a * a);
        s[3].add(b * b);
        s[4].add(a * b);
        const float e = a - b;
        s[5].add(e * e);
    }
    double acc[kRedSlots] = {s[0].value(), s[1].value(), s[2].value(), s[3].value(), 0.0, 0.0, s[4].value(),
                             s[5].value()};
    block_reduce_store<kQThreads>(acc, partial + (size_t)blockIdx.x * kRedSlots, threadIdx.x);
}

constexpr int kQBlocks = 152 * 4;

size_t quality_layout(Carver& cv, RedBuf& rb) {
    carve_red(cv, rb, kQBlocks);
    return cv.used();
}

}  // namespace tvs

using namespace tvs;

extern "C" tvs_status tvs_quality(const float* d, const float* gt, int n2, int n1, void* ws, size_t ws_bytes,
                                  cudaStream_t stream, double* psnr, double* mssim) {
    if (!d || !gt || !psnr || !mssim || n2 < 1 || n1 < 1) return TVS_ERR_ARG;
    Carver cv0(nullptr);
    RedBuf rb0;
    tvs_status st = check_ws(ws, ws_bytes, quality_layout(cv0, rb0));
    if (st != TVS_OK) return st;
    Carver cv(ws);
    RedBuf rb;
    quality_layout(cv, rb);
    const long n = (long)n2 * n1;
    TVS_CUDA(cudaMemsetAsync(rb.err, 0, sizeof(unsigned), stream));
    quality_kernel<<<kQBlocks, kQThreads, 0, stream>>>(d, gt, n, rb.partial);
    TVS_CUDA(cudaGetLastError());
    double r[kRedSlots];
    st = read_result(rb, kQBlocks, stream, r);
    if (st != TVS_OK) return st;
    const double inv = 1.0 / (double)n;
    const double md = r[kQd] * inv, mg = r[kQg] * inv;
    const double sd2 = r[kQdd] * inv - md * md, sg2 = r[kQgg] * inv - mg * mg, sdg = r[kQdg] * inv - md * mg;
    const double mse = r[kQee] * inv;
    const double c1 = 1e-4, c2 = 9e-4;   // (0.01 R)^2, (0.03 R)^2 with R = 1
    *psnr = mse > 0.0 ? -10.0 * std::log10(mse) : INFINITY;
    *mssim = (2 * md * mg + c1) * (2 * sdg + c2) / ((md * md + mg * mg + c1) * (sd2 + sg2 + c2));
    return TVS_OK;
}
