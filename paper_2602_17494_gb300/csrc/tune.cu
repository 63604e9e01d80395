// Autotuner of the step-2 Schwarz decomposition (include/tvs.h,
// tvs_tune_schwarz2).  The paper fixes no tile size, overlap or inner
// iteration count; this picks them per image class by measurement: every
// candidate (core size, overlap, k) runs Algorithm 2 with Algorithm 3 from a
// zero dual to the requested relative duality gap on the caller's image, is
// timed with CUDA events on the caller's stream, and the fastest candidate
// that reached the gap wins.
#include "drivers.h"
#include "graphs.h"

#include <algorithm>

namespace tvs {
namespace {

tvs_decomp tune_decomp(int n2, int n1, int tile, int overlap, int k) {
    tvs_decomp dd{};
    dd.m2 = std::max(1, (n2 + tile - 1) / tile);
    dd.m1 = std::max(1, (n1 + tile - 1) / tile);
    dd.overlap = overlap;
    dd.k_inner = k;
    dd.alpha_hat = 0.0;
    return dd;
}

size_t tune_bytes(int n2, int n1, int tile, int overlap, int storage) {
    const tvs_decomp dd = tune_decomp(n2, n1, tile, overlap, 1);
    if (schwarz2_check(n2, n1, dd) != TVS_OK) return 0;
    Carver cv(nullptr);
    cv.take<float>((size_t)n2 * n1);   // d of the candidate runs
    Step2Layout L;
    layout_step2(cv, n2, n1, L, storage);
    return schwarz2_extend(cv, n2, n1, dd, L.P, storage);
}

}  // namespace
}  // namespace tvs

using namespace tvs;

extern "C" {

size_t tvs_tune_workspace_bytes(int n2, int n1, const int* tiles, int ntiles, const int* overlaps, int noverlaps,
                                int storage) {
    if (!tiles || !overlaps || ntiles < 1 || noverlaps < 1 || !side_ok(n2) || !side_ok(n1) ||
        storage_bytes(storage) == 0)
        return 0;
    size_t need = 0;
    for (int a = 0; a < ntiles; ++a)
        for (int b = 0; b < noverlaps; ++b) need = std::max(need, tune_bytes(n2, n1, tiles[a], overlaps[b], storage));
    return need;
}

tvs_status tvs_tune_schwarz2(const float* d0, const float* tau, int n2, int n1, double alpha, double eps,
                             const tvs_iter* it, const int* tiles, int ntiles, const int* overlaps, int noverlaps,
                             const int* ks, int nks, void* ws, size_t ws_bytes, cudaStream_t stream, int* best,
                             float* best_ms) {
    if (!d0 || !tau || !best || !side_ok(n2) || !side_ok(n1) || !(alpha > 0.0) || !(eps > 0.0) || !tiles ||
        !overlaps || !ks || ntiles < 1 || noverlaps < 1 || nks < 1)
        return TVS_ERR_ARG;
    tvs_status st = check_iter(it, true);
    if (st != TVS_OK) return st;
    if (!(it->rel_gap_tol > 0.0) || it->check_every < 1) return TVS_ERR_ARG;
    for (int i = 0; i < nks; ++i)
        if (ks[i] < 1) return TVS_ERR_ARG;
    const size_t need = tvs_tune_workspace_bytes(n2, n1, tiles, ntiles, overlaps, noverlaps, it->storage);
    if (need == 0) return TVS_ERR_ARG;
    st = check_ws(ws, ws_bytes, need);
    if (st != TVS_OK) return st;
    cudaEvent_t e0, e1;
    TVS_CUDA(cudaEventCreate(&e0));
    TVS_CUDA(cudaEventCreate(&e1));
    float best_t = -1.0f;
    tvs_status result = TVS_ERR_NOT_CONVERGED;
    const int R = n2 + 1, C = n1 + 1;
    for (int a = 0; a < ntiles; ++a)
        for (int b = 0; b < noverlaps; ++b) {
            if (tune_bytes(n2, n1, tiles[a], overlaps[b], it->storage) == 0) continue;   // cores narrower than s
            for (int c = 0; c < nks; ++c) {
                tvs_decomp dd = tune_decomp(n2, n1, tiles[a], overlaps[b], ks[c]);
                Carver cv(ws);
                float* d = cv.take<float>((size_t)n2 * n1);
                Step2Layout L;
                layout_step2(cv, n2, n1, L, it->storage);
                Schwarz2State S2;
                schwarz2_carve(cv, n2, n1, dd, L.P, it->storage, S2);
                cudaError_t ce = cudaEventRecord(e0, stream);
                if (ce == cudaSuccess)
                    ce = launch_xi_f2(d0, n1, tau, (long)R * C, C, n2, n1, (float)alpha, (float)eps, L.f2, L.P, stream);
                if (ce != cudaSuccess) {
                    set_error("tvs_tune_schwarz2", ce);
                    result = TVS_ERR_CUDA;
                    goto out;
                }
                tvs_report rep;
                {
                    GraphsOff direct;   // the timed run must not include graph capture
                    st = run_schwarz2(L, S2, n2, n1, alpha, *it, d, nullptr, stream, &rep);
                }
                if (st != TVS_OK && st != TVS_ERR_NOT_CONVERGED) {
                    result = st;
                    goto out;
                }
                float ms = 0.0f;
                if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                    cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                    set_error_text("tvs_tune_schwarz2: event timing failed");
                    result = TVS_ERR_CUDA;
                    goto out;
                }
                if (st == TVS_OK && (best_t < 0.0f || ms < best_t)) {
                    best_t = ms;
                    best[0] = tiles[a];
                    best[1] = overlaps[b];
                    best[2] = ks[c];
                    result = TVS_OK;
                }
            }
        }
out:
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (best_ms) *best_ms = best_t;
    return result;
}

}  // extern "C"
