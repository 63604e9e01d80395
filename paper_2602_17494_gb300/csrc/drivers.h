// Workspace layouts and host-side helpers shared by the C ABI (api.cu) and
// the batching engine (engine.cu).
#pragma once

#include "tvs_internal.cuh"
#include "launchers.h"

namespace tvs {

constexpr int kMaxSide = 8192;   // transform length <= 8193 keeps one FFT line in shared memory

#define TVS_CUDA(call)                                       \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) {                             \
            set_error(#call, e_);                            \
            return TVS_ERR_CUDA;                             \
        }                                                    \
    } while (0)

// ---------------------------------------------------------------------------
// Workspace layouts
// ---------------------------------------------------------------------------
struct Step1Layout {
    int R, C, P;
    long plane;
    int st = TVS_F32;   // tvs_storage of the dual p (pa, pb; 4 planes each)
    PoissonPlans pp;
    float *pa, *pb, *f1, *S;
    float* src = nullptr;   // div(vecdiv p) of the current dual (the global loop's Poisson source)
    RedBuf red;
};


struct Step2Layout {
    int R, C, P;
    long plane;
    int st;            // tvs_storage of the dual p (pa, pb)
    void *pa, *pb;
    float* f2;
    RedBuf red;
};

struct ProjLayout {
    int P;
    long plane;
    PoissonPlans pp;
    float *u, *S;
};

size_t layout_step1(Carver& cv, int n2, int n1, Step1Layout& L, int storage = TVS_F32);
size_t layout_step2(Carver& cv, int n2, int n1, Step2Layout& L, int storage);
size_t layout_project(Carver& cv, int rows, int cols, ProjLayout& L);
bool side_ok(int n);
tvs_status check_iter(const tvs_iter* it, bool narrow_ok);
tvs_status check_ws(void* ws, size_t ws_bytes, size_t need);
// finalize the block partials of rb, copy them to the host (synchronizes s)
tvs_status read_result(const RedBuf& rb, int nblocks, cudaStream_t s, double out[kRedSlots]);
void report_tfs(const double r[kRedSlots], double delta, int iters, tvs_report* rep);
void report_irv1(const double r[kRedSlots], double alpha, int iters, tvs_report* rep);
cudaError_t to_pitched(float* dst, int dpitch, const float* src, int rows, int cols, int planes, cudaStream_t s);
cudaError_t from_pitched(float* dst, const float* src, int spitch, int rows, int cols, int planes, cudaStream_t s);
cudaError_t p2_in(const Step2Layout& L, const float* src, cudaStream_t s);
cudaError_t p2_out(const Step2Layout& L, float* dst, const void* cur, cudaStream_t s);
cudaError_t p2_zero(const Step2Layout& L, cudaStream_t s);
// f1 = P_K tau0 / delta into L.f1 (L.S as scratch); clears the error word
tvs_status tfs_setup(const Step1Layout& L, const float* d0, int n2, int n1, double delta, cudaStream_t s);

// Algorithm 2 with Algorithm 3 for step 2 from p_user (or zero), f2 already in L.f2.
tvs_status run_schwarz2(const Step2Layout& L, Schwarz2State& S2, int n2, int n1, double alpha, const tvs_iter& it,
                        float* d, float* p_user, cudaStream_t s, tvs_report* rep);

// quality.cu: workspace of tvs_quality
size_t quality_layout(Carver& cv, RedBuf& rb);

}  // namespace tvs
