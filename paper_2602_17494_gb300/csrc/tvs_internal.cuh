// Internal declarations shared by the CUDA translation units of libtvs.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/tvs.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

namespace tvs {

constexpr int kPitchAlign = 32;        // floats; internal planes start rows on 128-byte lines
constexpr int kFftThreads = 1024;      // upper bound on threads of the DCT kernels
constexpr int kSmemBudget = 200 * 1024;  // dynamic shared memory the DCT kernels may use

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline size_t round_up_sz(size_t x, size_t m) { return (x + m - 1) / m * m; }

// --------------------------------------------------------------------------
// Complex helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }
__device__ __forceinline__ float2 c_mulconj(float2 a, float2 b) {  // a * conj(b)
    return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// --------------------------------------------------------------------------
// Workspace carving: every call lays its scratch out in the caller's buffer.
// --------------------------------------------------------------------------
struct Carver {
    char* base;
    size_t off;
    explicit Carver(void* b) : base(static_cast<char*>(b)), off(0) {}
    template <class T>
    T* take(size_t count) {
        off = round_up_sz(off, 256);
        T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
        off += count * sizeof(T);
        return p;
    }
    size_t used() const { return round_up_sz(off, 256); }
};

// A scalar field on rows x cols points stored with a padded row pitch.
struct Plane {
    float* ptr;
    int rows, cols, pitch;
};

// --------------------------------------------------------------------------
// DCT plan for one transform length L (Makhoul's reordering + Bluestein's
// chirp-z transform with one input sample peeled off, see dct.cu).
// --------------------------------------------------------------------------
struct DctPlan {
    int L;          // transform length
    int M;          // power-of-two FFT length, M >= 2L-2
    int logM;
    float2* chirp;  // c_n = exp(-i pi n^2 / L), n < L
    float2* rot;    // exp(+2 pi i k / L), k < L (the peeled sample's phase)
    float2* post;   // exp(-i pi k / (2L)), k < L (Makhoul's post-twiddle)
    float2* tw;     // exp(-2 pi i j / M), j < M/2
    float2* bhat;   // FFT_M of the chirp filter, bit-reversed order, times 1/M
};

int fft_len_for(int L);
void carve_plan(Carver& cv, DctPlan& pl, int L);
cudaError_t build_plan(const DctPlan& pl, cudaStream_t s);

// Poisson / projection machinery on a rows x cols grid (pitch in floats).
//   s_to_phi: in place, S <- Delta^dagger S (Neumann, min-norm).
struct PoissonPlans {
    DctPlan row;   // length cols (x transforms)
    DctPlan col;   // length rows (y transforms)
};
void carve_poisson(Carver& cv, PoissonPlans& pp, int rows, int cols);
cudaError_t build_poisson(const PoissonPlans& pp, cudaStream_t s);

// Source functors for the fused forward row transform.
enum class RowSource : int {
    Plain = 0,       // x = S[r][c]
    DivField = 1,    // x = div(u) for a 2-plane vector field u
    DivVecdiv = 2    // x = div(vecdiv p) for the 4-plane step-1 dual p
};
struct RowSrcArgs {
    const float* a;  // plane base (Plain: S; DivField: u; DivVecdiv: p)
    long plane;      // plane stride in floats
    int pitch;
};
cudaError_t poisson_solve(float* S, int rows, int cols, int pitch, const PoissonPlans& pp,
                          RowSource src, const RowSrcArgs& sa, cudaStream_t s);
// nbatch independent rows x cols problems; problem b's source is zero outside
// rows [ranges[b].x, ranges[b].y) and only those rows are stored, packed, at
// S + b * bstride (storage row 0 = grid row ranges[b].x).  Only those rows of
// Delta^dagger of the source are produced (in place).  maxrows bounds
// ranges[b].y - ranges[b].x; ranges is a device array.
cudaError_t poisson_solve_batched(float* S, int nbatch, long bstride, const int2* ranges, int maxrows, int rows,
                                  int cols, int pitch, const PoissonPlans& pp, cudaStream_t s);

// --------------------------------------------------------------------------
// Reductions for the gap / energy checks (FP64, deterministic two-pass).
// --------------------------------------------------------------------------
// Reduction slots: 0 sum |psi|, 1 sum (|psi| - psi . p) (the duality gap
// terms, each >= 0 while |p| <= 1), 2 sum z^2, 3 sum (z + f)^2, 4 max |p|,
// 5 max |div z|; 6, 7 unused.
constexpr int kRedSlots = 8;
struct RedBuf {
    double* partial;   // [nblocks][kRedSlots]
    double* result;    // [kRedSlots]
    int cap;           // capacity in blocks
};
void carve_red(Carver& cv, RedBuf& rb, int cap);
// slots: 0 sum|psi|, 1 sum psi.p, 2 sum z^2, 3 sum (z+f)^2, 4 max|p|, 5 max|div z|
cudaError_t finalize_red(const RedBuf& rb, int nblocks, cudaStream_t s);

// Block-level reduction of kRedSlots doubles: slots 0..3 summed, 4..5 max'ed,
// 6..7 summed.  NT = threads of the block, tid = linear thread index.  The
// result lands in out[0..kRedSlots) (written by threads 0..kRedSlots-1).
__device__ __forceinline__ bool red_is_max(int k) { return k == 4 || k == 5; }

// Per-thread compensated (Kahan) FP32 sum: the check kernels add FP32
// per-pixel terms here and hand the total to FP64 for the cross-thread
// reduction, so no FP64 arithmetic runs per pixel.
struct KSum {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float x) {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

template <int NT>
__device__ __forceinline__ void block_reduce_store(double v[kRedSlots], double* out, int tid) {
    __shared__ double red_sm[NT / 32][kRedSlots];
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) {
        double x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const double y = __shfl_xor_sync(0xffffffffu, x, o);
            x = red_is_max(k) ? fmax(x, y) : x + y;
        }
        if (lane == 0) red_sm[wid][k] = x;
    }
    __syncthreads();
    if (tid < kRedSlots) {
        const int k = tid;
        double x = red_sm[0][k];
        for (int w = 1; w < NT / 32; ++w) x = red_is_max(k) ? fmax(x, red_sm[w][k]) : x + red_sm[w][k];
        out[k] = x;
    }
}

// --------------------------------------------------------------------------
// Error bookkeeping
// --------------------------------------------------------------------------
void set_error(const char* what, cudaError_t e);
void set_error_text(const char* msg);


// ---------------------------------------------------------------------------
// Storage formats of the dual fields: values live in HBM as float, bf16 or
// fp16 and are widened to float for all arithmetic; stores round to nearest.
// ld* go through the read-only path; ld*c are plain loads for data the same
// kernel also writes.
// ---------------------------------------------------------------------------
template <class S>
struct Stor;
template <>
struct Stor<float> {
    static __device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
    static __device__ __forceinline__ float4 ld4c(const float* p) { return *reinterpret_cast<const float4*>(p); }
    static __device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float ld1c(const float* p) { return *p; }
    static __device__ __forceinline__ void st4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
    static __device__ __forceinline__ void st1(float* p, float v) { *p = v; }
};
template <>
struct Stor<__nv_bfloat16> {
    using T = __nv_bfloat16;
    static __device__ __forceinline__ float4 ld4(const T* p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        __nv_bfloat162 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ float ld1(const T* p) { return __bfloat162float(p[0]); }
    static __device__ __forceinline__ float ld1c(const T* p) { return __bfloat162float(p[0]); }
    static __device__ __forceinline__ float4 ld4c(const T* p) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        __nv_bfloat162 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ void st4(T* p, float4 v) {
        const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y), b = __floats2bfloat162_rn(v.z, v.w);
        uint2 u;
        memcpy(&u.x, &a, 4);
        memcpy(&u.y, &b, 4);
        *reinterpret_cast<uint2*>(p) = u;
    }
    static __device__ __forceinline__ void st1(T* p, float v) { p[0] = __float2bfloat16_rn(v); }
};
template <>
struct Stor<__half> {
    using T = __half;
    static __device__ __forceinline__ float4 ld4(const T* p) {
        const uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
        __half2 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ float ld1(const T* p) { return __half2float(p[0]); }
    static __device__ __forceinline__ float ld1c(const T* p) { return __half2float(p[0]); }
    static __device__ __forceinline__ float4 ld4c(const T* p) {
        const uint2 u = *reinterpret_cast<const uint2*>(p);
        __half2 a, b;
        memcpy(&a, &u.x, 4);
        memcpy(&b, &u.y, 4);
        const float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    static __device__ __forceinline__ void st4(T* p, float4 v) {
        const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, v.w);
        uint2 u;
        memcpy(&u.x, &a, 4);
        memcpy(&u.y, &b, 4);
        *reinterpret_cast<uint2*>(p) = u;
    }
    static __device__ __forceinline__ void st1(T* p, float v) { p[0] = __float2half_rn(v); }
};

// Bytes per element of a tvs_storage value (0 if unknown).
inline size_t storage_bytes(int storage) {
    return storage == TVS_F32 ? 4 : (storage == TVS_BF16 || storage == TVS_F16) ? 2 : 0;
}

// Runs the statement (the variadic arguments) with the type S for the
// runtime storage value v.
#define TVS_STORAGE_SWITCH(v, ...)           \
    switch (v) {                             \
        case TVS_BF16: {                     \
            using S = __nv_bfloat16;         \
            __VA_ARGS__;                     \
        } break;                             \
        case TVS_F16: {                      \
            using S = __half;                \
            __VA_ARGS__;                     \
        } break;                             \
        default: {                           \
            using S = float;                 \
            __VA_ARGS__;                     \
        } break;                             \
    }


}  // namespace tvs
