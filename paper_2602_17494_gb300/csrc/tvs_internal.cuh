// Internal declarations shared by the CUDA translation units of libtvs.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

#include "../../include/tvs.h"

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <utility>

namespace tvs {

// Programmatic dependent launch.  A kernel launched with launch_pdl may be
// scheduled while the previous kernel of the stream is still running (after
// every CTA of that kernel has called pdl_trigger or exited); it must call
// pdl_wait, which returns once the previous kernel has completed and its
// writes are visible, before any other statement.  Both are no-ops for a
// kernel launched the ordinary way.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

constexpr int kPitchAlign = 32;        // floats; internal planes start rows on 128-byte lines
constexpr int kFftThreads = 1024;      // upper bound on threads of the DCT kernels
constexpr int kSmemBudget = 200 * 1024;  // dynamic shared memory the DCT kernels may use

inline int round_up(int x, int m) { return (x + m - 1) / m * m; }
inline size_t round_up_sz(size_t x, size_t m) { return (x + m - 1) / m * m; }

// --------------------------------------------------------------------------
// Complex helpers
// --------------------------------------------------------------------------
// Sums and differences are one packed f32x2 instruction (each lane rounded
// to nearest, the same result as the two scalar operations).
__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.0f, -1.0f), a); }
__device__ __forceinline__ float2 c_mul(float2 a, float2 b) {
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 c_conj(float2 a) { return make_float2(a.x, -a.y); }

// Single-instruction hardware approximations (about 2 ulp; subnormals flushed
// to zero) of 1/sqrt(x) and 1/x.
__device__ __forceinline__ float rsqrt_ftz(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
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
    float2* bhat;   // FFT_M of the chirp filter times 1/M: natural order for M < 2048, else the
                    // digit-reversed order of the in-place passes, point 16 u + i at i M/16 + u
    float* sig2;    // sigma_{L,k}^2 = (2 sin(pi k / (2L)))^2, k < L: eigenvalues of the 1-D Neumann Laplacian
};

int fft_len_for(int L);
void carve_plan(Carver& cv, DctPlan& pl, int L);
cudaError_t build_plan(const DctPlan& pl, cudaStream_t s);

// Poisson / projection machinery on a rows x cols grid (pitch in floats).
//   s_to_phi: in place, S <- Delta^dagger S (Neumann, min-norm).
struct PoissonPlans {
    DctPlan row;         // length cols (x transforms)
    int rows = 0;        // y length; the y pass is a tridiagonal solve per column
    float4* tri = nullptr;  // its per-column coefficients, two float4 per column (tri_solve.cu)
    // Long columns (rows >= kTriChunkRows) are solved in chunks of 32 rows
    // with coalesced row accesses (tri_solve.cu); tsum holds the per-chunk
    // summaries and carries (tri_chunk_floats(rows, cols) floats), tnch the
    // number of chunks.  nullptr / 0 for short columns.
    float* tsum = nullptr;
    int tnch = 0;
};
constexpr int kTriChunk = 32;          // rows per chunk of the chunked column solve
constexpr int kTriChunkRows = 1537;    // shortest column solved in chunks
inline int tri_chunks(int rows) { return (rows + kTriChunk - 1) / kTriChunk; }
// five [chunk][column] planes, the k_x = 0 column's weighted sums [chunk] and two scalars
inline size_t tri_chunk_floats(int rows, int cols) {
    const size_t n = (size_t)tri_chunks(rows);
    return 5 * n * (size_t)cols + n + 2;
}
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
constexpr int kFinCTAs = 128;   // CTAs of the first pass of finalize_red
struct RedBuf {
    double* partial;   // [nblocks][kRedSlots]
    double* stage;     // [kFinCTAs][kRedSlots]: the first pass of finalize_red
    double* result;    // [kRedSlots]
    unsigned* err;     // bit 0: a bounded device-side wait gave up
    int cap;           // capacity in blocks
};
void carve_red(Carver& cv, RedBuf& rb, int cap);
// slots: 0 sum|psi|, 1 sum psi.p, 2 sum z^2, 3 sum (z+f)^2, 4 max|p|, 5 max|div z|
cudaError_t finalize_red(const RedBuf& rb, int nblocks, cudaStream_t s);

// Block-level reduction of kRedSlots doubles: slots 0..3 summed, 4..5 max'ed,
// 6..7 summed.  NT = threads of the block, tid = linear thread index.  The
// result lands in out[0..kRedSlots) (written by threads 0..kRedSlots-1).
__device__ __forceinline__ bool red_is_max(int k) { return k == 4 || k == 5; }

// An FP32 value with its rounding error carried separately (hi + lo); ff_add
// is the error-free two-sum followed by a renormalisation.
struct FF {
    float hi, lo;
};
__device__ __forceinline__ FF ff_add(FF a, FF b) {
    const float s = a.hi + b.hi;
    const float bb = s - a.hi;
    const float e = (a.hi - (s - bb)) + (b.hi - bb);
    const float lo = e + (a.lo + b.lo);
    const float h = s + lo;
    return FF{h, lo - (h - s)};
}

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
    __device__ __forceinline__ FF pair() const { return FF{s, -c}; }
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

// The same block reduction with the sums carried as unevaluated pairs of
// FP32 values (hi + lo, combined with the error-free two-sum), so the
// per-block partial keeps about 44 significant bits without FP64 arithmetic
// per thread; each block writes its kRedSlots values as doubles.  v[k] =
// (hi, lo) of slot k; max slots use hi only.  Deterministic: fixed shuffle
// pattern and warp order.
template <int NT>
__device__ __forceinline__ void block_reduce_store_ff(FF v[kRedSlots], double* out, int tid) {
    __shared__ FF red_ff[NT / 32][kRedSlots];
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) {
        FF x = v[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const FF y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
            x = red_is_max(k) ? FF{fmaxf(x.hi, y.hi), 0.0f} : ff_add(x, y);
        }
        if (lane == 0) red_ff[wid][k] = x;
    }
    __syncthreads();
    if (tid < kRedSlots) {
        const int k = tid;
        FF x = red_ff[0][k];
        for (int w = 1; w < NT / 32; ++w) x = red_is_max(k) ? FF{fmaxf(x.hi, red_ff[w][k].hi), 0.0f} : ff_add(x, red_ff[w][k]);
        out[k] = (double)x.hi + (double)x.lo;
    }
}

// The TFS check layout of block_reduce_store_ff with only its live slots
// reduced: the four sums (slots 0-3) as FP32 pairs, the two maxima (slots 4,
// 5) as plain FP32, slots 6 and 7 written as zero.  Same results as
// block_reduce_store_ff on that layout, at about half the shuffles and adds
// (which matter: a 32 x 32 tile's reduction costs a third of its update).
template <int NT>
__device__ __forceinline__ void block_reduce_store_tfs(const float (&sum)[4], float mx4, float mx5, double* out,
                                                       int tid) {
    __shared__ FF red_s[NT / 32][4];
    __shared__ float red_m[NT / 32][2];
    const int lane = tid & 31, wid = tid >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        FF x{sum[k], 0.0f};
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const FF y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
            x = ff_add(x, y);
        }
        if (lane == 0) red_s[wid][k] = x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx4 = fmaxf(mx4, __shfl_xor_sync(0xffffffffu, mx4, o));
        mx5 = fmaxf(mx5, __shfl_xor_sync(0xffffffffu, mx5, o));
    }
    if (lane == 0) {
        red_m[wid][0] = mx4;
        red_m[wid][1] = mx5;
    }
    __syncthreads();
    if (tid < kRedSlots) {
        const int k = tid;
        double v = 0.0;
        if (k < 4) {
            FF x = red_s[0][k];
            for (int w = 1; w < NT / 32; ++w) x = ff_add(x, red_s[w][k]);
            v = (double)x.hi + (double)x.lo;
        } else if (k < 6) {
            float m = red_m[0][k - 4];
            for (int w = 1; w < NT / 32; ++w) m = fmaxf(m, red_m[w][k - 4]);
            v = (double)m;
        }
        out[k] = v;
    }
}

// --------------------------------------------------------------------------
// Error bookkeeping
// --------------------------------------------------------------------------
void set_error(const char* what, cudaError_t e);
void set_error_text(const char* msg);


// ---------------------------------------------------------------------------
// Storage formats of the dual fields: values live in HBM as float, bf16,
// fp16 or 16-bit fixed point on [-1, 1] and are widened to float for all
// arithmetic.  16-bit stores round stochastically: the value rounds up with
// probability equal to the discarded fraction, so updates smaller than one
// unit in the last place are kept in expectation instead of being lost (with
// round-to-nearest the iteration stalls at a duality gap of 1e-3 (fp16) or
// 1e-2 (bf16)).  The random bits come from a counter-based hash of (update
// seed, element index, plane), so runs are reproducible bit for bit.
// ld* go through the read-only path; ld*c are plain loads for data the same
// kernel also writes.
// ---------------------------------------------------------------------------

// lowbias32 integer hash (C. Wellons, "Prospecting for hash functions", 2018).
__host__ __device__ __forceinline__ uint32_t hash32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352dU;
    x ^= x >> 15;
    x *= 0x846ca68bU;
    x ^= x >> 16;
    return x;
}
// Random bits for the element at index o of plane pl in update `seed`: one
// hash of a counter built from the three (a 16-bit store uses 16 of them, a
// 4-wide store 8 per element).
__device__ __forceinline__ uint32_t rkey(uint32_t seed, size_t o, int pl) {
    return hash32((uint32_t)o * 0x9e3779b1U + seed * 0x85ebca77U + (uint32_t)pl * 0xc2b2ae3dU);
}

// Stochastic rounding from float; r is `bits` random bits (8 or 16) and the
// remaining discarded bits are dithered at their midpoint.
template <int BITS>
__device__ __forceinline__ __nv_bfloat16 bf16_sr(float x, uint32_t r) {
    uint32_t b = __float_as_uint(x);
    if ((b & 0x7f800000U) == 0x7f800000U) return __float2bfloat16_rn(x);
    b += (r << (16 - BITS)) + ((1u << (16 - BITS)) >> 1);   // a carry rounds the magnitude up
    return __ushort_as_bfloat16((unsigned short)(b >> 16));
}
template <int BITS>
__device__ __forceinline__ __half f16_sr(float x, uint32_t r) {
    const float ax = fabsf(x);
    if (!(ax >= 6.103515625e-05f && ax < 32768.0f)) return __float2half_rn(x);   // outside the normal range
    const uint32_t add = BITS >= 13 ? (r & 0x1fffU) : ((r << (13 - BITS)) + ((1u << (13 - BITS)) >> 1));
    const uint32_t b = (__float_as_uint(x) + add) & ~0x1fffU;                    // 10 mantissa bits remain
    return __float2half_rz(__uint_as_float(b));
}
constexpr float kS16Scale = 32767.0f;   // fixed point: value = code / 32767, |code| <= 32767
// code = floor(x S + u), u = (r + 1/2) / 2^BITS, clamped to |code| <= S (the
// bounds are integers, so clamping before the round-down conversion is the same)
__device__ __forceinline__ int16_t s16_from_dithered(float x, float u) {
    const float y = fmaf(x, kS16Scale, u);
    return (int16_t)__float2int_rd(fminf(fmaxf(y, -kS16Scale), kS16Scale));
}
template <int BITS>
__device__ __forceinline__ int16_t s16_sr(float x, uint32_t r) {
    return s16_from_dithered(x, ((float)r + 0.5f) * (1.0f / (float)(1u << BITS)));
}
// The same with the 8 random bits taken from byte E of k: the byte goes into
// the mantissa of 1.0f (bits 8..15, one byte permute), f = 1 + b / 2^15, and
// u = 128 f - 128 + 2^-9 = (b + 1/2) / 256 exactly.
template <int E>
__device__ __forceinline__ int16_t s16_sr_byte(float x, uint32_t k) {
    const float f = __uint_as_float(__byte_perm(k, 0x3F800000u, 0x7604u | (E << 4)));
    return s16_from_dithered(x, fmaf(f, 128.0f, -128.0f + 1.0f / 512.0f));
}

template <class S>
struct Stor;
template <>
struct Stor<float> {
    static __device__ __forceinline__ float4 ld4(const float* p) { return __ldg(reinterpret_cast<const float4*>(p)); }
    static __device__ __forceinline__ float4 ld4c(const float* p) { return *reinterpret_cast<const float4*>(p); }
    // L2-coherent loads (ld.global.cg) for data other CTAs of the same launch write
    static __device__ __forceinline__ float4 ld4g(const float* p) { return __ldcg(reinterpret_cast<const float4*>(p)); }
    static __device__ __forceinline__ float ld1g(const float* p) { return __ldcg(p); }
    static __device__ __forceinline__ float ld1(const float* p) { return __ldg(p); }
    static __device__ __forceinline__ float ld1c(const float* p) { return *p; }
    static __device__ __forceinline__ void st4(float* p, float4 v, uint32_t) { *reinterpret_cast<float4*>(p) = v; }
    static __device__ __forceinline__ void st1(float* p, float v, uint32_t) { *p = v; }
    static __device__ __forceinline__ void st1r8(float* p, float v, uint32_t) { *p = v; }
};

// Shared code of the 16-bit formats: D supplies to_f(uint16) and from_f<BITS>(float, random bits).
template <class T, class D>
struct Stor16 {
    static __device__ __forceinline__ float4 unpack(uint2 u) {
        return make_float4(D::to_f((uint16_t)(u.x & 0xffffU)), D::to_f((uint16_t)(u.x >> 16)),
                           D::to_f((uint16_t)(u.y & 0xffffU)), D::to_f((uint16_t)(u.y >> 16)));
    }
    static __device__ __forceinline__ float4 ld4(const T* p) { return unpack(__ldg(reinterpret_cast<const uint2*>(p))); }
    static __device__ __forceinline__ float4 ld4c(const T* p) { return unpack(*reinterpret_cast<const uint2*>(p)); }
    static __device__ __forceinline__ float ld1(const T* p) {
        return D::to_f(__ldg(reinterpret_cast<const unsigned short*>(p)));
    }
    static __device__ __forceinline__ float ld1c(const T* p) { return D::to_f(*reinterpret_cast<const uint16_t*>(p)); }
    static __device__ __forceinline__ float4 ld4g(const T* p) { return unpack(__ldcg(reinterpret_cast<const uint2*>(p))); }
    static __device__ __forceinline__ float ld1g(const T* p) {
        return D::to_f(__ldcg(reinterpret_cast<const unsigned short*>(p)));
    }
    static __device__ __forceinline__ void st4(T* p, float4 v, uint32_t k) {
        uint2 u;
        u.x = (uint32_t)D::template from_f_byte<0>(v.x, k) | ((uint32_t)D::template from_f_byte<1>(v.y, k) << 16);
        u.y = (uint32_t)D::template from_f_byte<2>(v.z, k) | ((uint32_t)D::template from_f_byte<3>(v.w, k) << 16);
        *reinterpret_cast<uint2*>(p) = u;
    }
    static __device__ __forceinline__ void st1(T* p, float v, uint32_t k) {
        *reinterpret_cast<uint16_t*>(p) = D::template from_f<16>(v, k & 0xffffU);
    }
    // one element with 8 random bits (r8 < 256), for stores that share one hash
    static __device__ __forceinline__ void st1r8(T* p, float v, uint32_t r8) {
        *reinterpret_cast<uint16_t*>(p) = D::template from_f<8>(v, r8);
    }
};
// from_f_byte<E>(x, k): from_f<8> with the random bits of byte E of k
struct Bf16Bits {
    static __device__ __forceinline__ float to_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }
    template <int BITS>
    static __device__ __forceinline__ uint16_t from_f(float x, uint32_t r) {
        return __bfloat16_as_ushort(bf16_sr<BITS>(x, r));
    }
    template <int E>
    static __device__ __forceinline__ uint16_t from_f_byte(float x, uint32_t k) {
        return from_f<8>(x, (k >> (8 * E)) & 0xffU);
    }
};
struct F16Bits {
    static __device__ __forceinline__ float to_f(uint16_t b) { return __half2float(__ushort_as_half(b)); }
    template <int BITS>
    static __device__ __forceinline__ uint16_t from_f(float x, uint32_t r) { return __half_as_ushort(f16_sr<BITS>(x, r)); }
    template <int E>
    static __device__ __forceinline__ uint16_t from_f_byte(float x, uint32_t k) {
        return from_f<8>(x, (k >> (8 * E)) & 0xffU);
    }
};
struct S16Bits {
    static __device__ __forceinline__ float to_f(uint16_t b) { return (float)(int16_t)b * (1.0f / kS16Scale); }
    template <int BITS>
    static __device__ __forceinline__ uint16_t from_f(float x, uint32_t r) { return (uint16_t)s16_sr<BITS>(x, r); }
    template <int E>
    static __device__ __forceinline__ uint16_t from_f_byte(float x, uint32_t k) { return (uint16_t)s16_sr_byte<E>(x, k); }
};
template <>
struct Stor<__nv_bfloat16> : Stor16<__nv_bfloat16, Bf16Bits> {};
template <>
struct Stor<__half> : Stor16<__half, F16Bits> {};
template <>
struct Stor<int16_t> : Stor16<int16_t, S16Bits> {};

// Bytes per element of a tvs_storage value (0 if unknown).
inline size_t storage_bytes(int storage) {
    return storage == TVS_F32 ? 4 : (storage == TVS_BF16 || storage == TVS_F16 || storage == TVS_S16) ? 2 : 0;
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
        case TVS_S16: {                      \
            using S = int16_t;               \
            __VA_ARGS__;                     \
        } break;                             \
        default: {                           \
            using S = float;                 \
            __VA_ARGS__;                     \
        } break;                             \
    }


}  // namespace tvs
