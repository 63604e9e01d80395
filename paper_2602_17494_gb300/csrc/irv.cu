// Step 2, image reconstruction IRV1 (Section 4.2, eq. ir1dualdis):
//   xi = tau_perp / sqrt(|tau_perp|^2 + eps), tau_perp = R_Omega(tau_2, -tau_1)
//   f2 = alpha d0 - div xi
//   Chambolle: z = div p - f2, psi = grad z, p <- (p + t psi) / (1 + t |psi|)
//   d = (f2 - div p) / alpha = -z / alpha
//
// The backward difference D^-_x of Section 4.1 equals the plain difference of
// the field with its last column (and everything left of the grid) read as
// zero; D^-_y likewise with the last row.  The kernels below read the dual with
// exactly those zeros, so one stencil covers the interior and the boundary.
#include "tvs_internal.cuh"
#include "prof.h"
#include "tma.cuh"

#include <mutex>
#include <type_traits>

namespace tvs {

// ---------------------------------------------------------------------------
// xi and f2 (eq. defXi2:discrete, eq. ir1dualdis)
// ---------------------------------------------------------------------------
// tau is stored as TT (float, or a 16-bit float type for tau kept inside the library)
template <class TT = float>
__device__ __forceinline__ float2 xi_at(const TT* __restrict__ tau, long tplane, int tpitch,
                                        int i, int j, float eps) {
    const float tp1 = Stor<TT>::ld1(&tau[tplane + (size_t)i * tpitch + j]);    // tau_2
    const float tp2 = -Stor<TT>::ld1(&tau[(size_t)i * tpitch + j]);            // -tau_1
    const float den = sqrtf(tp1 * tp1 + tp2 * tp2 + eps);
    return make_float2(tp1 / den, tp2 / den);
}

template <class TT>
__global__ void xi_f2_kernel(const float* __restrict__ d0, int d0_pitch, const TT* __restrict__ tau,
                             long tplane, int tpitch, int R, int C, float alpha, float eps,
                             float* __restrict__ f2, int fpitch) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= R || j >= C) return;
    // div xi on the image grid with the zero-extension rule of D^-
    const float x_c = (j <= C - 2) ? xi_at(tau, tplane, tpitch, i, j, eps).x : 0.f;
    const float x_l = (j >= 1 && j - 1 <= C - 2) ? xi_at(tau, tplane, tpitch, i, j - 1, eps).x : 0.f;
    const float y_c = (i <= R - 2) ? xi_at(tau, tplane, tpitch, i, j, eps).y : 0.f;
    const float y_u = (i >= 1 && i - 1 <= R - 2) ? xi_at(tau, tplane, tpitch, i - 1, j, eps).y : 0.f;
    const float divxi = (x_c - x_l) + (y_c - y_u);
    f2[(size_t)i * fpitch + j] = alpha * __ldg(&d0[(size_t)i * d0_pitch + j]) - divxi;
}

cudaError_t launch_xi_f2_st(const float* d0, int d0_pitch, const void* tau, int tau_storage, long tplane,
                            int tpitch, int R, int C, float alpha, float eps, float* f2, int fpitch, cudaStream_t s) {
    dim3 blk(32, 8), grd((C + 31) / 32, (R + 7) / 8);
    ProfScope ps(kProfSetup, s);
    if (tau_storage == TVS_F16)
        xi_f2_kernel<__half><<<grd, blk, 0, s>>>(d0, d0_pitch, static_cast<const __half*>(tau), tplane, tpitch, R,
                                                 C, alpha, eps, f2, fpitch);
    else if (tau_storage == TVS_BF16)
        xi_f2_kernel<__nv_bfloat16><<<grd, blk, 0, s>>>(d0, d0_pitch, static_cast<const __nv_bfloat16*>(tau),
                                                        tplane, tpitch, R, C, alpha, eps, f2, fpitch);
    else if (tau_storage == TVS_F32)
        xi_f2_kernel<float><<<grd, blk, 0, s>>>(d0, d0_pitch, static_cast<const float*>(tau), tplane, tpitch, R, C,
                                                alpha, eps, f2, fpitch);
    else
        return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_xi_f2(const float* d0, int d0_pitch, const float* tau, long tplane, int tpitch,
                         int R, int C, float alpha, float eps, float* f2, int fpitch, cudaStream_t s) {
    return launch_xi_f2_st(d0, d0_pitch, tau, TVS_F32, tplane, tpitch, R, C, alpha, eps, f2, fpitch, s);
}

// ---------------------------------------------------------------------------
// Streaming IRV1 update: each warp owns a strip of 128 columns (4 per lane)
// and walks down a chunk of rows, keeping the previous row's dual and
// residual in registers.  Rows arrive through TMA: lane 0 keeps kStages row
// loads in flight per warp (p as one 3-D box covering both planes, f2 as a
// 2-D box), each box spanning the strip plus 16 bytes of halo on either side;
// reads outside the grid come back as zeros, which is the zero extension of
// D^- at the left edge.  Left/right neighbours of the computed residual come
// from warp shuffles.  No block-level barriers; HBM traffic is the 20 (FP32)
// or 12 (16-bit) algorithmic bytes per pixel plus the halo columns and one
// extra row per chunk.
//   CHECK  : per-warp partial sums of the gap/energy terms at the input p
//   WRITE_P: write the updated dual
//   WRITE_D: write d = -z / alpha at the input p
// ---------------------------------------------------------------------------
constexpr int kStrip = 128;      // columns per warp
constexpr int kChunk = 32;       // output rows per warp
constexpr int kStreamWarps = 4;  // warps per block
constexpr int kRows = 2;         // rows per TMA load (item)
constexpr int kStages = 2;       // items in flight per warp

template <class S>
struct StreamGeom {
    static constexpr int HP = 16 / (int)sizeof(S);                  // halo columns of the p box
    static constexpr int WP = kStrip + 2 * HP;                      // p box width (elements)
    static constexpr int HF = 4, WF = kStrip + 8;                   // f2 box (float)
    static constexpr int PBYTES = 2 * kRows * WP * (int)sizeof(S);  // [plane][row][WP]
    static constexpr int FBYTES = kRows * WF * 4;                   // [row][WF]
    static constexpr int POFF = 0;
    static constexpr int FOFF = (PBYTES + 127) / 128 * 128;
    static constexpr int STAGE = FOFF + (FBYTES + 127) / 128 * 128;
    static constexpr int WARP_BYTES = kStages * STAGE;
};
template <class S>
constexpr size_t stream_smem_bytes() {
    return (size_t)kStreamWarps * StreamGeom<S>::WARP_BYTES + (size_t)kStreamWarps * kStages * sizeof(uint64_t) + 128;
}

__device__ __forceinline__ float comp(const float4& v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}
// sqrt(a^2 + b^2) through the hardware reciprocal square root (about 2 ulp);
// the 1e-30 keeps rsqrt finite at 0 and is below the resolution of any
// nonzero a^2 + b^2 that matters here.
__device__ __forceinline__ float fast_norm(float a, float b) {
    const float s2 = fmaf(a, a, fmaf(b, b, 1e-30f));
    return s2 * rsqrtf(s2);
}
// Two-lane FP32 arithmetic on pixel pairs (one instruction for two pixels,
// each lane rounded exactly like the scalar operation).
__device__ __forceinline__ float2 p_sub(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 p_add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 p_mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 p_fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// 4 consecutive elements of a box row in shared memory, widened to float
template <class S>
__device__ __forceinline__ float4 sm_ld4(const S* p) {
    if constexpr (sizeof(S) == 4) return *reinterpret_cast<const float4*>(p);
    else return Stor<S>::ld4c(p);
}
template <class S>
__device__ __forceinline__ float sm_ld1(const S* p) {
    if constexpr (sizeof(S) == 4) return *reinterpret_cast<const float*>(p);
    else return Stor<S>::ld1c(p);
}

template <class S, bool CHECK, bool WRITE_P, bool WRITE_D>
__global__ void __launch_bounds__(32 * kStreamWarps, CHECK ? 5 : 8)
irv1_stream_kernel(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap fmap,
                   const S* __restrict__ pin, S* __restrict__ pout, int R, int C, int pitch, long plane, float t,
                   float alpha_inv, float* __restrict__ d_out, int d_pitch, double* __restrict__ partial,
                   uint32_t seed, unsigned* __restrict__ err) {
    pdl_wait();
    pdl_trigger();
    using G = StreamGeom<S>;
    using St = Stor<S>;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    // TMA destinations are kept 128-byte aligned; offsetting the array (not an
    // integer copy of its address) keeps the accesses in the shared space
    unsigned char* smem_raw = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int strip = blockIdx.x;
    const int chunk = blockIdx.y * kStreamWarps + wib;
    const int r0 = chunk * kChunk;
    const int x0 = strip * kStrip;                // first column of the strip
    const int j0 = x0 + 4 * lane;                 // first column of this lane
    const int r1 = min(r0 + kChunk, R);           // output rows [r0, r1)
    unsigned char* wbase = smem_raw + (size_t)wib * G::WARP_BYTES;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + (size_t)kStreamWarps * G::WARP_BYTES) + wib * kStages;
    KSum ks[4];
    float pmax = 0.0f;
    (void)pin;

    if (r0 < R) {
        // Rows r0 - 1 .. r1 are visited in order (row r0 - 1 only for p_y above
        // the first row, row r1 only for z below the last); item k holds rows
        // r0 - 1 + kRows k + h.  Rows at or past R arrive as zeros.
        const int rend = min(r1 + 1, R);         // rows whose z is needed
        const int nitems = (r1 - r0 + 2 + kRows - 1) / kRows;
        if (lane == 0) {
            for (int s = 0; s < kStages; ++s) mbar_init(&bars[s], 1);
            mbar_init_fence();
        }
        __syncwarp();
        auto issue = [&](int k) {                 // lane 0 only
            const int s = k % kStages;
            unsigned char* st = wbase + s * G::STAGE;
            const int row = r0 - 1 + kRows * k;
            mbar_expect_tx(&bars[s], (uint32_t)(G::PBYTES + G::FBYTES));
            tma_load_3d(st + G::POFF, &pmap, x0 - G::HP, row, 0, &bars[s]);
            tma_load_2d(st + G::FOFF, &fmap, x0 - G::HF, row, &bars[s]);
        };
        if (lane == 0)
            for (int k = 0; k < kStages && k < nitems; ++k) issue(k);
        int issued = min(kStages, nitems);       // items whose load has been issued (same on every lane)
        int failed = -1;                          // item whose wait gave up

        // Only the strip holding column C - 1 needs column masks (D^- reads p_x
        // as zero there; D^+ is zero across it); columns left of 0 and right of
        // C - 1 arrive as zeros.  z beyond the grid is never used.
        const bool edge_col = x0 + kStrip > C - 1;     // warp-uniform
        const int jr = x0 + kStrip;               // first column right of the strip
        float4 pyu = make_float4(0.f, 0.f, 0.f, 0.f);   // p_y of the row above (masked)
        float pyu_r = 0.f;                        // p_y(row above, jr) on lane 31
        float zp[4] = {0.f, 0.f, 0.f, 0.f};       // z of the previous row
        float zpr = 0.f;                          // z(prev row, jr) on lane 31
        float4 pprevx = make_float4(0.f, 0.f, 0.f, 0.f), pprevy = pprevx;
        bool finished = false;

        for (int k = 0; k < nitems && !finished; ++k) {
            const int s = k % kStages;
            const bool arrived = mbar_wait(&bars[s], (uint32_t)((k / kStages) & 1));
            if (!__all_sync(0xffffffffu, arrived)) {
                failed = k;
                break;
            }
            const unsigned char* st = wbase + s * G::STAGE;
            const S* sp0 = reinterpret_cast<const S*>(st + G::POFF);
            const float* sf0 = reinterpret_cast<const float*>(st + G::FOFF);
#pragma unroll
            for (int h = 0; h < kRows; ++h) {
                const int i = r0 - 1 + kRows * k + h;
                if (i > r1) break;
                const S* spx = sp0 + h * G::WP;                 // p_x of row i
                const S* spy = sp0 + (kRows + h) * G::WP;       // p_y of row i
                const float* sf = sf0 + h * G::WF;
                const float4 cpx = sm_ld4<S>(spx + G::HP + 4 * lane);
                const float4 cpy = sm_ld4<S>(spy + G::HP + 4 * lane);
                float cpxl = 0.f, cpxr = 0.f, cpyr = 0.f, cfr = 0.f;
                if (lane == 0) cpxl = sm_ld1<S>(spx + G::HP - 1);
                if (lane == 31) {
                    cpxr = sm_ld1<S>(spx + G::HP + kStrip);
                    cpyr = sm_ld1<S>(spy + G::HP + kStrip);
                    cfr = sf[G::HF + kStrip];
                }
                const float4 cf = *reinterpret_cast<const float4*>(sf + G::HF + 4 * lane);
                if (i == r0 - 1) {
                    // row r0 - 1 supplies p_y above the first row (zero outside the grid or in the last row)
                    if (i <= R - 2) {
                        pyu = cpy;
                        pyu_r = cpyr;
                    }
                    continue;
                }
                const bool have = i < rend;
                float zc[4] = {0.f, 0.f, 0.f, 0.f};
                float zcr = 0.f;
                if (have) {
                    // z = div p - f2 at row i (zero-extension rule of D^-)
                    float pxs[4] = {cpx.x, cpx.y, cpx.z, cpx.w};
                    if (edge_col) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (j0 + e > C - 2) pxs[e] = 0.f;
                    }
                    float left = __shfl_up_sync(0xffffffffu, pxs[3], 1);
                    if (lane == 0) left = cpxl;               // column x0 - 1 (zero left of the grid)
                    float pyc[4] = {cpy.x, cpy.y, cpy.z, cpy.w};
                    float cpyr_m = cpyr;
                    if (i > R - 2) {                          // last row: D^- reads p_y as zero
                        pyc[0] = pyc[1] = pyc[2] = pyc[3] = 0.f;
                        cpyr_m = 0.f;
                    }
                    // z = ((p_x - p_x,left) + (p_y - p_y,up)) - f2, two pixels per instruction
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        const float2 px2 = make_float2(pxs[2 * h2], pxs[2 * h2 + 1]);
                        const float2 pl2 = make_float2(h2 == 0 ? left : pxs[1], pxs[2 * h2]);
                        const float2 py2 = make_float2(pyc[2 * h2], pyc[2 * h2 + 1]);
                        const float2 pu2 = h2 == 0 ? make_float2(pyu.x, pyu.y) : make_float2(pyu.z, pyu.w);
                        const float2 f2v = h2 == 0 ? make_float2(cf.x, cf.y) : make_float2(cf.z, cf.w);
                        const float2 z2 = p_sub(p_add(p_sub(px2, pl2), p_sub(py2, pu2)), f2v);
                        zc[2 * h2] = z2.x;
                        zc[2 * h2 + 1] = z2.y;
                    }
                    if (lane == 31 && jr < C) {
                        const float pxr_m = (jr <= C - 2) ? cpxr : 0.f;
                        zcr = (pxr_m - pxs[3]) + (cpyr_m - pyu_r) - cfr;
                    }
                    if (WRITE_D && i < r1) {
                        float* dd = d_out + (size_t)i * d_pitch;
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (j0 + e < C) dd[j0 + e] = -zc[e] * alpha_inv;
                    }
                    if (CHECK && i < r1) {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (j0 + e < C) {
                                const float dv = zc[e] + comp(cf, e);   // div p
                                ks[3].add(dv * dv);
                            }
                    }
                    pyu = make_float4(pyc[0], pyc[1], pyc[2], pyc[3]);
                    pyu_r = cpyr_m;
                }
                if (i - 1 >= r0) {
                    // update row i - 1 from z(i-1) (zp) and z(i) (zc)
                    const int ir = i - 1;
                    float zright = __shfl_down_sync(0xffffffffu, zp[0], 1);
                    if (lane == 31) zright = zpr;
                    float res_x[4], res_y[4];
                    const bool last_row = ir >= R - 1;       // D^+ is zero across the last row
                    const float2 t2 = make_float2(t, t);
#pragma unroll
                    for (int h2 = 0; h2 < 2; ++h2) {
                        // pixels e = 2 h2, 2 h2 + 1 as one pair
                        const float2 zp2 = make_float2(zp[2 * h2], zp[2 * h2 + 1]);
                        const float2 zn2 = make_float2(zp[2 * h2 + 1], h2 == 1 ? zright : zp[2]);
                        float2 gx2 = p_sub(zn2, zp2);
                        if (edge_col) {
                            if (j0 + 2 * h2 >= C - 1) gx2.x = 0.f;
                            if (j0 + 2 * h2 + 1 >= C - 1) gx2.y = 0.f;
                        }
                        const float2 gy2 = last_row ? make_float2(0.f, 0.f)
                                                    : p_sub(make_float2(zc[2 * h2], zc[2 * h2 + 1]), zp2);
                        const float2 px2 = h2 == 0 ? make_float2(pprevx.x, pprevx.y) : make_float2(pprevx.z, pprevx.w);
                        const float2 py2 = h2 == 0 ? make_float2(pprevy.x, pprevy.y) : make_float2(pprevy.z, pprevy.w);
                        // |psi| = s2 rsqrt(s2), s2 = gx^2 + gy^2 + 1e-30 (as fast_norm)
                        const float2 s2 = p_fma(gx2, gx2, p_fma(gy2, gy2, make_float2(1e-30f, 1e-30f)));
                        const float2 ng2 = p_mul(s2, make_float2(rsqrtf(s2.x), rsqrtf(s2.y)));
                        if (WRITE_P) {
                            // p <- (p + t psi) / (1 + t |psi|)
                            const float2 den = p_fma(t2, ng2, make_float2(1.f, 1.f));
                            const float2 inv = make_float2(__fdividef(1.0f, den.x), __fdividef(1.0f, den.y));
                            const float2 rx = p_mul(p_fma(t2, gx2, px2), inv);
                            const float2 ry = p_mul(p_fma(t2, gy2, py2), inv);
                            res_x[2 * h2] = rx.x;
                            res_x[2 * h2 + 1] = rx.y;
                            res_y[2 * h2] = ry.x;
                            res_y[2 * h2 + 1] = ry.y;
                        }
                        if (CHECK) {
#pragma unroll
                            for (int l = 0; l < 2; ++l) {
                                const int e = 2 * h2 + l;
                                if (j0 + e < C) {
                                    const float gx = l ? gx2.y : gx2.x, gy = l ? gy2.y : gy2.x;
                                    const float ng = l ? ng2.y : ng2.x;
                                    const float pxv = l ? px2.y : px2.x, pyv = l ? py2.y : py2.x;
                                    ks[0].add(ng);
                                    ks[1].add(ng - (gx * pxv + gy * pyv));
                                    ks[2].add(zp[e] * zp[e]);
                                    pmax = fmaxf(pmax, fast_norm(pxv, pyv));
                                }
                            }
                        }
                    }
                    if (WRITE_P) {
                        const size_t o = (size_t)ir * pitch + j0;
                        if (j0 + 3 < C) {
                            St::st4(pout + o, make_float4(res_x[0], res_x[1], res_x[2], res_x[3]), rkey(seed, o, 0));
                            St::st4(pout + plane + o, make_float4(res_y[0], res_y[1], res_y[2], res_y[3]),
                                    rkey(seed, o, 1));
                        } else {
#pragma unroll
                            for (int e = 0; e < 4; ++e)
                                if (j0 + e < C) {
                                    St::st1(pout + o + e, res_x[e], rkey(seed, o + e, 0));
                                    St::st1(pout + plane + o + e, res_y[e], rkey(seed, o + e, 1));
                                }
                        }
                    }
                }
                // rotate
#pragma unroll
                for (int e = 0; e < 4; ++e) zp[e] = zc[e];
                zpr = zcr;
                pprevx = cpx;
                pprevy = cpy;
                if (i >= r1) finished = true;    // row r1 only supplied z for the update of row r1 - 1
            }
            __syncwarp();
            if (issued < nitems && !finished) {
                if (lane == 0) {
                    fence_proxy_async();          // this warp's reads of stage s precede its refill
                    issue(issued);
                }
                ++issued;
            }
        }
        if (failed >= 0) {
            // a row never arrived: record it and drain this warp's copies still in flight
            if (lane == 0) atomicOr(err, 1u);
            for (int k = failed; k < issued; ++k) (void)mbar_drain(&bars[k % kStages], (uint32_t)((k / kStages) & 1));
        } else {
            // loads issued past the last visited item (none when the chunk ends on an item boundary)
            for (int k = nitems; k < issued; ++k) (void)mbar_drain(&bars[k % kStages], (uint32_t)((k / kStages) & 1));
        }
    }
    if (CHECK) {
        // deterministic warp reduction of FP32 pairs (two-sum), one FP64 partial per warp
        FF acc[kRedSlots];
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) acc[k] = k < 4 ? ks[k].pair() : FF{k == 4 ? pmax : 0.0f, 0.0f};
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) {
            FF x = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const FF y{__shfl_xor_sync(0xffffffffu, x.hi, o), __shfl_xor_sync(0xffffffffu, x.lo, o)};
                x = red_is_max(k) ? FF{fmaxf(x.hi, y.hi), 0.0f} : ff_add(x, y);
            }
            acc[k] = x;
        }
        if (lane < kRedSlots) {
            const size_t w = (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kStreamWarps + wib;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < kRedSlots; ++k)
                if (k == lane) v = (double)acc[k].hi + (double)acc[k].lo;
            partial[w * kRedSlots + lane] = v;
        }
    }
}

int irv1_blocks(int R, int C) {
    // partial slots: one per warp of the streaming kernel
    const int strips = (C + kStrip - 1) / kStrip;
    const int chunks = (R + kChunk - 1) / kChunk;
    return strips * ((chunks + kStreamWarps - 1) / kStreamWarps) * kStreamWarps;
}

template <class S>
static cudaError_t launch_irv1_t(const S* pin, S* pout, const float* f2, int R, int C, int pitch, long plane,
                                 float t, float alpha, bool check, bool write_p, float* d_out, int d_pitch,
                                 double* partial, uint32_t seed, unsigned* err, cudaStream_t s) {
    using G = StreamGeom<S>;
    CUtensorMap pmap, fmap;
    if (!make_tensor_map(&pmap, pin, std::is_same<S, float>::value ? TVS_F32
                                     : std::is_same<S, __nv_bfloat16>::value ? TVS_BF16
                                     : std::is_same<S, __half>::value ? TVS_F16 : TVS_S16,
                         R, C, pitch, plane, 2, G::WP, kRows) ||
        !make_tensor_map(&fmap, f2, TVS_F32, R, C, pitch, (long)R * pitch, 1, G::WF, kRows))
        return cudaErrorInvalidValue;
    const int strips = (C + kStrip - 1) / kStrip;
    const int chunks = (R + kChunk - 1) / kChunk;
    const dim3 blk(32 * kStreamWarps), grd(strips, (chunks + kStreamWarps - 1) / kStreamWarps);
    const size_t smem = stream_smem_bytes<S>();
    const float ainv = 1.0f / alpha;
    const bool wd = d_out != nullptr;
    cudaError_t e = cudaSuccess;
#define TVS_IRV1(CK, WP, WD)                                                                                   \
    do {                                                                                                       \
        static std::once_flag once;                                                                           \
        std::call_once(once, [] {                                                                             \
            cudaFuncSetAttribute(irv1_stream_kernel<S, CK, WP, WD>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 (int)stream_smem_bytes<S>());                                               \
        });                                                                                                    \
        e = launch_pdl(irv1_stream_kernel<S, CK, WP, WD>, grd, blk, smem, s, pmap, fmap, pin, pout, R, C, pitch, \
                       plane, t, ainv, d_out, d_pitch, partial, seed, err);                                   \
    } while (0)
    if (!check && write_p && !wd) TVS_IRV1(false, true, false);
    else if (check && write_p && !wd) TVS_IRV1(true, true, false);
    else if (check && !write_p && wd) TVS_IRV1(true, false, true);
    else if (check && !write_p && !wd) TVS_IRV1(true, false, false);
    else if (!check && !write_p && wd) TVS_IRV1(false, false, true);
    else TVS_IRV1(true, true, true);
#undef TVS_IRV1
    return e;
}

cudaError_t launch_irv1_update(const void* pin, void* pout, const float* f2, int R, int C, int pitch,
                               long plane, float t, float alpha, bool check, bool write_p,
                               float* d_out, int d_pitch, double* partial, int storage, uint32_t seed,
                               unsigned* err, cudaStream_t s) {
    ProfScope ps((check || !write_p) ? kProfIrv1Check : kProfIrv1Update, s);
    TVS_STORAGE_SWITCH(storage, {
        return launch_irv1_t<S>(static_cast<const S*>(pin), static_cast<S*>(pout), f2, R, C, pitch, plane, t, alpha,
                                check, write_p, d_out, d_pitch, partial, seed, err, s);
    })
    return cudaErrorInvalidValue;
}

// ---------------------------------------------------------------------------
// Plane copies between layouts and storage formats (dense or pitched; float,
// bf16 or fp16), rounding to nearest when narrowing.  blockIdx.z = plane.
// ---------------------------------------------------------------------------
template <class SD, class SS>
__global__ void convert_planes_kernel(SD* __restrict__ dst, int dpitch, long dplane, const SS* __restrict__ src,
                                      int spitch, long splane, int rows, int cols) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= rows || j >= cols) return;
    const float v = Stor<SS>::ld1(src + (size_t)blockIdx.z * splane + (size_t)i * spitch + j);
    const size_t o = (size_t)i * dpitch + j;
    Stor<SD>::st1(dst + (size_t)blockIdx.z * dplane + o, v, rkey(0x2545f491U, o, blockIdx.z));
}

cudaError_t convert_planes(void* dst, int dst_storage, int dpitch, long dplane, const void* src, int src_storage,
                           int spitch, long splane, int rows, int cols, int planes, cudaStream_t s) {
    const dim3 blk(32, 8), grd((cols + 31) / 32, (rows + 7) / 8, planes);
    ProfScope ps(kProfSetup, s);
    TVS_STORAGE_SWITCH(dst_storage, {
        using SD = S;
        TVS_STORAGE_SWITCH(src_storage, {
            convert_planes_kernel<SD, S><<<grd, blk, 0, s>>>(static_cast<SD*>(dst), dpitch, dplane,
                                                             static_cast<const S*>(src), spitch, splane, rows, cols);
        })
    })
    return cudaGetLastError();
}

}  // namespace tvs

namespace tvs {

// ---------------------------------------------------------------------------
// IRV2 (Section 3.3, eq. ir2dualdis) and the W^{1,1} dual (eq. IRW11:dual)
// ---------------------------------------------------------------------------
// Source of the potential g with grad g = tau_perp in the least-squares sense
// over the differences between neighbouring image pixels: div v for the
// forward-edge field v_x(i, j) = tau_2(i, j+1) (j <= n1-2), v_y(i, j) =
// -tau_1(i+1, j) (i <= n2-2), both zero on the last column / row, with the
// zero extension of D^-.  g = Delta^dagger div v on the n2 x n1 grid.
__global__ void potential_src_kernel(const float* __restrict__ tau, long tplane, int tpitch, int n2, int n1,
                                     float* __restrict__ S, int spitch) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n2 || j >= n1) return;
    const float* t1 = tau;
    const float* t2 = tau + tplane;
    float s = 0.f;
    if (j <= n1 - 2) s += __ldg(&t2[(size_t)i * tpitch + j + 1]);   // v_x(i, j)
    if (j >= 1) s -= __ldg(&t2[(size_t)i * tpitch + j]);            // v_x(i, j-1)
    if (i <= n2 - 2) s -= __ldg(&t1[(size_t)(i + 1) * tpitch + j]); // v_y(i, j)
    if (i >= 1) s += __ldg(&t1[(size_t)i * tpitch + j]);            // v_y(i-1, j)
    S[(size_t)i * spitch + j] = s;
}

// f = alpha (d0 - g), the data of eq. ir2dualdis
__global__ void irv2_f_kernel(const float* __restrict__ d0, int d0_pitch, const float* __restrict__ g, int gpitch,
                              int n2, int n1, float alpha, float* __restrict__ f, int fpitch) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n2 || j >= n1) return;
    f[(size_t)i * fpitch + j] = alpha * (__ldg(&d0[(size_t)i * d0_pitch + j]) - __ldg(&g[(size_t)i * gpitch + j]));
}

// d += g (d = u + g after the ROF problem in u = d - g)
__global__ void add_plane_kernel(float* __restrict__ d, int dpitch, const float* __restrict__ g, int gpitch, int n2,
                                 int n1) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n2 || j >= n1) return;
    d[(size_t)i * dpitch + j] += __ldg(&g[(size_t)i * gpitch + j]);
}

// p += sign * xi on the dense n2 x n1 two-plane field p (W^{1,1} dual p = q + xi)
__global__ void shift_xi_kernel(float* __restrict__ p, int n2, int n1, const float* __restrict__ tau, long tplane,
                                int tpitch, float eps, float sign) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= n2 || j >= n1) return;
    const float2 xi = xi_at(tau, tplane, tpitch, i, j, eps);
    const size_t o = (size_t)i * n1 + j;
    p[o] = fmaf(sign, xi.x, p[o]);
    p[(size_t)n2 * n1 + o] = fmaf(sign, xi.y, p[(size_t)n2 * n1 + o]);
}

static inline dim3 grid_2d(int rows, int cols) { return dim3((cols + 31) / 32, (rows + 7) / 8); }

cudaError_t launch_potential_src(const float* tau, long tplane, int tpitch, int n2, int n1, float* S, int spitch,
                                 cudaStream_t s) {
    ProfScope ps(kProfSetup, s);
    potential_src_kernel<<<grid_2d(n2, n1), dim3(32, 8), 0, s>>>(tau, tplane, tpitch, n2, n1, S, spitch);
    return cudaGetLastError();
}

cudaError_t launch_irv2_f(const float* d0, int d0_pitch, const float* g, int gpitch, int n2, int n1, float alpha,
                          float* f, int fpitch, cudaStream_t s) {
    ProfScope ps(kProfSetup, s);
    irv2_f_kernel<<<grid_2d(n2, n1), dim3(32, 8), 0, s>>>(d0, d0_pitch, g, gpitch, n2, n1, alpha, f, fpitch);
    return cudaGetLastError();
}

cudaError_t launch_add_plane(float* d, int dpitch, const float* g, int gpitch, int n2, int n1, cudaStream_t s) {
    ProfScope ps(kProfSetup, s);
    add_plane_kernel<<<grid_2d(n2, n1), dim3(32, 8), 0, s>>>(d, dpitch, g, gpitch, n2, n1);
    return cudaGetLastError();
}

cudaError_t irv_set_wait_limit(long long cycles) { return set_wait_limit_here(cycles); }

cudaError_t launch_shift_xi(float* p, int n2, int n1, const float* tau, long tplane, int tpitch, float eps,
                            float sign, cudaStream_t s) {
    ProfScope ps(kProfSetup, s);
    shift_xi_kernel<<<grid_2d(n2, n1), dim3(32, 8), 0, s>>>(p, n2, n1, tau, tplane, tpitch, eps, sign);
    return cudaGetLastError();
}

}  // namespace tvs
