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

namespace tvs {

// ---------------------------------------------------------------------------
// xi and f2 (eq. defXi2:discrete, eq. ir1dualdis)
// ---------------------------------------------------------------------------
__device__ __forceinline__ float2 xi_at(const float* __restrict__ tau, long tplane, int tpitch,
                                        int i, int j, float eps) {
    const float tp1 = __ldg(&tau[tplane + (size_t)i * tpitch + j]);    // tau_2
    const float tp2 = -__ldg(&tau[(size_t)i * tpitch + j]);            // -tau_1
    const float den = sqrtf(tp1 * tp1 + tp2 * tp2 + eps);
    return make_float2(tp1 / den, tp2 / den);
}

__global__ void xi_f2_kernel(const float* __restrict__ d0, int d0_pitch, const float* __restrict__ tau,
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

cudaError_t launch_xi_f2(const float* d0, int d0_pitch, const float* tau, long tplane, int tpitch,
                         int R, int C, float alpha, float eps, float* f2, int fpitch, cudaStream_t s) {
    dim3 blk(32, 8), grd((C + 31) / 32, (R + 7) / 8);
    xi_f2_kernel<<<grd, blk, 0, s>>>(d0, d0_pitch, tau, tplane, tpitch, R, C, alpha, eps, f2, fpitch);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Streaming IRV1 update: each warp owns a strip of 128 columns (4 per lane,
// float4 loads) and walks down a chunk of rows, keeping the previous row's
// dual and residual in registers.  Left/right neighbours come from warp
// shuffles; only the strip edges load scalar halo values.  No shared memory
// and no barriers, so HBM traffic is the 20 algorithmic bytes per pixel plus
// one extra row per chunk.  Requires pitch % 4 == 0 and 16-byte aligned planes.
//   CHECK  : per-warp partial sums of the gap/energy terms at the input p
//   WRITE_P: write the updated dual
//   WRITE_D: write d = -z / alpha at the input p
// ---------------------------------------------------------------------------
constexpr int kStrip = 128;      // columns per warp
constexpr int kChunk = 32;       // output rows per warp
constexpr int kStreamWarps = 4;  // warps per block

struct Row4 {
    float4 px, py, f;
};
__device__ __forceinline__ float comp(const float4& v, int e) {
    return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w));
}

template <class S, bool CHECK, bool WRITE_P, bool WRITE_D>
__global__ void __launch_bounds__(32 * kStreamWarps, CHECK ? 5 : 8)
irv1_stream_kernel(const S* __restrict__ pin, S* __restrict__ pout, const float* __restrict__ f2, int R,
                   int C, int pitch, long plane, float t, float alpha_inv, float* __restrict__ d_out, int d_pitch,
                   double* __restrict__ partial) {
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const int strip = blockIdx.x;
    const int chunk = blockIdx.y * kStreamWarps + wib;
    const int r0 = chunk * kChunk;
    const int j0 = strip * kStrip + 4 * lane;     // first column of this lane
    const int r1 = min(r0 + kChunk, R);           // output rows [r0, r1)
    using St = Stor<S>;
    const S* __restrict__ px = pin;
    const S* __restrict__ py = pin + plane;
    KSum ks[4];
    float pmax = 0.0f;

    if (r0 < R) {
        const int jr = strip * kStrip + kStrip;   // first column right of the strip
        // column masks: D^- reads p_x as zero in the last column and beyond the grid
        float mx[4], mv[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            mv[e] = (j0 + e < C) ? 1.f : 0.f;
            mx[e] = (j0 + e <= C - 2) ? 1.f : 0.f;
        }
        const size_t cbase = (size_t)j0;
        // row r0 - 1: p_y (for div at row r0)
        float4 pyu = make_float4(0.f, 0.f, 0.f, 0.f);
        float pyu_r = 0.f;                         // p_y(r0 - 1, jr) for the right halo (lane 31)
        if (r0 >= 1 && r0 - 1 <= R - 2) {
            pyu = St::ld4(py + (size_t)(r0 - 1) * pitch + cbase);
            if (lane == 31 && jr < C) pyu_r = St::ld1(py + (size_t)(r0 - 1) * pitch + jr);
        }
        auto load_row = [&](int i, Row4& rw, float& pxl, float& pxr, float& pyr, float& fr) {
            const size_t o = (size_t)i * pitch + cbase;
            rw.px = St::ld4(px + o);
            rw.py = St::ld4(py + o);
            rw.f = Stor<float>::ld4(f2 + o);
            pxl = (lane == 0 && j0 >= 1) ? St::ld1(px + (size_t)i * pitch + j0 - 1) : 0.f;
            pxr = 0.f;
            pyr = 0.f;
            fr = 0.f;
            if (lane == 31 && jr < C) {
                pxr = St::ld1(px + (size_t)i * pitch + jr);
                pyr = St::ld1(py + (size_t)i * pitch + jr);
                fr = __ldg(&f2[(size_t)i * pitch + jr]);
            }
        };
        Row4 cur, nxt;
        float cpxl, cpxr, cpyr, cfr, npxl = 0.f, npxr = 0.f, npyr = 0.f, nfr = 0.f;
        load_row(r0, cur, cpxl, cpxr, cpyr, cfr);
        float zp[4] = {0.f, 0.f, 0.f, 0.f};        // z of the previous row
        float zpr = 0.f;                           // z(prev row, jr) on lane 31
        float4 pprevx = make_float4(0.f, 0.f, 0.f, 0.f), pprevy = pprevx;
        const int rend = min(r1 + 1, R);           // rows whose z is needed
        for (int i = r0; i <= r1; ++i) {
            const bool have = i < rend;
            if (i + 1 < rend) load_row(i + 1, nxt, npxl, npxr, npyr, nfr);
            float zc[4] = {0.f, 0.f, 0.f, 0.f};
            float zcr = 0.f;
            if (have) {
                // z = div p - f2 at row i (zero-extension rule of D^-)
                const float ymask = (i <= R - 2) ? 1.f : 0.f;
                float pxs[4] = {cur.px.x * mx[0], cur.px.y * mx[1], cur.px.z * mx[2], cur.px.w * mx[3]};
                float left = __shfl_up_sync(0xffffffffu, pxs[3], 1);
                if (lane == 0) left = (j0 >= 1 && j0 - 1 <= C - 2) ? cpxl : 0.f;
                const float pyc[4] = {cur.py.x * ymask, cur.py.y * ymask, cur.py.z * ymask, cur.py.w * ymask};
                const float pyp[4] = {pyu.x, pyu.y, pyu.z, pyu.w};
                const float fv[4] = {cur.f.x, cur.f.y, cur.f.z, cur.f.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float pl = e == 0 ? left : pxs[e - 1];
                    zc[e] = ((pxs[e] - pl) + (pyc[e] - pyp[e]) - fv[e]) * mv[e];
                }
                if (lane == 31 && jr < C) {
                    const float pxr_m = (jr <= C - 2) ? cpxr : 0.f;
                    zcr = (pxr_m - pxs[3]) + (cpyr * ymask - pyu_r) - cfr;
                }
                if (WRITE_D && i < r1) {
                    float* dd = d_out + (size_t)i * d_pitch;
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (j0 + e < C) dd[j0 + e] = -zc[e] * alpha_inv;
                }
                pyu = make_float4(pyc[0], pyc[1], pyc[2], pyc[3]);
                pyu_r = cpyr * ymask;
            }
            if (i > r0) {
                // update row i - 1 from z(i-1) (zp), z(i) (zc)
                const int ir = i - 1;
                float zright = __shfl_down_sync(0xffffffffu, zp[0], 1);
                if (lane == 31) zright = zpr;
                float res_x[4], res_y[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float zn = e == 3 ? zright : zp[e + 1];
                    const float gx = (j0 + e < C - 1) ? zn - zp[e] : 0.f;
                    const float gy = (ir < R - 1) ? zc[e] - zp[e] : 0.f;
                    const float pxv = comp(pprevx, e), pyv = comp(pprevy, e);
                    if (WRITE_P) {
                        const float den = 1.0f + t * sqrtf(gx * gx + gy * gy);
                        res_x[e] = (pxv + t * gx) / den;
                        res_y[e] = (pyv + t * gy) / den;
                    }
                    if (CHECK && j0 + e < C) {
                        const float ng = sqrtf(gx * gx + gy * gy);
                        ks[0].add(ng);
                        ks[1].add(ng - (gx * pxv + gy * pyv));
                        ks[2].add(zp[e] * zp[e]);
                        pmax = fmaxf(pmax, sqrtf(pxv * pxv + pyv * pyv));
                    }
                }
                if (WRITE_P) {
                    const size_t o = (size_t)ir * pitch + cbase;
                    if (j0 + 3 < C) {
                        St::st4(pout + o, make_float4(res_x[0], res_x[1], res_x[2], res_x[3]));
                        St::st4(pout + plane + o, make_float4(res_y[0], res_y[1], res_y[2], res_y[3]));
                    } else {
#pragma unroll
                        for (int e = 0; e < 4; ++e)
                            if (j0 + e < C) {
                                St::st1(pout + o + e, res_x[e]);
                                St::st1(pout + plane + o + e, res_y[e]);
                            }
                    }
                }
            }
            if (CHECK && have && i < r1) {
                const float fv[4] = {cur.f.x, cur.f.y, cur.f.z, cur.f.w};
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j0 + e < C) {
                        const float dv = zc[e] + fv[e];   // div p
                        ks[3].add(dv * dv);
                    }
            }
            // rotate
#pragma unroll
            for (int e = 0; e < 4; ++e) zp[e] = zc[e];
            zpr = zcr;
            if (have) {
                pprevx = cur.px;
                pprevy = cur.py;
            }
            cur = nxt;
            cpxl = npxl;
            cpxr = npxr;
            cpyr = npyr;
            cfr = nfr;
        }
    }
    if (CHECK) {
        double acc[kRedSlots];
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) acc[k] = k < 4 ? ks[k].value() : (k == 4 ? (double)pmax : 0.0);
        // deterministic warp reduction, one partial per warp
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) {
            double x = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const double y = __shfl_xor_sync(0xffffffffu, x, o);
                x = red_is_max(k) ? fmax(x, y) : x + y;
            }
            acc[k] = x;
        }
        if (lane < kRedSlots) {
            const size_t w = (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kStreamWarps + wib;
            double v = 0.0;
#pragma unroll
            for (int k = 0; k < kRedSlots; ++k)
                if (k == lane) v = acc[k];
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

cudaError_t launch_irv1_update(const void* pin, void* pout, const float* f2, int R, int C, int pitch,
                               long plane, float t, float alpha, bool check, bool write_p,
                               float* d_out, int d_pitch, double* partial, int storage, cudaStream_t s) {
    const int strips = (C + kStrip - 1) / kStrip;
    const int chunks = (R + kChunk - 1) / kChunk;
    dim3 blk(32 * kStreamWarps), grd(strips, (chunks + kStreamWarps - 1) / kStreamWarps);
    const float ainv = 1.0f / alpha;
    const bool wd = d_out != nullptr;
    ProfScope ps((check || !write_p) ? kProfIrv1Check : kProfIrv1Update, s);
#define TVS_IRV1(CK, WP, WD)                                                                              \
    irv1_stream_kernel<S, CK, WP, WD><<<grd, blk, 0, s>>>(static_cast<const S*>(pin), static_cast<S*>(pout), f2, R, \
                                                          C, pitch, plane, t, ainv, d_out, d_pitch, partial)
    TVS_STORAGE_SWITCH(storage, {
        if (!check && write_p && !wd) TVS_IRV1(false, true, false);
        else if (check && write_p && !wd) TVS_IRV1(true, true, false);
        else if (check && !write_p && wd) TVS_IRV1(true, false, true);
        else if (check && !write_p && !wd) TVS_IRV1(true, false, false);
        else if (!check && !write_p && wd) TVS_IRV1(false, false, true);
        else TVS_IRV1(true, true, true);
    })
#undef TVS_IRV1
    return cudaGetLastError();
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
    Stor<SD>::st1(dst + (size_t)blockIdx.z * dplane + (size_t)i * dpitch + j, v);
}

cudaError_t convert_planes(void* dst, int dst_storage, int dpitch, long dplane, const void* src, int src_storage,
                           int spitch, long splane, int rows, int cols, int planes, cudaStream_t s) {
    const dim3 blk(32, 8), grd((cols + 31) / 32, (rows + 7) / 8, planes);
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
