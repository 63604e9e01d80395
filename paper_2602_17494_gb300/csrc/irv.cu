// Step 2, image reconstruction IRV1 (Section 4.2, eq. ir1dualdis):
//   xi = tau_perp / sqrt(|tau_perp|^2 + eps), tau_perp = R_Omega(tau_2, -tau_1)
//   f2 = alpha d0 - div xi
//   Chambolle: z = div p - f2, psi = grad z, p <- (p + t psi) / (1 + t |psi|)
//   d = (f2 - div p) / alpha = -z / alpha
//
// The backward difference D^-_x of Section 4.1 equals the plain difference of
// the field with its last column (and everything left of the grid) read as
// zero; D^-_y likewise with the last row.  The tiles below load the dual with
// exactly those zeros, so one stencil covers the interior and the boundary.
#include "tvs_internal.cuh"
#include "prof.h"

namespace tvs {

constexpr int kTX = 32;   // tile width (one 128-byte line of floats)
constexpr int kTY = 16;   // tile height
constexpr int kBY = 8;    // thread rows; each thread does kTY / kBY output rows

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
// Fused IRV1 update (and/or check) kernel.
//   CHECK  : block partial sums of the gap/energy terms at the input p
//   WRITE_P: write the updated dual
//   WRITE_D: write d = -z / alpha at the input p
// ---------------------------------------------------------------------------
template <bool CHECK, bool WRITE_P, bool WRITE_D>
__global__ void __launch_bounds__(kTX * kBY)
irv1_update_kernel(const float* __restrict__ pin, float* __restrict__ pout, const float* __restrict__ f2,
                   int R, int C, int pitch, long plane, float t, float alpha_inv,
                   float* __restrict__ d_out, int d_pitch, double* __restrict__ partial) {
    __shared__ float sx[kTY + 1][kTX + 2];  // p_x rows i0..i0+TY, cols j0-1..j0+TX
    __shared__ float sy[kTY + 2][kTX + 1];  // p_y rows i0-1..i0+TY, cols j0..j0+TX
    __shared__ float sf[kTY + 1][kTX + 1];
    __shared__ float sz[kTY + 1][kTX + 1];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    constexpr int NT = kTX * kBY;
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;
    const float* __restrict__ px = pin;
    const float* __restrict__ py = pin + plane;

    for (int idx = tid; idx < (kTY + 1) * (kTX + 2); idx += NT) {
        const int r = idx / (kTX + 2), c = idx - r * (kTX + 2);
        const int i = i0 + r, j = j0 - 1 + c;
        sx[r][c] = (i < R && j >= 0 && j <= C - 2) ? __ldg(&px[(size_t)i * pitch + j]) : 0.f;
    }
    for (int idx = tid; idx < (kTY + 2) * (kTX + 1); idx += NT) {
        const int r = idx / (kTX + 1), c = idx - r * (kTX + 1);
        const int i = i0 - 1 + r, j = j0 + c;
        sy[r][c] = (i >= 0 && i <= R - 2 && j < C) ? __ldg(&py[(size_t)i * pitch + j]) : 0.f;
    }
    for (int idx = tid; idx < (kTY + 1) * (kTX + 1); idx += NT) {
        const int r = idx / (kTX + 1), c = idx - r * (kTX + 1);
        const int i = i0 + r, j = j0 + c;
        sf[r][c] = (i < R && j < C) ? __ldg(&f2[(size_t)i * pitch + j]) : 0.f;
    }
    __syncthreads();
    for (int idx = tid; idx < (kTY + 1) * (kTX + 1); idx += NT) {
        const int r = idx / (kTX + 1), c = idx - r * (kTX + 1);
        sz[r][c] = (sx[r][c + 1] - sx[r][c]) + (sy[r + 1][c] - sy[r][c]) - sf[r][c];
    }
    __syncthreads();

    double acc[kRedSlots];
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) acc[k] = 0.0;
#pragma unroll
    for (int rr = ty; rr < kTY; rr += kBY) {
        const int i = i0 + rr, j = j0 + tx;
        if (i < R && j < C) {
            const float z = sz[rr][tx];
            const float gx = (j < C - 1) ? sz[rr][tx + 1] - z : 0.f;
            const float gy = (i < R - 1) ? sz[rr + 1][tx] - z : 0.f;
            const size_t o = (size_t)i * pitch + j;
            const float pxv = __ldg(&px[o]), pyv = __ldg(&py[o]);
            if (WRITE_P) {
                const float den = 1.0f + t * sqrtf(gx * gx + gy * gy);
                pout[o] = (pxv + t * gx) / den;
                pout[plane + o] = (pyv + t * gy) / den;
            }
            if (WRITE_D) d_out[(size_t)i * d_pitch + j] = -z * alpha_inv;
            if (CHECK) {
                const double dgx = gx, dgy = gy, dpx = pxv, dpy = pyv;
                acc[0] += sqrt(dgx * dgx + dgy * dgy);
                acc[1] += dgx * dpx + dgy * dpy;
                acc[2] += (double)z * (double)z;
                const double dv = (double)z + (double)sf[rr][tx];
                acc[3] += dv * dv;
                acc[4] = fmax(acc[4], sqrt(dpx * dpx + dpy * dpy));
            }
        }
    }
    if (CHECK) block_reduce_store<NT>(acc, partial + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kRedSlots, tid);
}

int irv1_blocks(int R, int C) { return ((C + kTX - 1) / kTX) * ((R + kTY - 1) / kTY); }

cudaError_t launch_irv1_update(const float* pin, float* pout, const float* f2, int R, int C, int pitch,
                               long plane, float t, float alpha, bool check, bool write_p,
                               float* d_out, int d_pitch, double* partial, cudaStream_t s) {
    dim3 blk(kTX, kBY), grd((C + kTX - 1) / kTX, (R + kTY - 1) / kTY);
    const float ainv = 1.0f / alpha;
    const bool wd = d_out != nullptr;
    ProfScope ps((check || !write_p) ? kProfIrv1Check : kProfIrv1Update, s);
#define TVS_IRV1(CK, WP, WD) \
    irv1_update_kernel<CK, WP, WD><<<grd, blk, 0, s>>>(pin, pout, f2, R, C, pitch, plane, t, ainv, d_out, d_pitch, partial)
    if (!check && write_p && !wd) TVS_IRV1(false, true, false);
    else if (check && write_p && !wd) TVS_IRV1(true, true, false);
    else if (check && !write_p && wd) TVS_IRV1(true, false, true);
    else if (check && !write_p && !wd) TVS_IRV1(true, false, false);
    else if (!check && !write_p && wd) TVS_IRV1(false, false, true);
    else TVS_IRV1(true, true, true);
#undef TVS_IRV1
    return cudaGetLastError();
}

}  // namespace tvs
