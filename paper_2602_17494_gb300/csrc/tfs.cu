// Step 1, tangent field smoothing (Section 4.2, eq. tfsdualdis, Algorithm 1):
//   tau0 = (-D^{neum-}_y d0, D^{neum-}_x d0)             (def:backdiffNeumann)
//   f1   = P_K tau0 / delta
//   per iteration: w = vecdiv p, phi = Delta^dagger div w  (dct.cu)
//                  z = P_K w - f1 = w - grad phi - f1
//                  psi_k = grad z_k, p_k <- (p_k + t psi_k) / (1 + t |psi_k|)
//   tau = P_K tau0 - delta P_K vecdiv p = -delta z
// Arrays live on the extended grid R x C = (N2+1) x (N1+1) with a padded pitch.
#include "tvs_internal.cuh"
#include "prof.h"

namespace tvs {

constexpr int kTX = 32;
constexpr int kTY = 16;
constexpr int kBY = 8;

// ---------------------------------------------------------------------------
// tau0 (Neumann backward differences onto the extended grid)
// ---------------------------------------------------------------------------
__global__ void tau0_kernel(const float* __restrict__ d0, int d_pitch, int n2, int n1,
                            float* __restrict__ tau, int pitch, long plane) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i > n2 || j > n1) return;
    // tau_1 = -D^{neum-}_y d0: zero in the first and last row; the extra last
    // column repeats the last image column.
    float t1 = 0.f;
    if (i != 0 && i != n2) {
        const int c = j < n1 - 1 ? j : n1 - 1;
        t1 = -(__ldg(&d0[(size_t)i * d_pitch + c]) - __ldg(&d0[(size_t)(i - 1) * d_pitch + c]));
    }
    // tau_2 = D^{neum-}_x d0: zero in the first and last column; the extra last
    // row repeats the last image row.
    float t2 = 0.f;
    if (j != 0 && j != n1) {
        const int r = i < n2 - 1 ? i : n2 - 1;
        t2 = __ldg(&d0[(size_t)r * d_pitch + j]) - __ldg(&d0[(size_t)r * d_pitch + j - 1]);
    }
    tau[(size_t)i * pitch + j] = t1;
    tau[plane + (size_t)i * pitch + j] = t2;
}

cudaError_t launch_tau0(const float* d0, int d_pitch, int n2, int n1, float* tau, int pitch, long plane,
                        cudaStream_t s) {
    dim3 blk(32, 8), grd((n1 + 1 + 31) / 32, (n2 + 1 + 7) / 8);
    tau0_kernel<<<grd, blk, 0, s>>>(d0, d_pitch, n2, n1, tau, pitch, long(plane));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// s = div(vecdiv p) on the extended grid (the source of the Poisson solve in
// every TFS iteration), tiled: p with a two-point halo, then w = vecdiv p with
// a one-point halo, then s.  D^- reads its argument as zero in the last
// column (x-part) or row (y-part) and outside the grid.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kTX * kBY)
div_vecdiv_kernel(const float* __restrict__ p, int R, int C, int pitch, long plane, float* __restrict__ S) {
    constexpr int PH = kTY + 2, PW = kTX + 2;      // p region: rows i0-2.., cols j0-2..
    __shared__ float sp[4][PH][PW + 1];
    __shared__ float sw[2][PH - 1][PW];            // w region: rows i0-1.., cols j0-1..
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    constexpr int NT = kTX * kBY;
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;
    for (int q = 0; q < 4; ++q) {
        const bool xpart = (q & 1) == 0;
        for (int idx = tid; idx < PH * PW; idx += NT) {
            const int r = idx / PW, c = idx - r * PW;
            const int i = i0 - 2 + r, j = j0 - 2 + c;
            const bool ok = i >= 0 && j >= 0 && i < R && j < C && (xpart ? j <= C - 2 : i <= R - 2);
            sp[q][r][c] = ok ? __ldg(&p[(size_t)q * plane + (size_t)i * pitch + j]) : 0.f;
        }
    }
    __syncthreads();
    for (int idx = tid; idx < (PH - 1) * (PW - 1); idx += NT) {
        const int r = idx / (PW - 1), c = idx - r * (PW - 1);   // w point (i0-1+r, j0-1+c)
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        const int pr = r + 1, pc = c + 1;                          // same point in the p region
        const float w1 = (sp[0][pr][pc] - sp[0][pr][pc - 1]) + (sp[1][pr][pc] - sp[1][pr - 1][pc]);
        const float w2 = (sp[2][pr][pc] - sp[2][pr][pc - 1]) + (sp[3][pr][pc] - sp[3][pr - 1][pc]);
        const bool in = i >= 0 && j >= 0 && i < R && j < C;
        sw[0][r][c] = (in && j <= C - 2) ? w1 : 0.f;
        sw[1][r][c] = (in && i <= R - 2) ? w2 : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int rr = ty; rr < kTY; rr += kBY) {
        const int i = i0 + rr, j = j0 + tx;
        if (i < R && j < C) {
            const int r = rr + 1, c = tx + 1;
            S[(size_t)i * pitch + j] = (sw[0][r][c] - sw[0][r][c - 1]) + (sw[1][r][c] - sw[1][r - 1][c]);
        }
    }
}

cudaError_t launch_div_vecdiv(const float* p, int R, int C, int pitch, long plane, float* S, cudaStream_t s) {
    dim3 blk(kTX, kBY), grd((C + kTX - 1) / kTX, (R + kTY - 1) / kTY);
    ProfScope ps(kProfOther, s);
    div_vecdiv_kernel<<<grd, blk, 0, s>>>(p, R, C, pitch, plane, S);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// out = scale * (u - grad phi) for a 2-plane field u (the last step of P_K).
// ---------------------------------------------------------------------------
__global__ void grad_sub_kernel(const float* __restrict__ u, int upitch, long uplane,
                                const float* __restrict__ phi, int ppitch, int R, int C, float scale,
                                float* __restrict__ out, int opitch, long oplane) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= R || j >= C) return;
    const float pc = __ldg(&phi[(size_t)i * ppitch + j]);
    const float gx = (j < C - 1) ? __ldg(&phi[(size_t)i * ppitch + j + 1]) - pc : 0.f;
    const float gy = (i < R - 1) ? __ldg(&phi[(size_t)(i + 1) * ppitch + j]) - pc : 0.f;
    const float ux = __ldg(&u[(size_t)i * upitch + j]);
    const float uy = __ldg(&u[uplane + (size_t)i * upitch + j]);
    out[(size_t)i * opitch + j] = scale * (ux - gx);
    out[oplane + (size_t)i * opitch + j] = scale * (uy - gy);
}

cudaError_t launch_grad_sub(const float* u, int upitch, long uplane, const float* phi, int ppitch, int R,
                            int C, float scale, float* out, int opitch, long oplane, cudaStream_t s) {
    dim3 blk(32, 8), grd((C + 31) / 32, (R + 7) / 8);
    grad_sub_kernel<<<grd, blk, 0, s>>>(u, upitch, uplane, phi, ppitch, R, C, scale, out, opitch, oplane);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused TFS update / check.  The tile computes z on rows i0-1..i0+TY and
// columns j0-1..j0+TX (the extra leading row/column serves div z for the
// residual check), psi on the TY x TX outputs.
// ---------------------------------------------------------------------------
template <bool CHECK, bool WRITE_P, bool WRITE_TAU>
__global__ void __launch_bounds__(kTX * kBY)
tfs_update_kernel(const float* __restrict__ pin, float* __restrict__ pout, const float* __restrict__ phi,
                  const float* __restrict__ f1, int R, int C, int pitch, long plane, float t, float delta,
                  float* __restrict__ tau_out, int tau_pitch, long tau_plane, double* __restrict__ partial) {
    constexpr int ZH = kTY + 2, ZW = kTX + 2;     // z region: rows i0-1.., cols j0-1..
    __shared__ float sxa[2][ZH][ZW + 1];           // p_kx rows i0-1..i0+TY, cols j0-2..j0+TX
    __shared__ float sya[2][ZH + 1][ZW];           // p_ky rows i0-2..i0+TY, cols j0-1..j0+TX
    __shared__ float sphi[ZH + 1][ZW + 1];         // phi  rows i0-1..i0+TY+1, cols j0-1..j0+TX+1
    __shared__ float sz[2][ZH][ZW];
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    constexpr int NT = kTX * kBY;
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;

    for (int k = 0; k < 2; ++k) {
        const float* __restrict__ pkx = pin + (size_t)(2 * k) * plane;
        const float* __restrict__ pky = pin + (size_t)(2 * k + 1) * plane;
        for (int idx = tid; idx < ZH * (ZW + 1); idx += NT) {
            const int r = idx / (ZW + 1), c = idx - r * (ZW + 1);
            const int i = i0 - 1 + r, j = j0 - 2 + c;
            sxa[k][r][c] = (i >= 0 && i < R && j >= 0 && j <= C - 2) ? __ldg(&pkx[(size_t)i * pitch + j]) : 0.f;
        }
        for (int idx = tid; idx < (ZH + 1) * ZW; idx += NT) {
            const int r = idx / ZW, c = idx - r * ZW;
            const int i = i0 - 2 + r, j = j0 - 1 + c;
            sya[k][r][c] = (i >= 0 && i <= R - 2 && j >= 0 && j < C) ? __ldg(&pky[(size_t)i * pitch + j]) : 0.f;
        }
    }
    for (int idx = tid; idx < (ZH + 1) * (ZW + 1); idx += NT) {
        const int r = idx / (ZW + 1), c = idx - r * (ZW + 1);
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        sphi[r][c] = (i >= 0 && i < R && j >= 0 && j < C) ? __ldg(&phi[(size_t)i * pitch + j]) : 0.f;
    }
    __syncthreads();
    // z = w - grad phi - f1 on the z region (zero outside the grid)
    for (int idx = tid; idx < ZH * ZW; idx += NT) {
        const int r = idx / ZW, c = idx - r * ZW;
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        float z1 = 0.f, z2 = 0.f;
        if (i >= 0 && i < R && j >= 0 && j < C) {
            const float w1 = (sxa[0][r][c + 1] - sxa[0][r][c]) + (sya[0][r + 1][c] - sya[0][r][c]);
            const float w2 = (sxa[1][r][c + 1] - sxa[1][r][c]) + (sya[1][r + 1][c] - sya[1][r][c]);
            const float pc = sphi[r][c];
            const float gx = (j < C - 1) ? sphi[r][c + 1] - pc : 0.f;
            const float gy = (i < R - 1) ? sphi[r + 1][c] - pc : 0.f;
            const size_t o = (size_t)i * pitch + j;
            z1 = w1 - gx - __ldg(&f1[o]);
            z2 = w2 - gy - __ldg(&f1[plane + o]);
        }
        sz[0][r][c] = z1;
        sz[1][r][c] = z2;
    }
    __syncthreads();

    KSum ks[4];
    float pmax = 0.0f, dmax = 0.0f;
#pragma unroll
    for (int rr = ty; rr < kTY; rr += kBY) {
        const int i = i0 + rr, j = j0 + tx;
        if (i < R && j < C) {
            const int r = rr + 1, c = tx + 1;   // position in the z region
            const size_t o = (size_t)i * pitch + j;
            float zc[2], gx[2], gy[2], pv[4];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                zc[k] = sz[k][r][c];
                gx[k] = (j < C - 1) ? sz[k][r][c + 1] - zc[k] : 0.f;
                gy[k] = (i < R - 1) ? sz[k][r + 1][c] - zc[k] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) pv[q] = __ldg(&pin[(size_t)q * plane + o]);
            if (WRITE_P) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float den = 1.0f + t * sqrtf(gx[k] * gx[k] + gy[k] * gy[k]);
                    pout[(size_t)(2 * k) * plane + o] = (pv[2 * k] + t * gx[k]) / den;
                    pout[(size_t)(2 * k + 1) * plane + o] = (pv[2 * k + 1] + t * gy[k]) / den;
                }
            }
            if (WRITE_TAU) {
                tau_out[(size_t)i * tau_pitch + j] = -delta * zc[0];
                tau_out[tau_plane + (size_t)i * tau_pitch + j] = -delta * zc[1];
            }
            if (CHECK) {
                const size_t fo = o;
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float a = gx[k], b = gy[k], px = pv[2 * k], py = pv[2 * k + 1];
                    const float ng = sqrtf(a * a + b * b);
                    ks[0].add(ng);
                    ks[1].add(ng - (a * px + b * py));
                    ks[2].add(zc[k] * zc[k]);
                    const float zf = zc[k] + __ldg(&f1[(size_t)k * plane + fo]);
                    ks[3].add(zf * zf);
                    pmax = fmaxf(pmax, sqrtf(px * px + py * py));
                }
                // div z with the zero-extension rule of D^- (z_1 read as zero in
                // the last column, z_2 in the last row)
                const float z1c = (j <= C - 2) ? zc[0] : 0.f;
                const float z1l = (j >= 1) ? sz[0][r][c - 1] : 0.f;
                const float z2c = (i <= R - 2) ? zc[1] : 0.f;
                const float z2u = (i >= 1) ? sz[1][r - 1][c] : 0.f;
                dmax = fmaxf(dmax, fabsf((z1c - z1l) + (z2c - z2u)));
            }
        }
    }
    if (CHECK) {
        double acc[kRedSlots];
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k)
            acc[k] = k < 4 ? ks[k].value() : (k == 4 ? (double)pmax : (k == 5 ? (double)dmax : 0.0));
        block_reduce_store<NT>(acc, partial + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kRedSlots, tid);
    }
}

int tfs_blocks(int R, int C) { return ((C + kTX - 1) / kTX) * ((R + kTY - 1) / kTY); }

cudaError_t launch_tfs_update(const float* pin, float* pout, const float* phi, const float* f1, int R, int C,
                              int pitch, long plane, float t, float delta, bool check, bool write_p,
                              float* tau_out, int tau_pitch, long tau_plane, double* partial, cudaStream_t s) {
    dim3 blk(kTX, kBY), grd((C + kTX - 1) / kTX, (R + kTY - 1) / kTY);
    const bool wt = tau_out != nullptr;
    ProfScope ps((check || !write_p) ? kProfTfsCheck : kProfTfsUpdate, s);
#define TVS_TFS(CK, WP, WT)                                                                              \
    tfs_update_kernel<CK, WP, WT><<<grd, blk, 0, s>>>(pin, pout, phi, f1, R, C, pitch, plane, t, delta, \
                                                      tau_out, tau_pitch, tau_plane, partial)
    if (!check && write_p && !wt) TVS_TFS(false, true, false);
    else if (check && write_p && !wt) TVS_TFS(true, true, false);
    else if (check && !write_p && wt) TVS_TFS(true, false, true);
    else if (check && !write_p && !wt) TVS_TFS(true, false, false);
    else if (!check && !write_p && wt) TVS_TFS(false, false, true);
    else TVS_TFS(true, true, true);
#undef TVS_TFS
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Deterministic second pass of the block partials (fixed order).
// ---------------------------------------------------------------------------
__global__ void finalize_red_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ result) {
    constexpr int NT = 256;
    double acc[kRedSlots];
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) acc[k] = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += NT) {
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) {
            const double v = partial[(size_t)b * kRedSlots + k];
            acc[k] = red_is_max(k) ? fmax(acc[k], v) : acc[k] + v;
        }
    }
    block_reduce_store<NT>(acc, result, threadIdx.x);
}

void carve_red(Carver& cv, RedBuf& rb, int cap) {
    rb.cap = cap;
    rb.partial = cv.take<double>((size_t)cap * kRedSlots);
    rb.result = cv.take<double>(kRedSlots);
    rb.err = cv.take<unsigned>(1);
}

cudaError_t finalize_red(const RedBuf& rb, int nblocks, cudaStream_t s) {
    finalize_red_kernel<<<1, 256, 0, s>>>(rb.partial, nblocks, rb.result);
    return cudaGetLastError();
}

}  // namespace tvs
