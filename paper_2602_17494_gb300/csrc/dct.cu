// DCT-II / DCT-III of arbitrary length and the Neumann Poisson pseudo-inverse
// Delta^dagger = C^T (tilde Delta)^dagger C of eqs. form:DiscInvLapl,
// form:DiscInvLaplTild, eq:DCT2D (Section 4.1).
//
// The extended grid of an N2 x N1 image has (N2+1) x (N1+1) points, so the
// transform lengths are awkward (1025 = 5^2*41, 8193 = 3*2731, ...).  Every
// length L is handled the same way:
//   * Makhoul's reordering turns an L-point DCT-II of real data into one
//     L-point complex DFT; two real lines are packed into one complex DFT and
//     separated afterwards by conjugate symmetry.  The inverse (DCT-III) runs
//     the same steps backwards.
//   * The L-point DFT is Bluestein's chirp-z transform: a circular
//     convolution of length M = 2^m done with two power-of-two FFTs in shared
//     memory (radix-2 decimation in frequency forward -> bit-reversed
//     spectrum -> pointwise filter in bit-reversed order -> decimation in time
//     inverse, so no explicit bit reversal is needed).  The last input sample
//     is added separately (one complex multiply-add per output), which lets the
//     remaining L-1 samples fit a convolution of length M >= 2L-2; for
//     L = 2^k + 1 that is M = 2^(k+1) instead of 2^(k+2).
// Transforms here are unnormalised: the forward gives X'_k = sum_n x_n
// cos(pi (2n+1) k / (2L)) and the inverse is its exact inverse.  The
// orthonormal scalings of C_N cancel in C^T Lambda C because Lambda is
// diagonal, so Delta^dagger = D'^{-1} Lambda D' with the unnormalised pair.
//
// Kernels:
//   dct_rows_fwd  : per pair of rows, optional fused stencil source -> X'
//   dct_cols_solve: per strip of column pairs, forward DCT along y, multiply
//                   by Lambda(k_y, k_x), inverse DCT along y (in place)
//   dct_rows_inv  : per pair of rows, inverse DCT along x (in place)
#include "tvs_internal.cuh"
#include "prof.h"

#include <cmath>
#include <mutex>

namespace tvs {

// --------------------------------------------------------------------------
// Plan tables
// --------------------------------------------------------------------------
int fft_len_for(int L) {
    const int need = 2 * L - 2;
    int m = 2;
    while (m < need) m <<= 1;
    return m;
}

void carve_plan(Carver& cv, DctPlan& pl, int L) {
    pl.L = L;
    pl.M = fft_len_for(L);
    pl.logM = 0;
    while ((1 << pl.logM) < pl.M) ++pl.logM;
    pl.chirp = cv.take<float2>(L);
    pl.rot = cv.take<float2>(L);
    pl.post = cv.take<float2>(L);
    pl.tw = cv.take<float2>(pl.M / 2);
    pl.bhat = cv.take<float2>(pl.M);
}

__global__ void plan_tables_kernel(DctPlan pl) {
    const int L = pl.L, M = pl.M;
    const int n = L > M / 2 ? L : M / 2;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        double s, c;
        if (i < L) {
            const long long q = ((long long)i * (long long)i) % (2LL * L);  // n^2 mod 2L
            sincospi((double)q / (double)L, &s, &c);
            pl.chirp[i] = make_float2((float)c, (float)-s);
            sincospi(2.0 * (double)i / (double)L, &s, &c);
            pl.rot[i] = make_float2((float)c, (float)s);
            sincospi((double)i / (2.0 * (double)L), &s, &c);
            pl.post[i] = make_float2((float)c, (float)-s);
        }
        if (i < M / 2) {
            sincospi(2.0 * (double)i / (double)M, &s, &c);
            pl.tw[i] = make_float2((float)c, (float)-s);
        }
    }
}

// ---- shared-memory FFTs ------------------------------------------------------

// Radix-2 decimation in frequency: natural order in, bit-reversed order out.
// nfft arrays of length M at buf + g * stride.  Two consecutive radix-2 stages
// are done by one thread on four elements (same arithmetic as two separate
// stages, half the passes over shared memory and half the barriers).
__device__ __forceinline__ void fft_dif(float2* buf, int stride, int nfft, int M, int logM,
                                        const float2* __restrict__ tw) {
    int s = 0;
    for (; s + 1 < logM; s += 2) {
        const int lh = logM - 1 - s;          // log2 of the stage-s half length h
        const int h = 1 << lh, q = h >> 1;
        const int per = M >> 2;               // radix-4 butterflies per array
        for (int b = threadIdx.x; b < nfft * per; b += blockDim.x) {
            const int g = b / per;
            const int r = b - g * per;
            const int grp = r >> (lh - 1);    // r / q
            const int pos = r & (q - 1);
            float2* x = buf + (size_t)g * stride + grp * 2 * h + pos;
            const float2 a = x[0], bb = x[q], c = x[h], d = x[h + q];
            const float2 a1 = c_add(a, c);
            const float2 c1 = c_mul(c_sub(a, c), __ldg(&tw[pos << s]));
            const float2 b1 = c_add(bb, d);
            const float2 d1 = c_mul(c_sub(bb, d), __ldg(&tw[(pos + q) << s]));
            const float2 w2 = __ldg(&tw[pos << (s + 1)]);
            x[0] = c_add(a1, b1);
            x[q] = c_mul(c_sub(a1, b1), w2);
            x[h] = c_add(c1, d1);
            x[h + q] = c_mul(c_sub(c1, d1), w2);
        }
        __syncthreads();
    }
    if (s < logM) {                           // last stage (h = 1) when logM is odd
        const int halfM = M >> 1;
        for (int b = threadIdx.x; b < nfft * halfM; b += blockDim.x) {
            const int g = b / halfM;
            const int r = b - g * halfM;
            float2* x = buf + (size_t)g * stride + 2 * r;
            const float2 u = x[0], v = x[1];
            x[0] = c_add(u, v);
            x[1] = c_sub(u, v);
        }
        __syncthreads();
    }
}

// Radix-2 decimation in time with conjugate twiddles (unnormalised inverse):
// bit-reversed order in, natural order out; stages fused in pairs as above.
__device__ __forceinline__ void ifft_dit(float2* buf, int stride, int nfft, int M, int logM,
                                         const float2* __restrict__ tw) {
    int s = 0;
    if (logM & 1) {                           // first stage (h = 1) when logM is odd
        const int halfM = M >> 1;
        for (int b = threadIdx.x; b < nfft * halfM; b += blockDim.x) {
            const int g = b / halfM;
            const int r = b - g * halfM;
            float2* x = buf + (size_t)g * stride + 2 * r;
            const float2 u = x[0], v = x[1];
            x[0] = c_add(u, v);
            x[1] = c_sub(u, v);
        }
        __syncthreads();
        s = 1;
    }
    for (; s + 1 < logM; s += 2) {
        const int h = 1 << s;                 // stage-s half length; stage s+1 uses 2h
        const int per = M >> 2;
        for (int b = threadIdx.x; b < nfft * per; b += blockDim.x) {
            const int g = b / per;
            const int r = b - g * per;
            const int grp = r >> s;           // r / h
            const int pos = r & (h - 1);
            float2* x = buf + (size_t)g * stride + grp * 4 * h + pos;
            const float2 w1 = __ldg(&tw[pos << (logM - 1 - s)]);
            const float2 a = x[0];
            const float2 tb = c_mulconj(x[h], w1);
            const float2 c = x[2 * h];
            const float2 td = c_mulconj(x[3 * h], w1);
            const float2 a1 = c_add(a, tb), b1 = c_sub(a, tb);
            const float2 c1 = c_add(c, td), d1 = c_sub(c, td);
            const float2 tc = c_mulconj(c1, __ldg(&tw[pos << (logM - 2 - s)]));
            const float2 tdd = c_mulconj(d1, __ldg(&tw[(pos + h) << (logM - 2 - s)]));
            x[0] = c_add(a1, tc);
            x[2 * h] = c_sub(a1, tc);
            x[h] = c_add(b1, tdd);
            x[3 * h] = c_sub(b1, tdd);
        }
        __syncthreads();
    }
}

// Chirp filter spectrum: b[m] = conj(c_m) for lags m in [-(L-2), L-1] stored
// circularly, FFT'd (bit-reversed order) and scaled by 1/M.  One block.
__global__ void plan_bhat_kernel(DctPlan pl) {
    extern __shared__ float2 sm[];
    const int L = pl.L, M = pl.M;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        int lag = -1;
        if (m <= L - 1) lag = m;
        else if (m >= M - (L - 2)) lag = M - m;
        float2 v = make_float2(0.f, 0.f);
        if (lag >= 0) {
            const long long q = ((long long)lag * (long long)lag) % (2LL * L);
            double s, c;
            sincospi((double)q / (double)L, &s, &c);
            v = make_float2((float)c, (float)s);  // conj(exp(-i pi lag^2 / L))
        }
        sm[m] = v;
    }
    __syncthreads();
    fft_dif(sm, M, 1, M, pl.logM, pl.tw);
    const float inv = 1.0f / (float)M;
    for (int m = threadIdx.x; m < M; m += blockDim.x)
        pl.bhat[m] = make_float2(sm[m].x * inv, sm[m].y * inv);
}

cudaError_t build_plan(const DctPlan& pl, cudaStream_t s) {
    const int n = pl.L > pl.M / 2 ? pl.L : pl.M / 2;
    plan_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(pl);
    const size_t smem = (size_t)pl.M * sizeof(float2);
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(plan_bhat_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmemBudget);
    });
    plan_bhat_kernel<<<1, kFftThreads, smem, s>>>(pl);
    return cudaGetLastError();
}

void carve_poisson(Carver& cv, PoissonPlans& pp, int rows, int cols) {
    carve_plan(cv, pp.row, cols);
    carve_plan(cv, pp.col, rows);
}

cudaError_t build_poisson(const PoissonPlans& pp, cudaStream_t s) {
    cudaError_t e = build_plan(pp.row, s);
    if (e != cudaSuccess) return e;
    return build_plan(pp.col, s);
}

// --------------------------------------------------------------------------
// Bluestein core: buf[g][0 .. L-2] holds the chirped input a_n = z_n c_n,
// buf[g][L-1 .. M) is zero and peel[g] = z_{L-1}.  On return buf[g][k] =
// Z_k = sum_n z_n exp(-2 pi i n k / L) for k < L.
// --------------------------------------------------------------------------
__device__ void bluestein(float2* buf, int stride, int G, const DctPlan& pl, const float2* peel) {
    const int L = pl.L, M = pl.M;
    fft_dif(buf, stride, G, M, pl.logM, pl.tw);
    for (int b = threadIdx.x; b < G * M; b += blockDim.x) {
        const int g = b >> pl.logM;
        const int k = b & (M - 1);
        float2* x = buf + (size_t)g * stride + k;
        *x = c_mul(*x, __ldg(&pl.bhat[k]));
    }
    __syncthreads();
    ifft_dit(buf, stride, G, M, pl.logM, pl.tw);
    for (int b = threadIdx.x; b < G * L; b += blockDim.x) {
        const int g = b / L;
        const int k = b - g * L;
        float2* x = buf + (size_t)g * stride + k;
        *x = c_add(c_mul(__ldg(&pl.chirp[k]), *x), c_mul(peel[g], __ldg(&pl.rot[k])));
    }
    __syncthreads();
}

// Makhoul's reordering: position of input sample j in the reordered line.
__device__ __forceinline__ int mk_perm(int j, int L) { return (j & 1) ? (L - 1 - (j >> 1)) : (j >> 1); }

// Stage one packed complex sample z (position n of the reordered line).
__device__ __forceinline__ void stage_sample(float2* bufg, float2* peelg, int n, int L, float2 z,
                                            const DctPlan& pl) {
    if (n == L - 1) *peelg = z;
    else bufg[n] = c_mul(z, __ldg(&pl.chirp[n]));
}

__device__ __forceinline__ void zero_tail(float2* buf, int stride, int G, int L, int M) {
    const int t = M - (L - 1);
    for (int b = threadIdx.x; b < G * t; b += blockDim.x) {
        const int g = b / t;
        buf[(size_t)g * stride + (L - 1) + (b - g * t)] = make_float2(0.f, 0.f);
    }
}

// Separate two real lines packed as z = x1 + i x2 from Z = DFT(z) and return
// the unnormalised DCT-II values X'_k of both lines.
__device__ __forceinline__ float2 unpack_dct2(const float2* bufg, int k, int L, const DctPlan& pl) {
    const float2 zk = bufg[k];
    const float2 zm = bufg[k == 0 ? 0 : L - k];
    const float2 v1 = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    const float2 v2 = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    const float2 w = __ldg(&pl.post[k]);
    return make_float2(w.x * v1.x - w.y * v1.y, w.x * v2.x - w.y * v2.y);
}

// Input of the inverse: conj(Z_k) with Z = V1 + i V2, V = e^{i pi k/2L}(X_k - i X_{L-k}).
__device__ __forceinline__ float2 pack_dct3(float x1k, float x1m, float x2k, float x2m, int k,
                                            const DctPlan& pl) {
    const float2 w = __ldg(&pl.post[k]);  // e^{-i pi k / 2L}; we need its conjugate
    // V1 = conj(w) * (x1k - i x1m)
    const float2 v1 = make_float2(w.x * x1k - w.y * x1m, -w.x * x1m - w.y * x1k);
    const float2 v2 = make_float2(w.x * x2k - w.y * x2m, -w.x * x2m - w.y * x2k);
    const float2 z = make_float2(v1.x - v2.y, v1.y + v2.x);
    return c_conj(z);
}

// --------------------------------------------------------------------------
// Row sources (stencils evaluated on the fly; Section 4.1 operators)
// --------------------------------------------------------------------------
struct Fld {
    const float* a;
    int pitch;
    __device__ __forceinline__ float operator()(int r, int c) const { return __ldg(&a[(size_t)r * pitch + c]); }
};

// D^-_x u at (r, c) on a grid with C columns.
template <class F>
__device__ __forceinline__ float dxm_at(const F& u, int r, int c, int C) {
    if (c == 0) return u(r, 0);
    if (c == C - 1) return -u(r, C - 2);
    return u(r, c) - u(r, c - 1);
}
template <class F>
__device__ __forceinline__ float dym_at(const F& u, int r, int c, int R) {
    if (r == 0) return u(0, c);
    if (r == R - 1) return -u(R - 2, c);
    return u(r, c) - u(r - 1, c);
}

struct DivOf {  // div of the 2-plane field (ux, uy)
    Fld ux, uy;
    int R, C;
    __device__ __forceinline__ float operator()(int r, int c) const {
        return dxm_at(ux, r, c, C) + dym_at(uy, r, c, R);
    }
};

template <RowSource SRC>
__device__ __forceinline__ float row_source(const RowSrcArgs& sa, int r, int c, int R, int C) {
    if (SRC == RowSource::Plain) {
        return __ldg(&sa.a[(size_t)r * sa.pitch + c]);
    } else if (SRC == RowSource::DivField) {
        DivOf d{Fld{sa.a, sa.pitch}, Fld{sa.a + sa.plane, sa.pitch}, R, C};
        return d(r, c);
    } else {
        // s = div(vecdiv p) = D-x w1 + D-y w2, w_k = div(p_kx, p_ky)
        DivOf w1{Fld{sa.a, sa.pitch}, Fld{sa.a + sa.plane, sa.pitch}, R, C};
        DivOf w2{Fld{sa.a + 2 * sa.plane, sa.pitch}, Fld{sa.a + 3 * sa.plane, sa.pitch}, R, C};
        return dxm_at(w1, r, c, C) + dym_at(w2, r, c, R);
    }
}

// --------------------------------------------------------------------------
// Kernels
// --------------------------------------------------------------------------
// Batch mode (Schwarz step 1): blockIdx.y selects one of several arrays spaced
// `bstride` floats apart; `ranges[b]` = (first row, end row) restricts the
// transform to the rows a subdomain touches.  ranges == nullptr: all rows.
// With `packed`, array b stores only its rows: row r lives at storage row
// r - ranges[b].x.
struct BatchArgs {
    const int2* ranges;
    long bstride;
    int packed;
};

__device__ __forceinline__ int2 batch_rows(const BatchArgs& ba, int rows) {
    return ba.ranges ? ba.ranges[blockIdx.y] : make_int2(0, rows);
}
__device__ __forceinline__ size_t row_off(const BatchArgs& ba, int2 rr, int r, int pitch) {
    return (size_t)(ba.packed ? r - rr.x : r) * pitch;
}

template <RowSource SRC>
__global__ void __launch_bounds__(kFftThreads)
dct_rows_fwd_kernel(float* __restrict__ out, int rows, int cols, int pitch, DctPlan pl, RowSrcArgs sa,
                    int G, BatchArgs ba) {
    extern __shared__ float2 sm[];
    const int L = cols, M = pl.M, stride = M + 4;
    float2* buf = sm;
    float2* peel = sm + (size_t)G * stride;
    const int2 rr = batch_rows(ba, rows);
    out += (size_t)blockIdx.y * ba.bstride;
    sa.a += (size_t)blockIdx.y * ba.bstride;
    const int npairs = (rr.y - rr.x + 1) >> 1;
    for (int base = blockIdx.x * G; base < npairs; base += gridDim.x * G) {
        const int gc = min(G, npairs - base);
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int g = b / L;
            const int j = b - g * L;
            const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
            float x0, x1;
            if (SRC == RowSource::Plain) {
                x0 = __ldg(&sa.a[row_off(ba, rr, r0, sa.pitch) + j]);
                x1 = (r1 < rr.y) ? __ldg(&sa.a[row_off(ba, rr, r1, sa.pitch) + j]) : 0.f;
            } else {
                x0 = row_source<SRC>(sa, r0, j, rows, cols);
                x1 = (r1 < rr.y) ? row_source<SRC>(sa, r1, j, rows, cols) : 0.f;
            }
            stage_sample(buf + (size_t)g * stride, peel + g, mk_perm(j, L), L, make_float2(x0, x1), pl);
        }
        zero_tail(buf, stride, gc, L, M);
        __syncthreads();
        bluestein(buf, stride, gc, pl, peel);
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int g = b / L;
            const int k = b - g * L;
            const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
            const float2 X = unpack_dct2(buf + (size_t)g * stride, k, L, pl);
            out[row_off(ba, rr, r0, pitch) + k] = X.x;
            if (r1 < rr.y) out[row_off(ba, rr, r1, pitch) + k] = X.y;
        }
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kFftThreads)
dct_rows_inv_kernel(float* __restrict__ S, int rows, int cols, int pitch, DctPlan pl, int G, BatchArgs ba) {
    extern __shared__ float2 sm[];
    const int L = cols, M = pl.M, stride = M + 4;
    float2* buf = sm;
    float2* peel = sm + (size_t)G * stride;
    const int2 rr = batch_rows(ba, rows);
    S += (size_t)blockIdx.y * ba.bstride;
    const int npairs = (rr.y - rr.x + 1) >> 1;
    const float invL = 1.0f / (float)L;
    for (int base = blockIdx.x * G; base < npairs; base += gridDim.x * G) {
        const int gc = min(G, npairs - base);
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int g = b / L;
            const int k = b - g * L;
            const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
            const float* a0 = S + row_off(ba, rr, r0, pitch);
            const float x1k = a0[k], x1m = k ? a0[L - k] : 0.f;
            float x2k = 0.f, x2m = 0.f;
            if (r1 < rr.y) {
                const float* a1 = S + row_off(ba, rr, r1, pitch);
                x2k = a1[k];
                x2m = k ? a1[L - k] : 0.f;
            }
            stage_sample(buf + (size_t)g * stride, peel + g, k, L, pack_dct3(x1k, x1m, x2k, x2m, k, pl), pl);
        }
        zero_tail(buf, stride, gc, L, M);
        __syncthreads();
        bluestein(buf, stride, gc, pl, peel);
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int g = b / L;
            const int j = b - g * L;
            const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
            const float2 Y = buf[(size_t)g * stride + mk_perm(j, L)];
            S[row_off(ba, rr, r0, pitch) + j] = Y.x * invL;
            if (r1 < rr.y) S[row_off(ba, rr, r1, pitch) + j] = -Y.y * invL;
        }
        __syncthreads();
    }
}

// Lambda(ky, kx) = -1 / (sigma_{R,ky}^2 + sigma_{C,kx}^2), 0 at (0, 0):
// the row frequency pairs with the row count (see the oracle's reading).
__device__ __forceinline__ float lap_symbol(int ky, int kx, int R, int C) {
    const float sy = 2.0f * sinpif((float)ky / (2.0f * (float)R));
    const float sx = 2.0f * sinpif((float)kx / (2.0f * (float)C));
    const float den = sy * sy + sx * sx;
    return den > 0.f ? -1.0f / den : 0.f;
}

__global__ void __launch_bounds__(kFftThreads)
dct_cols_solve_kernel(float* __restrict__ S, int rows, int cols, int pitch, DctPlan pl, int G, BatchArgs ba) {
    extern __shared__ float2 sm[];
    const int2 rr = batch_rows(ba, rows);       // rows outside rr are read as zero and not written
    S += (size_t)blockIdx.y * ba.bstride;
    const int L = rows, M = pl.M, stride = M + 4;
    float2* buf = sm;
    float2* ybuf = sm + (size_t)G * stride;       // G x L staged spectra
    float2* peel = ybuf + (size_t)G * L;
    const int npairs = (cols + 1) >> 1;
    const float invL = 1.0f / (float)L;
    for (int base = blockIdx.x * G; base < npairs; base += gridDim.x * G) {
        const int gc = min(G, npairs - base);
        // load with the pair index fastest so that a warp reads contiguous row segments
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int r = b / gc;
            const int g = b - r * gc;
            const int c0 = 2 * (base + g);
            const bool in = r >= rr.x && r < rr.y;
            const float* a = in ? S + row_off(ba, rr, r, pitch) + c0 : S;
            const float x0 = in ? a[0] : 0.f;
            const float x1 = (in && c0 + 1 < cols) ? a[1] : 0.f;
            stage_sample(buf + (size_t)g * stride, peel + g, mk_perm(r, L), L, make_float2(x0, x1), pl);
        }
        zero_tail(buf, stride, gc, L, M);
        __syncthreads();
        bluestein(buf, stride, gc, pl, peel);
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int g = b / L;
            const int k = b - g * L;
            const int c0 = 2 * (base + g);
            const float2 X = unpack_dct2(buf + (size_t)g * stride, k, L, pl);
            ybuf[(size_t)g * L + k] = make_float2(X.x * lap_symbol(k, c0, rows, cols),
                                                  X.y * lap_symbol(k, c0 + 1, rows, cols));
        }
        __syncthreads();
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int g = b / L;
            const int k = b - g * L;
            const float2 yk = ybuf[(size_t)g * L + k];
            const float2 ym = k ? ybuf[(size_t)g * L + L - k] : make_float2(0.f, 0.f);
            stage_sample(buf + (size_t)g * stride, peel + g, k, L, pack_dct3(yk.x, ym.x, yk.y, ym.y, k, pl), pl);
        }
        zero_tail(buf, stride, gc, L, M);
        __syncthreads();
        bluestein(buf, stride, gc, pl, peel);
        for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
            const int r = b / gc;
            const int g = b - r * gc;
            const int c0 = 2 * (base + g);
            if (r < rr.x || r >= rr.y) continue;
            const float2 Y = buf[(size_t)g * stride + mk_perm(r, L)];
            float* a = S + row_off(ba, rr, r, pitch) + c0;
            a[0] = Y.x * invL;
            if (c0 + 1 < cols) a[1] = -Y.y * invL;
        }
        __syncthreads();
    }
}

// --------------------------------------------------------------------------
// Host launchers
// --------------------------------------------------------------------------
namespace {
template <class K>
void allow_smem(K kernel) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget + 16 * 1024);
}
std::once_flag g_smem_once;
void set_all_smem_attrs() {
    allow_smem(dct_rows_fwd_kernel<RowSource::Plain>);
    allow_smem(dct_rows_fwd_kernel<RowSource::DivField>);
    allow_smem(dct_rows_fwd_kernel<RowSource::DivVecdiv>);
    allow_smem(dct_rows_inv_kernel);
    allow_smem(dct_cols_solve_kernel);
}
int blocks_for(int units, int G) {
    const int b = (units + G - 1) / G;
    return b > 0 ? b : 1;
}
}  // namespace

// Lines per CTA: one pair (the kernels are latency-bound, so resident warps
// matter more than batching); threads: one radix-4 butterfly per thread and pass.
int pick_batch(int units, size_t per_line) {
    (void)units;
    (void)per_line;
    return 1;
}
int fft_threads(int M) {
    int t = M / 4;
    if (t < 128) t = 128;
    if (t > 1024) t = 1024;
    return t;
}

static cudaError_t poisson_launch(float* S, int rows, int cols, int pitch, const PoissonPlans& pp, RowSource src,
                                  const RowSrcArgs& sa, int nbatch, const int2* ranges, long bstride, int maxrows,
                                  int packed, cudaStream_t s) {
    std::call_once(g_smem_once, set_all_smem_attrs);
    const BatchArgs ba{ranges, bstride, packed};
    const int rpairs = (maxrows + 1) / 2, cpairs = (cols + 1) / 2;
    const int units_r = rpairs * nbatch, units_c = cpairs * nbatch;
    {
        const size_t per = (size_t)(pp.row.M + 4 + 1) * sizeof(float2);
        const int G = pick_batch(units_r, per);
        const size_t smem = (size_t)G * per;
        const dim3 grid(blocks_for(rpairs, G), nbatch);
        const int nt = fft_threads(pp.row.M);
        ProfScope ps(kProfRowsFwd, s);
        switch (src) {
            case RowSource::Plain:
                dct_rows_fwd_kernel<RowSource::Plain><<<grid, nt, smem, s>>>(S, rows, cols, pitch, pp.row, sa, G, ba);
                break;
            case RowSource::DivField:
                dct_rows_fwd_kernel<RowSource::DivField><<<grid, nt, smem, s>>>(S, rows, cols, pitch, pp.row, sa, G, ba);
                break;
            case RowSource::DivVecdiv:
                dct_rows_fwd_kernel<RowSource::DivVecdiv><<<grid, nt, smem, s>>>(S, rows, cols, pitch, pp.row, sa, G, ba);
                break;
        }
    }
    {
        const size_t per = (size_t)(pp.col.M + 4 + rows + 1) * sizeof(float2);
        const int G = pick_batch(units_c, per);
        const size_t smem = (size_t)G * per;
        ProfScope ps(kProfCols, s);
        dct_cols_solve_kernel<<<dim3(blocks_for(cpairs, G), nbatch), fft_threads(pp.col.M), smem, s>>>(
            S, rows, cols, pitch, pp.col, G, ba);
    }
    {
        const size_t per = (size_t)(pp.row.M + 4 + 1) * sizeof(float2);
        const int G = pick_batch(units_r, per);
        const size_t smem = (size_t)G * per;
        ProfScope ps(kProfRowsInv, s);
        dct_rows_inv_kernel<<<dim3(blocks_for(rpairs, G), nbatch), fft_threads(pp.row.M), smem, s>>>(
            S, rows, cols, pitch, pp.row, G, ba);
    }
    return cudaGetLastError();
}

cudaError_t poisson_solve(float* S, int rows, int cols, int pitch, const PoissonPlans& pp,
                          RowSource src, const RowSrcArgs& sa, cudaStream_t s) {
    return poisson_launch(S, rows, cols, pitch, pp, src, sa, 1, nullptr, 0, rows, 0, s);
}

cudaError_t poisson_solve_batched(float* S, int nbatch, long bstride, const int2* ranges, int maxrows, int rows,
                                  int cols, int pitch, const PoissonPlans& pp, cudaStream_t s) {
    RowSrcArgs sa{S, 0, pitch};
    return poisson_launch(S, rows, cols, pitch, pp, RowSource::Plain, sa, nbatch, ranges, bstride, maxrows, 1, s);
}

}  // namespace tvs
