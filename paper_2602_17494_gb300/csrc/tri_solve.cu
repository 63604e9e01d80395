// Column pass of the Neumann Poisson pseudo-inverse as tridiagonal solves
// (eqs. form:DiscInvLapl, form:DiscInvLaplTild, Section 4.1).
//
// After the forward DCT along x (dct_rows_fwd), the pseudo-inverse acts on
// column k_x of the spectrum as D'^{-1} Lambda(:, k_x) D' along y, with D' the
// unnormalised DCT-II pair of length L = rows.  D' diagonalises the Neumann
// second difference
//   T = tridiag(-1, 2, -1) with 1 in both corners,  eigenvalues sigma_{R,k}^2,
// so that operator is exactly
//   -(T + lambda I)^{-1},  lambda = sigma_{C,k_x}^2 > 0        (k_x >= 1),
//   -T^dagger (zero-mean input part dropped, zero-mean output) (k_x = 0).
// Two more DCTs per column cost O(L log L) with Bluestein lengths 2L; the
// system itself is solved here in O(L).  With r + 1/r = 2 + lambda, 0 < r < 1
// and S the shift (S x)_i = x_{i-1},
//   T + lambda I = r^{-1} (1 - r S)(1 - r S^{-1})
// on the integers.  The Neumann rows are the interior rows applied to the
// half-sample symmetric extension of b (period 2L), whose bounded solution
// keeps that symmetry, so the two first-order recursions get closed-form
// start values:
//   c_i = b_i + r c_{i-1},  c_{-1} = sum_j b_j (r^j + r^{2L-1-j}) / (1 - r^{2L}),
//   w_i = c_i + r w_{i+1},  w_{L-1} = c_{L-1} / (1 - r)   (from w_L = w_{L-1}),
//   y = -r w.
// For k_x = 0 (r = 1) the input loses its mean, c_{-1} = 0, w_L = 0 and the
// output loses its mean.  1 - r is carried as q = (sqrt(lambda (4 + lambda))
// - lambda) / 2, which has no cancellation, and every recursion step is
// x + s - q s, so the solved system is the one for lambda up to rounding of q
// even where r is within 1e-3 of 1.  q and the powers of r that do not depend
// on the thread come from a per-column table built in FP64 with the plan.
//
// Chunked form (long columns, one unbatched problem): the rows are cut into
// chunks of kTriChunk = 32 and every kernel maps a warp to 32 adjacent
// columns of one chunk, so each row access is one coalesced 128-byte line.
// Both recursions are linear, so a chunk is summarised by values computed
// from a zero carry: its Horner sum h = sum_i r^(i-i0) b_i, its causal end
// value a, and g = sum_i r^(i-i0) c_i over its causal values c from zero.
//   tri_chunk_sum_kernel  : h, a, g per (chunk, column)
//   tri_chunk_scan_kernel : per column, c_{-1} and w_L from the h and a sums,
//                           the causal carry into every chunk (C_c) and the
//                           anti-causal carry after it (W_c), using
//                           w_{i0} = g_c + C_c sum_{m<n} r^(2m+1) + r^n W_c
//   tri_chunk_apply_kernel: re-reads the chunk and runs both recursions from
//                           its carries.
// Traffic is read, read + write (12 bytes per point) against 8 for the
// one-pass kernel below, but every access is a full line; at 8193 rows the
// one-pass kernel's strided 8-byte accesses are latency-bound.  For k_x = 0
// the input mean mu and the output mean enter as corrections of the
// summaries: a -> a - mu n, g -> g - mu n(n+1)/2, and the output mean of
// w is sum_c (K_c + C_c n(n+1)/2 + n W_c) / L with K_c = sum_i (i-i0+1) c_i.
//
// Parallel form of the one-pass kernel: one CTA per column pair (the pair is
// one 8-byte access per row), each thread N consecutive rows of both columns
// in registers.  The
// recursions run over the N rows in registers; the chunk carries combine with
// the constant multiplier r^N as Kogge-Stone scans within a warp and a short
// serial pass over the warps' totals.  The start value c_{-1} and c_{L-1} come
// from two block sums, so the whole solve needs two barriers (two more in the
// CTA holding k_x = 0).
#include "dct_launch.h"

namespace tvs {
namespace {

constexpr int kTriThreads = 256;   // threads per CTA at most (rows per thread chosen to fit)
constexpr int kTriWarps = kTriThreads / 32;

__device__ __forceinline__ float2 f2(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
// x + s - q s, one step of a recursion with r = 1 - q (nq = -q)
__device__ __forceinline__ float2 rstep(float2 s, float2 x, float2 nq) { return fma2(nq, s, add2(s, x)); }
// r^k of both columns from l2 = log2 r
__device__ __forceinline__ float2 rpow(float2 l2, int k) {
    const float kf = (float)k;
    return f2(exp2f(kf * l2.x), exp2f(kf * l2.y));
}
__device__ __forceinline__ float2 shfl_up2(float2 v, int d) {
    return f2(__shfl_up_sync(0xffffffffu, v.x, d), __shfl_up_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 shfl_down2(float2 v, int d) {
    return f2(__shfl_down_sync(0xffffffffu, v.x, d), __shfl_down_sync(0xffffffffu, v.y, d));
}
__device__ __forceinline__ float2 warp_sum2(float2 v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = add2(v, f2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o)));
    return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Removes the mean over rows [0, L) of the first column (the k_x = 0 column of
// the CTA with blockIdx.x == 0).  Rows >= L stay zero.
template <int N>
__device__ __forceinline__ void remove_mean_x(float2 (&v)[N], int row0, int L, float* sh, int lane, int wid, int nw) {
    float s = 0.f;
#pragma unroll
    for (int i = 0; i < N; ++i) s += v[i].x;
    s = warp_sum(s);
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    float tot = 0.f;
    for (int w = 0; w < nw; ++w) tot += sh[w];
    const float mean = tot / (float)L;
#pragma unroll
    for (int i = 0; i < N; ++i)
        if (row0 + i < L) v[i].x -= mean;
}

// S: the row-transformed planes (in place); rows = L; tab: build_tri_table(rows, cols).
// Batch mode as in the DCT kernels: blockIdx.y selects the array, rows outside
// batch_rows() are zero on input and not written.
template <int N>
__global__ void __launch_bounds__(kTriThreads)
tri_cols_solve_kernel(float* __restrict__ S, int rows, int cols, int pitch, const float4* __restrict__ tab,
                      const __grid_constant__ BatchArgs ba) {
    __shared__ float2 sh_fwd[kTriWarps], sh_s1[kTriWarps], sh_r2[kTriWarps], sh_bwd[kTriWarps];
    __shared__ float sh_m0[kTriWarps], sh_m1[kTriWarps];
    pdl_wait();
    pdl_trigger();
    const int2 rr = batch_rows(ba, rows);
    S += (size_t)blockIdx.y * ba.bstride;
    const int L = rows;
    const int c0 = 2 * blockIdx.x;
    const bool has1 = c0 + 1 < cols;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int row0 = threadIdx.x * N;
    const bool zero_mode = blockIdx.x == 0;  // column 0 is k_x = 0

    // per-column coefficients (a missing second column reuses the first's)
    const float4 a0 = __ldg(&tab[2 * c0]), b0 = __ldg(&tab[2 * c0 + 1]);
    const float4 a1 = has1 ? __ldg(&tab[2 * c0 + 2]) : a0, b1 = has1 ? __ldg(&tab[2 * c0 + 3]) : b0;
    const float2 q = f2(a0.x, a1.x), nq = f2(-a0.x, -a1.x);
    const float2 l2 = f2(a0.y, a1.y);   // log2 r
    const float2 m = f2(a0.z, a1.z);    // r^N
    const float2 m32 = f2(a0.w, a1.w);  // r^(32 N)
    const float2 rL = f2(b0.x, b1.x);   // r^L
    const float2 dnm = f2(b0.y, b1.y);  // 1 / (1 - r^(2L)), 0 for k_x = 0
    const float2 iq = f2(b0.z, b1.z);   // 1 / q, 0 for k_x = 0

    float2 v[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int r = row0 + i;
        float2 x = f2(0.f, 0.f);
        if (r >= rr.x && r < rr.y) {
            // with an even pitch the pair (c0, c0 + 1) is one 8-byte load; c0 + 1
            // is inside the row's storage even when it is the padding column
            const float* a = S + row_off(ba, rr, r, pitch) + c0;
            if ((pitch & 1) == 0) x = *reinterpret_cast<const float2*>(a);
            else x = f2(a[0], has1 ? a[1] : 0.f);
        }
        if (!has1) x.y = 0.f;
        v[i] = x;
    }
    if (zero_mode) remove_mean_x<N>(v, row0, L, sh_m0, lane, wid, nw);

    // sum_j b_j r^j over the chunk (Horner), then the causal recursion from zero
    float2 h = f2(0.f, 0.f);
#pragma unroll
    for (int i = N - 1; i >= 0; --i) h = rstep(h, v[i], nq);
    const float2 s1 = mul2(rpow(l2, row0), h);
    const int e = min(L - 1, row0 + N - 1);  // last row of the chunk (below row0 when the chunk is empty)
    // r^(L-1-e) = r^(L - min(L, row0 + N)): from the chunk's end to row L - 1, and from row L to the chunk's end
    const float2 rt = rpow(l2, L - min(L, row0 + N));
    float2 p = f2(0.f, 0.f), a = f2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < N; ++i) {
        p = rstep(p, v[i], nq);
        if (row0 + i == e) a = p;
        v[i] = row0 + i < L ? p : f2(0.f, 0.f);
    }
    // c0_{L-1} = sum over chunks of r^{L-1-e} a
    const float2 r2 = mul2(rt, a);

    // forward scan of the chunk carries within the warp (multiplier r^N)
    float2 f = a, md = m;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float2 y = shfl_up2(f, d);
        if (lane >= d) f = fma2(md, y, f);
        md = mul2(md, md);
    }
    const float2 s1w = warp_sum2(s1), r2w = warp_sum2(r2);
    if (lane == 31) sh_fwd[wid] = f;
    if (lane == 0) {
        sh_s1[wid] = s1w;
        sh_r2[wid] = r2w;
    }
    __syncthreads();
    float2 cw = f2(0.f, 0.f), S1 = f2(0.f, 0.f), R2 = f2(0.f, 0.f);
    for (int w = 0; w < nw; ++w) {
        if (w < wid) cw = fma2(m32, cw, sh_fwd[w]);
        S1 = add2(S1, sh_s1[w]);
        R2 = add2(R2, sh_r2[w]);
    }
    // start values: u0 = c_{-1}, cL = c_{L-1}, wL = w_L (all zero for k_x = 0)
    const float2 u0 = mul2(fma2(rL, R2, S1), dnm);
    const float2 cL = fma2(rL, u0, R2);
    const float2 wL = mul2(cL, iq);

    // true causal values: carry into the chunk = in-warp prefix + warp carry + u0
    float2 fex = shfl_up2(f, 1);
    if (lane == 0) fex = f2(0.f, 0.f);
    p = fma2(rpow(l2, row0), u0, fma2(rpow(l2, lane * N), cw, fex));
#pragma unroll
    for (int i = 0; i < N; ++i) {
        p = fma2(nq, p, p);
        if (row0 + i < L) v[i] = add2(v[i], p);
    }

    // anti-causal recursion from zero, then its scan (reversed, multiplier r^N)
    p = f2(0.f, 0.f);
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        p = rstep(p, v[i], nq);
        v[i] = p;
    }
    float2 g = v[0];
    md = m;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const float2 y = shfl_down2(g, d);
        if (lane + d < 32) g = fma2(md, y, g);
        md = mul2(md, md);
    }
    if (lane == 0) sh_bwd[wid] = g;
    __syncthreads();
    float2 cb = f2(0.f, 0.f);
    for (int w = nw - 1; w > wid; --w) cb = fma2(m32, cb, sh_bwd[w]);
    float2 gex = shfl_down2(g, 1);
    if (lane == 31) gex = f2(0.f, 0.f);
    // carry into the chunk from the right: w at row min(L, row0 + N)
    p = fma2(rt, wL, fma2(rpow(l2, (31 - lane) * N), cb, gex));
#pragma unroll
    for (int i = N - 1; i >= 0; --i) {
        if (row0 + i < L) {
            p = fma2(nq, p, p);
            v[i] = add2(v[i], p);
        }
    }
    if (zero_mode) remove_mean_x<N>(v, row0, L, sh_m1, lane, wid, nw);

    // y = -r w = q w - w
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const int r = row0 + i;
        if (r < rr.x || r >= rr.y) continue;
        const float2 y = fma2(q, v[i], f2(-v[i].x, -v[i].y));
        float* o = S + row_off(ba, rr, r, pitch) + c0;
        if (has1 && (pitch & 1) == 0) {
            *reinterpret_cast<float2*>(o) = y;
        } else {
            o[0] = y.x;
            if (has1) o[1] = y.y;
        }
    }
}

// Per-column coefficients in FP64 for a column pass of `rows` rows over
// `cols` x frequencies (lambda = sigma_{C,k}^2 = 4 sin^2(pi k / (2 cols))):
//   tab[2k]     = (q, log2 r, r^N, r^(32 N)),
//   tab[2k + 1] = (r^rows, 1 / (1 - r^(2 rows)), 1 / q, 0),
// with k = 0 stored as r = 1 and both start-value factors zero.
__global__ void tri_table_kernel(float4* __restrict__ tab, int rows, int cols, int N) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= cols) return;
    if (k == 0) {
        tab[0] = make_float4(0.f, 0.f, 1.f, 1.f);
        tab[1] = make_float4(1.f, 0.f, 0.f, 0.f);
        return;
    }
    double sn, cs;
    sincospi((double)k / (2.0 * (double)cols), &sn, &cs);
    const double lam = 4.0 * sn * sn;
    const double q = 0.5 * (sqrt(lam * (4.0 + lam)) - lam);
    const double lr = log1p(-q);  // ln r
    tab[2 * k] = make_float4((float)q, (float)(lr / 0.69314718055994531), (float)exp((double)N * lr),
                             (float)exp(32.0 * (double)N * lr));
    tab[2 * k + 1] = make_float4((float)exp((double)rows * lr), (float)(-1.0 / expm1(2.0 * (double)rows * lr)),
                                 (float)(1.0 / q), 0.f);
}

// Rows per thread: the fewest that keep the CTA within kTriThreads (0: too long).
int rows_per_thread(int rows) {
    for (int n : {3, 5, 9, 17, 33})
        if (rows <= n * kTriThreads) return n;
    return 0;
}

template <int N>
cudaError_t launch_n(float* S, int rows, int cols, int pitch, const float4* tab, const BatchArgs& ba, int nbatch,
                     cudaStream_t s) {
    const int threads = round_up((rows + N - 1) / N, 32);
    return launch_pdl(tri_cols_solve_kernel<N>, dim3((cols + 1) / 2, nbatch), dim3(threads), 0, s, S, rows, cols,
                      pitch, tab, ba);
}

// ---------------------------------------------------------------------------
// Chunked solve of long columns (see the header).  Summary planes in pp.tsum,
// each [chunk][column]: 0 h, 1 a, 2 g, 3 C (causal carry into the chunk),
// 4 W (anti-causal value just after the chunk); then K_c of column 0 [chunk]
// and (mu, mean w) of column 0.
// ---------------------------------------------------------------------------
constexpr int kChunkWarps = 8;    // warps (chunks) per CTA of the sum and apply kernels
constexpr int kScanWarps = 24;    // warps (chunk ranges) per CTA of the scan kernel

struct ChunkBufs {
    float *h, *a, *g, *cin, *win, *k0, *par;
};
__host__ __device__ __forceinline__ ChunkBufs chunk_bufs(float* base, int nch, int cols) {
    const size_t pl = (size_t)nch * cols;
    return ChunkBufs{base, base + pl, base + 2 * pl, base + 3 * pl, base + 4 * pl, base + 5 * pl,
                     base + 5 * pl + nch};
}

__device__ __forceinline__ float rstep1(float s, float x, float nq) { return fmaf(nq, s, s + x); }

// h, a, g (and K for column 0) of chunk blockIdx.y * kChunkWarps + warp, columns 32 blockIdx.x + lane
__global__ void __launch_bounds__(32 * kChunkWarps)
tri_chunk_sum_kernel(const float* __restrict__ S, int rows, int cols, int pitch, const float4* __restrict__ tab,
                     float* __restrict__ base, int nch) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * 32 + (threadIdx.x & 31);
    const int c = blockIdx.y * kChunkWarps + (threadIdx.x >> 5);
    if (k >= cols || c >= nch) return;
    const ChunkBufs cb = chunk_bufs(base, nch, cols);
    const float nq = -__ldg(&tab[2 * k]).x;
    const int i0 = c * kTriChunk;
    const int n = min(kTriChunk, rows - i0);
    const float* src = S + (size_t)i0 * pitch + k;
    float v[kTriChunk];
    float h = 0.f, an = 0.f, g = 0.f, kk = 0.f;   // an: the causal value at the chunk's last row n - 1
    const bool k0 = k == 0;                        // the k_x = 0 column also needs K
    if (n == kTriChunk) {
        // full chunk: no row predicates
#pragma unroll
        for (int i = 0; i < kTriChunk; ++i) v[i] = __ldg(src + (size_t)i * pitch);
#pragma unroll
        for (int i = kTriChunk - 1; i >= 0; --i) h = rstep1(h, v[i], nq);
        float p = 0.f;
#pragma unroll
        for (int i = 0; i < kTriChunk; ++i) {
            p = rstep1(p, v[i], nq);
            v[i] = p;
        }
        an = p;
#pragma unroll
        for (int i = kTriChunk - 1; i >= 0; --i) g = rstep1(g, v[i], nq);
        if (k0) {
#pragma unroll
            for (int i = 0; i < kTriChunk; ++i) kk = fmaf((float)(i + 1), v[i], kk);
        }
    } else {
#pragma unroll
        for (int i = 0; i < kTriChunk; ++i) v[i] = i < n ? __ldg(src + (size_t)i * pitch) : 0.f;
#pragma unroll
        for (int i = kTriChunk - 1; i >= 0; --i)
            if (i < n) h = rstep1(h, v[i], nq);
        float p = 0.f;
#pragma unroll
        for (int i = 0; i < kTriChunk; ++i) {
            p = rstep1(p, v[i], nq);
            v[i] = p;
            if (i == n - 1) an = p;
        }
#pragma unroll
        for (int i = kTriChunk - 1; i >= 0; --i)
            if (i < n) {
                g = rstep1(g, v[i], nq);
                kk = fmaf((float)(i + 1), v[i], kk);
            }
    }
    const size_t o = (size_t)c * cols + k;
    cb.h[o] = h;
    cb.a[o] = an;
    cb.g[o] = g;
    if (k == 0) cb.k0[c] = kk;
}

// Per column: start values and the carries of every chunk.  lane = column,
// warp w = chunks [w cpw, (w + 1) cpw); kScanWarps warps, so that each
// thread walks only a few chunks (the walks are sequential per column).
__global__ void __launch_bounds__(32 * kScanWarps)
tri_chunk_scan_kernel(int rows, int cols, const float4* __restrict__ tab, float* __restrict__ base, int nch) {
    __shared__ float sh_s1[kScanWarps][32], sh_r2[kScanWarps][32], sh_f[kScanWarps][32], sh_m[kScanWarps][32];
    __shared__ float sh_b[kScanWarps][32], sh_k[kScanWarps];
    pdl_wait();
    pdl_trigger();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = blockIdx.x * 32 + lane;
    const bool live = k < cols;
    const ChunkBufs cb = chunk_bufs(base, nch, cols);
    const int L = rows;
    const int cpw = (nch + kScanWarps - 1) / kScanWarps;
    const int c0 = min(nch, w * cpw), c1 = min(nch, c0 + cpw);
    const float4 ta = live ? __ldg(&tab[2 * k]) : make_float4(0.f, 0.f, 1.f, 1.f);
    const float4 tb = live ? __ldg(&tab[2 * k + 1]) : make_float4(1.f, 0.f, 0.f, 0.f);
    const float q = ta.x, nq = -ta.x, l2 = ta.y;
    const float rL = tb.x, dnm = tb.y, iq = tb.z;
    const bool zero_mode = k == 0;
    // r^n and sum_{m<n} r^(2m+1) for a full chunk and for the last one
    const int nlast = L - (nch - 1) * kTriChunk;
    float rfull = 1.f, rlast = 1.f, kfull = 0.f, klast = 0.f;
    {
        float pw = 1.f;
        for (int m = 0; m < kTriChunk; ++m) {
            const float r = 1.f - q;
            if (m == nlast) {
                rlast = pw;
                klast = kfull;
            }
            kfull = fmaf(pw * pw, r, kfull);   // + r^(2m+1)
            pw = fmaf(nq, pw, pw);             // * r
        }
        rfull = pw;
        if (nlast == kTriChunk) {
            rlast = rfull;
            klast = kfull;
        }
    }
    // phase 1: S1 = sum r^(i0) h, R2 = sum r^(L-1-e) a, and the range's forward composite
    float s1 = 0.f, r2 = 0.f, f = 0.f, mw = 1.f;
    if (live) {
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            const size_t o = (size_t)c * cols + k;
            const int i0 = c * kTriChunk;
            const int n = c == nch - 1 ? nlast : kTriChunk;
            const float rn = c == nch - 1 ? rlast : rfull;
            const float a = cb.a[o];
            s1 = fmaf(exp2f((float)i0 * l2), cb.h[o], s1);
            r2 = fmaf(exp2f((float)(L - i0 - n) * l2), a, r2);
            f = fmaf(rn, f, a);
            mw *= rn;
        }
    }
    sh_s1[w][lane] = s1;
    sh_r2[w][lane] = r2;
    sh_f[w][lane] = f;
    sh_m[w][lane] = mw;
    __syncthreads();
    float S1 = 0.f, R2 = 0.f;
    for (int x = 0; x < kScanWarps; ++x) {
        S1 += sh_s1[x][lane];
        R2 += sh_r2[x][lane];
    }
    const float mu = zero_mode ? S1 / (float)L : 0.f;   // k_x = 0: the input loses its mean
    // composite of range x with the mean removed (r = 1 there, so it is a plain sum)
    auto fx = [&](int x) {
        if (!zero_mode) return sh_f[x][lane];
        // rows of range x: full chunks, the last chunk of the column holding nlast
        const int xc0 = min(nch, x * cpw), xc1 = min(nch, xc0 + cpw);
        const int nr = (xc1 - xc0) * kTriChunk - ((xc1 == nch && xc1 > xc0) ? kTriChunk - nlast : 0);
        return sh_f[x][lane] - mu * (float)nr;
    };
    const float u0 = (S1 + rL * R2) * dnm;                 // c_{-1} (0 for k_x = 0)
    float carry = u0;
    for (int x = 0; x < w; ++x) carry = fmaf(sh_m[x][lane], carry, fx(x));
    float call = u0;
    for (int x = 0; x < kScanWarps; ++x) call = fmaf(sh_m[x][lane], call, fx(x));
    const float wL = call * iq;                            // w_L (0 for k_x = 0)

    // phase 2: causal carries into each chunk of the range
    if (live) {
#pragma unroll 4
        for (int c = c0; c < c1; ++c) {
            const size_t o = (size_t)c * cols + k;
            const int n = c == nch - 1 ? nlast : kTriChunk;
            const float rn = c == nch - 1 ? rlast : rfull;
            cb.cin[o] = carry;
            const float a = zero_mode ? cb.a[o] - mu * (float)n : cb.a[o];
            carry = fmaf(rn, carry, a);
        }
    }
    // phase 3: the range's anti-causal composite from zero after its last chunk
    float bsum = 0.f;
    if (live) {
#pragma unroll 4
        for (int c = c1 - 1; c >= c0; --c) {
            const size_t o = (size_t)c * cols + k;
            const int n = c == nch - 1 ? nlast : kTriChunk;
            const float rn = c == nch - 1 ? rlast : rfull;
            const float kn = c == nch - 1 ? klast : kfull;
            const float g = zero_mode ? cb.g[o] - mu * 0.5f * (float)n * (float)(n + 1) : cb.g[o];
            bsum = fmaf(rn, bsum, fmaf(cb.cin[o], kn, g));
        }
    }
    __syncthreads();
    sh_b[w][lane] = bsum;
    __syncthreads();
    float wa = wL;                                         // w just after the range
    for (int x = kScanWarps - 1; x > w; --x) wa = fmaf(sh_m[x][lane], wa, sh_b[x][lane]);
    float ksum = 0.f;
    if (live) {
#pragma unroll 4
        for (int c = c1 - 1; c >= c0; --c) {
            const size_t o = (size_t)c * cols + k;
            const int n = c == nch - 1 ? nlast : kTriChunk;
            const float rn = c == nch - 1 ? rlast : rfull;
            const float kn = c == nch - 1 ? klast : kfull;
            cb.win[o] = wa;
            const float cin = cb.cin[o];
            const float g = zero_mode ? cb.g[o] - mu * 0.5f * (float)n * (float)(n + 1) : cb.g[o];
            if (zero_mode) {
                const float nf = (float)n;
                const float kc = cb.k0[c] - mu * nf * (nf + 1.f) * (2.f * nf + 1.f) / 6.f;
                ksum += kc + cin * 0.5f * nf * (nf + 1.f) + nf * wa;
            }
            wa = fmaf(rn, wa, fmaf(cin, kn, g));
        }
    }
    if (blockIdx.x == 0 && lane == 0) sh_k[w] = ksum;   // lane 0 of block 0 is column 0 in every warp
    __syncthreads();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        float tot = 0.f;
        for (int x = 0; x < kScanWarps; ++x) tot += sh_k[x];
        cb.par[0] = mu;
        cb.par[1] = tot / (float)L;
    }
}

// Both recursions of one chunk from its carries; y = -r w (k_x = 0: the
// output mean is removed).
__global__ void __launch_bounds__(32 * kChunkWarps)
tri_chunk_apply_kernel(float* __restrict__ S, int rows, int cols, int pitch, const float4* __restrict__ tab,
                       const float* __restrict__ base, int nch) {
    pdl_wait();
    pdl_trigger();
    const int k = blockIdx.x * 32 + (threadIdx.x & 31);
    const int c = blockIdx.y * kChunkWarps + (threadIdx.x >> 5);
    if (k >= cols || c >= nch) return;
    const ChunkBufs cb = chunk_bufs(const_cast<float*>(base), nch, cols);
    const float q = __ldg(&tab[2 * k]).x, nq = -q;
    const int i0 = c * kTriChunk;
    const int n = min(kTriChunk, rows - i0);
    const size_t o = (size_t)c * cols + k;
    float mu = 0.f, shift = 0.f;
    if (k == 0) {
        mu = __ldg(&cb.par[0]);
        shift = __ldg(&cb.par[1]);
    }
    float* row = S + (size_t)i0 * pitch + k;
    float v[kTriChunk];
#pragma unroll
    for (int i = 0; i < kTriChunk; ++i) v[i] = i < n ? row[(size_t)i * pitch] - mu : 0.f;
    float p = __ldg(&cb.cin[o]);
#pragma unroll
    for (int i = 0; i < kTriChunk; ++i) {
        p = rstep1(p, v[i], nq);
        v[i] = p;
    }
    float wv = __ldg(&cb.win[o]);
#pragma unroll
    for (int i = kTriChunk - 1; i >= 0; --i)
        if (i < n) {
            wv = rstep1(wv, v[i], nq);
            row[(size_t)i * pitch] = fmaf(q, wv, -wv) + shift;
        }
}

}  // namespace

cudaError_t launch_tri_cols_chunked(float* S, int rows, int cols, int pitch, const PoissonPlans& pp,
                                    cudaStream_t s) {
    if (!pp.tsum || pp.tnch != tri_chunks(rows) || cols < 1) return cudaErrorInvalidValue;
    const int nch = pp.tnch;
    const dim3 blk(32 * kChunkWarps);
    const dim3 grd((cols + 31) / 32, (nch + kChunkWarps - 1) / kChunkWarps);
    cudaError_t e = launch_pdl(tri_chunk_sum_kernel, grd, blk, 0, s, (const float*)S, rows, cols, pitch,
                               (const float4*)pp.tri, pp.tsum, nch);
    if (e != cudaSuccess) return e;
    e = launch_pdl(tri_chunk_scan_kernel, dim3((cols + 31) / 32), dim3(32 * kScanWarps), 0, s, rows, cols,
                   (const float4*)pp.tri, pp.tsum, nch);
    if (e != cudaSuccess) return e;
    return launch_pdl(tri_chunk_apply_kernel, grd, blk, 0, s, S, rows, cols, pitch, (const float4*)pp.tri,
                      (const float*)pp.tsum, nch);
}

cudaError_t build_tri_table(float4* tab, int rows, int cols, cudaStream_t s) {
    const int n = rows_per_thread(rows);
    if (n == 0 || cols < 1) return cudaErrorInvalidValue;
    tri_table_kernel<<<(cols + 127) / 128, 128, 0, s>>>(tab, rows, cols, n);
    return cudaGetLastError();
}

cudaError_t launch_tri_cols(float* S, int rows, int cols, int pitch, const float4* tab, const BatchArgs& ba,
                            int nbatch, cudaStream_t s) {
    if (cols < 1) return cudaErrorInvalidValue;
    switch (rows_per_thread(rows)) {
        case 3: return launch_n<3>(S, rows, cols, pitch, tab, ba, nbatch, s);
        case 5: return launch_n<5>(S, rows, cols, pitch, tab, ba, nbatch, s);
        case 9: return launch_n<9>(S, rows, cols, pitch, tab, ba, nbatch, s);
        case 17: return launch_n<17>(S, rows, cols, pitch, tab, ba, nbatch, s);
        case 33: return launch_n<33>(S, rows, cols, pitch, tab, ba, nbatch, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvs
