// Overlapping Schwarz decomposition of the IRV1 dual (Section 6.1):
// Algorithm 2 (outer, additive with damping alpha_hat) with Algorithm 3
// (inner Chambolle iteration on one subdomain), Lambda = div, f = f2.
//
// GB300 mapping: one subdomain is one thread-block cluster; each CTA of the
// cluster keeps a horizontal band of the subdomain's inner dual v, the frozen
// data g_m = f2 - div((1 - theta_m) p^n) and the residual z in shared memory
// and runs all k inner updates on chip.  Rows next to a band boundary are read
// from the neighbouring CTA through distributed shared memory.  The outer
// combine p^{n+1} = (1 - alpha_hat) p^n + alpha_hat sum_l q_l goes through HBM
// between launches -- that is the grid-wide halo exchange.
//
// Decomposition (same reading as the oracle): cores split each axis as
// evenly as integers allow, core k = [floor(kN/M), floor((k+1)N/M)); two
// neighbours share a strip of s pixels [b - ceil(s/2), b + floor(s/2)) around
// their core boundary b with linear weights theta (pixel-centre values); the
// 2-D weight is the product of the 1-D weights.
#include "decomp.cuh"
#include "launchers.h"
#include "prof.h"

#include <cooperative_groups.h>

#include <algorithm>
#include <mutex>

namespace cg = cooperative_groups;

namespace tvs {

constexpr int kSchwarzThreads = 512;
constexpr size_t kSchwarzSmemMax = 200 * 1024;

struct TileArgs {
    const float* p;   // p^n, 2 planes
    const float* f2;
    int pitch;
    long plane;
    float* q;         // [sub][2][hmax][wpad]
    int hmax, wpad;
    Axis ay, ax;
    int band, k;
    float t;
};

// Shared memory of one CTA (floats):
//   v_x, v_y : (band + 2) x wpad each -- row 0 is the halo row above, rows
//              1..nown the CTA's own rows, row nown+1 the halo row below
//   g, z     : (band + 1) x wpad each
//   theta_x  : wpad;  theta_y : band + 1
//   outbox   : 2 parities x 3 rows x wpad -- the first row of v_x and v_y and
//              the last row of v_y, published for the neighbouring CTAs
__host__ __device__ __forceinline__ size_t tile_smem_floats(int band, int wpad) {
    return (size_t)2 * (band + 2) * wpad + (size_t)2 * (band + 1) * wpad + wpad + band + 1 + (size_t)6 * wpad;
}

__global__ void __launch_bounds__(kSchwarzThreads)
schwarz2_tile_kernel(TileArgs a) {
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float sm[];
    const int WP = a.wpad, B = a.band;
    float* vx = sm;                              // row r of the band at vx + (r + 1) * WP
    float* vy = vx + (size_t)(B + 2) * WP;
    float* g = vy + (size_t)(B + 2) * WP;
    float* z = g + (size_t)(B + 1) * WP;
    float* thx = z + (size_t)(B + 1) * WP;
    float* thy = thx + WP;
    float* outbox = thy + (B + 1);               // [parity][3][WP]

    const int N2 = a.ay.N, N1 = a.ax.N;
    const int sub = blockIdx.y;
    const int my = sub / a.ax.M, mx = sub - my * a.ax.M;
    const int y0 = a.ay.start(my), y1 = a.ay.end(my);
    const int x0 = a.ax.start(mx), x1 = a.ax.end(mx);
    const int w = x1 - x0;
    const int rank = (int)cl.block_rank();
    const int ncl = (int)cl.num_blocks();
    const int r_lo = y0 + rank * B;
    const int r_hi = min(y1, r_lo + B);
    const int nown = max(0, r_hi - r_lo);
    const bool has_above = rank > 0 && nown > 0;
    const bool has_below = rank + 1 < ncl && r_hi < y1;   // the next band owns row r_hi
    // z rows: own rows plus the next row when it exists in Gamma_{m,+}
    const int zrows = nown + ((nown > 0 && r_hi < N2) ? 1 : 0);
    const int zcols = w + (x1 < N1 ? 1 : 0);
    const float* __restrict__ px = a.p;
    const float* __restrict__ py = a.p + a.plane;
    float* qx = a.q + (size_t)sub * 2 * a.hmax * WP;
    float* qy = qx + (size_t)a.hmax * WP;
    const float t = a.t;
    const int nt = blockDim.x;
    const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5, nwy = blockDim.x >> 5;

    // ---- set-up: weights, warm start, frozen data g_m --------------------
    for (int c = threadIdx.x; c < WP; c += nt) thx[c] = (c < w) ? a.ax.theta(mx, x0 + c) : 0.0f;
    for (int r = threadIdx.x; r <= B; r += nt) {
        const int i = r_lo + r;
        thy[r] = (r < nown) ? a.ay.theta(my, i) : 0.0f;
    }
    for (int idx = threadIdx.x; idx < (B + 2) * WP; idx += nt) {
        const int r = idx / WP - 1, c = idx - (idx / WP) * WP;
        float ux = 0.0f, uy = 0.0f;
        if (r >= 0 && r < nown && c < w) {
            const size_t qo = (size_t)(r_lo - y0 + r) * WP + c;
            ux = qx[qo];
            uy = qy[qo];
        }
        vx[idx] = ux;
        vy[idx] = uy;
    }
    // g = f2 - div(w) with w = (1 - theta_m) p^n, D^- zero-extension rule
    for (int idx = threadIdx.x; idx < zrows * zcols; idx += nt) {
        const int r = idx / zcols, c = idx - r * zcols;
        const int i = r_lo + r, j = x0 + c;
        auto wx = [&](int ii, int jj) -> float {
            if (jj < 0 || jj > N1 - 2) return 0.0f;
            const float th = a.ay.theta_or0(my, ii) * a.ax.theta_or0(mx, jj);
            return (1.0f - th) * __ldg(&px[(size_t)ii * a.pitch + jj]);
        };
        auto wy = [&](int ii, int jj) -> float {
            if (ii < 0 || ii > N2 - 2) return 0.0f;
            const float th = a.ay.theta_or0(my, ii) * a.ax.theta_or0(mx, jj);
            return (1.0f - th) * __ldg(&py[(size_t)ii * a.pitch + jj]);
        };
        const float divw = (wx(i, j) - wx(i, j - 1)) + (wy(i, j) - wy(i - 1, j));
        g[(size_t)r * WP + c] = __ldg(&a.f2[(size_t)i * a.pitch + j]) - divw;
    }
    __syncthreads();
    // publish the boundary rows of the warm start (parity 0)
    if (nown > 0) {
        for (int c = threadIdx.x; c < WP; c += nt) {
            outbox[0 * WP + c] = vx[(size_t)1 * WP + c];
            outbox[1 * WP + c] = vy[(size_t)1 * WP + c];
            outbox[2 * WP + c] = vy[(size_t)nown * WP + c];
        }
    }

    // ---- k inner updates on chip (Algorithm 3) --------------------------
    const bool xlast = (x1 == N1);          // D^- reads v_x as zero in the grid's last column
    for (int it = 0; it < a.k; ++it) {
        const int par = it & 1;
        cl.sync();   // the neighbours' published rows of this parity are complete
        if (has_above) {
            const float* ob = cl.map_shared_rank(outbox, rank - 1) + (size_t)par * 3 * WP;
            for (int c = threadIdx.x; c < WP; c += nt) vy[c] = ob[2 * WP + c];
        }
        if (has_below) {
            const float* ob = cl.map_shared_rank(outbox, rank + 1) + (size_t)par * 3 * WP;
            for (int c = threadIdx.x; c < WP; c += nt) {
                vx[(size_t)(nown + 1) * WP + c] = ob[c];
                vy[(size_t)(nown + 1) * WP + c] = ob[WP + c];
            }
        }
        __syncthreads();
        for (int r = wy; r < zrows; r += nwy) {
            const int i = r_lo + r;
            const float* rx = vx + (size_t)(r + 1) * WP;
            const float* ry = vy + (size_t)(r + 1) * WP;
            for (int c = lane; c < zcols; c += 32) {
                const float vxc = (c < w && !(xlast && c == w - 1)) ? rx[c] : 0.0f;
                const float vxl = (c >= 1 && !(xlast && c - 1 == w - 1)) ? rx[c - 1] : 0.0f;
                const float vyc = (c < w && i <= N2 - 2) ? ry[c] : 0.0f;
                const float vyu = (c < w && i - 1 <= N2 - 2) ? ry[c - WP] : 0.0f;
                z[(size_t)r * WP + c] = (vxc - vxl) + (vyc - vyu) - g[(size_t)r * WP + c];
            }
        }
        __syncthreads();
        for (int r = wy; r < nown; r += nwy)
            for (int c = lane; c < w; c += 32) {
            const int i = r_lo + r, j = x0 + c;
            const float zc = z[(size_t)r * WP + c];
            const float gx = (j < N1 - 1) ? z[(size_t)r * WP + c + 1] - zc : 0.0f;
            const float gy = (i < N2 - 1) ? z[(size_t)(r + 1) * WP + c] - zc : 0.0f;
            const float th = thy[r] * thx[c];
            const float den = th + t * sqrtf(gx * gx + gy * gy);
            float* pvx = vx + (size_t)(r + 1) * WP + c;
            float* pvy = vy + (size_t)(r + 1) * WP + c;
            if (den > 0.0f) {
                const float sc = th / den;
                *pvx = (*pvx + t * gx) * sc;
                *pvy = (*pvy + t * gy) * sc;
            } else {
                *pvx = 0.0f;
                *pvy = 0.0f;
            }
            }
        __syncthreads();
        if (nown > 0) {
            float* ob = outbox + (size_t)(par ^ 1) * 3 * WP;
            for (int c = threadIdx.x; c < WP; c += nt) {
                ob[c] = vx[(size_t)1 * WP + c];
                ob[WP + c] = vy[(size_t)1 * WP + c];
                ob[2 * WP + c] = vy[(size_t)nown * WP + c];
            }
        }
    }
    // ---- store the new warm start q_m ------------------------------------
    for (int idx = threadIdx.x; idx < nown * w; idx += nt) {
        const int r = idx / w, c = idx - r * w;
        const size_t qo = (size_t)(r_lo - y0 + r) * WP + c;
        qx[qo] = vx[(size_t)(r + 1) * WP + c];
        qy[qo] = vy[(size_t)(r + 1) * WP + c];
    }
    cl.sync();   // no CTA leaves while a neighbour could still address its shared memory
}

// p^{n+1} = (1 - alpha_hat) p^n + alpha_hat sum over subdomains containing x of q_l(x)
__global__ void schwarz2_combine_kernel(const float* __restrict__ pin, float* __restrict__ pout,
                                        const float* __restrict__ q, int pitch, long plane, Axis ay, Axis ax,
                                        int hmax, int wpad, float ah) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= ay.L || j >= ax.L) return;
    const int ky = ay.core_of(i), kx = ax.core_of(j);
    float sx = 0.0f, sy = 0.0f;
    for (int a = ky - 1; a <= ky + 1; ++a) {
        if (a < 0 || a >= ay.M || i < ay.start(a) || i >= ay.end(a)) continue;
        for (int b = kx - 1; b <= kx + 1; ++b) {
            if (b < 0 || b >= ax.M || j < ax.start(b) || j >= ax.end(b)) continue;
            const int sub = a * ax.M + b;
            const size_t off = ((size_t)sub * 2 * hmax + (i - ay.start(a))) * wpad + (j - ax.start(b));
            sx += q[off];
            sy += q[off + (size_t)hmax * wpad];
        }
    }
    const size_t o = (size_t)i * pitch + j;
    pout[o] = (1.0f - ah) * pin[o] + ah * sx;
    pout[plane + o] = (1.0f - ah) * pin[plane + o] + ah * sy;
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static double colouring(int m2, int m1) {
    if (m2 == 1 && m1 == 1) return 1.0;
    if (m2 == 1 || m1 == 1) return 0.5;
    return 0.25;
}

tvs_status schwarz2_check(int n2, int n1, const tvs_decomp& dd) {
    if (dd.m2 < 1 || dd.m1 < 1 || dd.overlap < 0 || dd.k_inner < 1 || dd.alpha_hat > 1.0) return TVS_ERR_ARG;
    if (dd.m2 > n2 || dd.m1 > n1) return TVS_ERR_ARG;
    const int s = dd.overlap;
    Axis ay{n2, dd.m2, s, n2}, ax{n1, dd.m1, s, n1};
    for (int k = 0; k < dd.m2; ++k)
        if (ay.core(k + 1) - ay.core(k) < (s > 1 ? s : 1)) return TVS_ERR_ARG;
    for (int k = 0; k < dd.m1; ++k)
        if (ax.core(k + 1) - ax.core(k) < (s > 1 ? s : 1)) return TVS_ERR_ARG;
    Schwarz2State st;
    Carver cv(nullptr);
    schwarz2_carve(cv, n2, n1, dd, round_up(n1, kPitchAlign), st);
    if (st.ncl > 16 || st.smem > kSchwarzSmemMax) return TVS_ERR_UNSUPPORTED;
    return TVS_OK;
}

void schwarz2_carve(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch, Schwarz2State& st) {
    (void)pitch;
    st.m2 = dd.m2;
    st.m1 = dd.m1;
    st.s = dd.overlap;
    st.k = dd.k_inner;
    st.alpha_hat = dd.alpha_hat > 0.0 ? dd.alpha_hat : colouring(dd.m2, dd.m1);
    Axis ay{n2, dd.m2, dd.overlap, n2}, ax{n1, dd.m1, dd.overlap, n1};
    st.hmax = 0;
    st.wmax = 0;
    for (int k = 0; k < dd.m2; ++k) st.hmax = std::max(st.hmax, ay.end(k) - ay.start(k));
    for (int k = 0; k < dd.m1; ++k) st.wmax = std::max(st.wmax, ax.end(k) - ax.start(k));
    st.wpad = round_up(st.wmax + 1, 4);
    // fewest CTAs per subdomain whose band fits two CTAs per SM; else one CTA per SM
    st.ncl = 0;
    for (size_t budget : {size_t(110 * 1024), kSchwarzSmemMax}) {
        for (int ncl = 1; ncl <= 16 && !st.ncl; ++ncl) {
            const int band = (st.hmax + ncl - 1) / ncl;
            const size_t bytes = tile_smem_floats(band, st.wpad) * sizeof(float);
            if (bytes <= budget) {
                st.ncl = ncl;
                st.band = band;
                st.smem = bytes;
            }
        }
        if (st.ncl) break;
    }
    if (!st.ncl) {
        st.ncl = 17;
        st.band = (st.hmax + 16) / 17;
        st.smem = tile_smem_floats(st.band, st.wpad) * sizeof(float);
    }
    st.q = cv.take<float>((size_t)dd.m2 * dd.m1 * 2 * st.hmax * st.wpad);
}

size_t schwarz2_extend(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch) {
    Schwarz2State st;
    schwarz2_carve(cv, n2, n1, dd, pitch, st);
    return cv.used();
}

cudaError_t schwarz2_reset(const Schwarz2State& st, cudaStream_t s) {
    return cudaMemsetAsync(st.q, 0, (size_t)st.m2 * st.m1 * 2 * st.hmax * st.wpad * sizeof(float), s);
}

cudaError_t schwarz2_iterate(float** cur, float** nxt, const float* f2, int pitch, long plane, int n2, int n1,
                             const Schwarz2State& st, float t, int n_outer, cudaStream_t s) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(schwarz2_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kSchwarzSmemMax);
        cudaFuncSetAttribute(schwarz2_tile_kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    });
    Axis ay{n2, st.m2, st.s, n2}, ax{n1, st.m1, st.s, n1};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(st.ncl, st.m2 * st.m1, 1);
    cfg.blockDim = dim3(kSchwarzThreads, 1, 1);
    cfg.dynamicSmemBytes = st.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = st.ncl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    dim3 cblk(32, 8), cgrd((n1 + 31) / 32, (n2 + 7) / 8);
    for (int n = 0; n < n_outer; ++n) {
        TileArgs a{*cur, f2, pitch, plane, st.q, st.hmax, st.wpad, ay, ax, st.band, st.k, t};
        cudaError_t e;
        {
            ProfScope ps(kProfSchwarzTile, s);
            e = cudaLaunchKernelEx(&cfg, schwarz2_tile_kernel, a);
        }
        if (e != cudaSuccess) return e;
        {
            ProfScope ps(kProfSchwarzCombine, s);
            schwarz2_combine_kernel<<<cgrd, cblk, 0, s>>>(*cur, *nxt, st.q, pitch, plane, ay, ax, st.hmax,
                                                           st.wpad, (float)st.alpha_hat);
        }
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        float* tmp = *cur;
        *cur = *nxt;
        *nxt = tmp;
    }
    return cudaSuccess;
}

}  // namespace tvs
