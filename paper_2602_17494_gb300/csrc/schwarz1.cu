// Overlapping Schwarz decomposition of the TFS dual (Section 6): Algorithm 2
// with the fully localized inner loop of Algorithm 5.
//
// Per outer iteration n:
//   Q      = P_K vecdiv p^n                                  (global transform)
//   omega_m = R_{m,+}(f1 - Q) + R_{m,+} P_K E_{m,+} vecdiv(theta_m p^n)
//           (equal to R_{m,+}(f1 - P_K vecdiv sum_{l != m} theta_l p^n) by
//            linearity, since the theta_l sum to one)
//   k times: u   = vecdiv_{m,+} E_m v                      on tilde Omega_{m,+}
//            P   = R_{m,+} P_K E_{m,+} u = u - grad_B phi,  phi = R_B Delta^dagger E_A div_A u
//            psi = R_m vecgrad_{m,+} (P - omega_m);   v <- (theta v + t theta psi)/(theta + t|psi|)
//   p^{n+1} = (1 - alpha_hat) p^n + alpha_hat sum_m E_m v_m
// with A = B = (tilde Omega_{m,+})_+ (eqs. locglobprojpart1, locglobprojpart3).
//
// The localized inverse Laplacian R_B Delta^dagger E_A (eq. invLaplLowCapLong)
// is the sum over all frequency blocks of products of DCT matrix blocks; it is
// evaluated here with the fast transforms of dct.cu restricted to the rows of
// A: forward x-transforms of A's rows only, full-length y-transforms that read
// and write only A's rows, inverse x-transforms of A's rows only.  Memory per
// subdomain is (rows of A) x (grid width), never the whole grid; all
// subdomains run as one batch.
#include "decomp.cuh"
#include "launchers.h"
#include "prof.h"

#include <vector>

namespace tvs {

struct S1Geom {
    Axis ay, ax;   // extended-grid axes (N image pixels, L = N + 1 points)
    int R, C;      // extended grid
    int hbox, wpad;
    int pitch;     // row pitch of the global arrays and of the packed Poisson rows
    long plane;    // global plane stride
};

struct Box {
    int y0, y1, x0, x1;   // tilde Omega_m
    int yp, xp;           // ends of tilde Omega_{m,+}
    int ya, xa;           // ends of A = B = (tilde Omega_{m,+})_+
};

__host__ __device__ __forceinline__ Box tile_box(const S1Geom& g, int tile) {
    const int my = tile / g.ax.M, mx = tile - my * g.ax.M;
    Box b;
    b.y0 = g.ay.start(my);
    b.y1 = g.ay.end(my);
    b.x0 = g.ax.start(mx);
    b.x1 = g.ax.end(mx);
    b.yp = b.y1 + 1 < g.R ? b.y1 + 1 : g.R;
    b.xp = b.x1 + 1 < g.C ? b.x1 + 1 : g.C;
    b.ya = b.y1 + 2 < g.R ? b.y1 + 2 : g.R;
    b.xa = b.x1 + 2 < g.C ? b.x1 + 2 : g.C;
    return b;
}

// per-tile plane q of a tile array with `np` planes
__device__ __forceinline__ float* tplane(float* base, const S1Geom& g, int tile, int np, int q) {
    return base + ((size_t)tile * np + q) * g.hbox * g.wpad;
}

// ---------------------------------------------------------------------------
// u = vecdiv(E_m v) on tilde Omega_{m,+}; v is the tile's inner variable
// (FROM_P = false) or theta_m p^n (FROM_P = true).
// ---------------------------------------------------------------------------
template <bool FROM_P>
__global__ void s1_u_kernel(S1Geom g, float* V, const float* __restrict__ p, float* U) {
    const int tile = blockIdx.z;
    const Box b = tile_box(g, tile);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = b.y0 + r, j = b.x0 + c;
    if (i >= b.yp || j >= b.xp) return;
    const int my = tile / g.ax.M, mx = tile - my * g.ax.M;
    auto val = [&](int q, int ii, int jj) -> float {   // component q of v at (ii, jj), zero outside tilde Omega_m
        if (ii < b.y0 || ii >= b.y1 || jj < b.x0 || jj >= b.x1) return 0.0f;
        if (FROM_P) {
            const float th = g.ay.theta(my, ii) * g.ax.theta(mx, jj);
            return th * __ldg(&p[(size_t)q * g.plane + (size_t)ii * g.pitch + jj]);
        }
        return tplane(V, g, tile, 4, q)[(size_t)(ii - b.y0) * g.wpad + (jj - b.x0)];
    };
    for (int k = 0; k < 2; ++k) {
        auto vx = [&](int ii, int jj) { return (jj >= 0 && jj <= g.C - 2) ? val(2 * k, ii, jj) : 0.0f; };
        auto vy = [&](int ii, int jj) { return (ii >= 0 && ii <= g.R - 2) ? val(2 * k + 1, ii, jj) : 0.0f; };
        const float u = (vx(i, j) - vx(i, j - 1)) + (vy(i, j) - vy(i - 1, j));
        tplane(U, g, tile, 2, k)[(size_t)r * g.wpad + c] = u;
    }
}

// ---------------------------------------------------------------------------
// Poisson source on the rows of A, full grid width: s = div_A(E_{m,+} u) on A,
// zero elsewhere in those rows.
// ---------------------------------------------------------------------------
__global__ void s1_s_kernel(S1Geom g, const float* __restrict__ U, float* S) {
    const int tile = blockIdx.z;
    const Box b = tile_box(g, tile);
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = b.y0 + r;
    if (i >= b.ya || j >= g.C) return;
    float s = 0.0f;
    if (j >= b.x0 && j < b.xa) {
        const float* ux = U + ((size_t)tile * 2 + 0) * g.hbox * g.wpad;
        const float* uy = U + ((size_t)tile * 2 + 1) * g.hbox * g.wpad;
        auto in_plus = [&](int ii, int jj) { return ii >= b.y0 && ii < b.yp && jj >= b.x0 && jj < b.xp; };
        auto fx = [&](int ii, int jj) {
            return (in_plus(ii, jj) && jj <= g.C - 2) ? ux[(size_t)(ii - b.y0) * g.wpad + (jj - b.x0)] : 0.0f;
        };
        auto fy = [&](int ii, int jj) {
            return (in_plus(ii, jj) && ii <= g.R - 2) ? uy[(size_t)(ii - b.y0) * g.wpad + (jj - b.x0)] : 0.0f;
        };
        s = (fx(i, j) - fx(i, j - 1)) + (fy(i, j) - fy(i - 1, j));
    }
    S[(size_t)tile * g.hbox * g.pitch + (size_t)r * g.pitch + j] = s;
}

// P_k(i, j) = u_k - (grad_B phi)_k on tilde Omega_{m,+} (local gradient on B)
__device__ __forceinline__ float proj_at(const S1Geom& g, const Box& b, const float* ux, const float* uy,
                                         const float* phi, int k, int i, int j) {
    const float* u = k == 0 ? ux : uy;
    const size_t lo = (size_t)(i - b.y0) * g.wpad + (j - b.x0);
    const float pc = phi[(size_t)(i - b.y0) * g.pitch + j];
    float gphi;
    if (k == 0) gphi = (j + 1 < b.xa) ? phi[(size_t)(i - b.y0) * g.pitch + j + 1] - pc : 0.0f;
    else gphi = (i + 1 < b.ya) ? phi[(size_t)(i + 1 - b.y0) * g.pitch + j] - pc : 0.0f;
    return u[lo] - gphi;
}

// omega_m = R_{m,+}(f1 - Q) + P on tilde Omega_{m,+}
__global__ void s1_omega_kernel(S1Geom g, const float* __restrict__ U, const float* __restrict__ S,
                                const float* __restrict__ f1, const float* __restrict__ Q, float* W) {
    const int tile = blockIdx.z;
    const Box b = tile_box(g, tile);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = b.y0 + r, j = b.x0 + c;
    if (i >= b.yp || j >= b.xp) return;
    const float* ux = U + ((size_t)tile * 2 + 0) * g.hbox * g.wpad;
    const float* uy = U + ((size_t)tile * 2 + 1) * g.hbox * g.wpad;
    const float* phi = S + (size_t)tile * g.hbox * g.pitch;
    const size_t go = (size_t)i * g.pitch + j;
    for (int k = 0; k < 2; ++k) {
        const float pk = proj_at(g, b, ux, uy, phi, k, i, j);
        W[((size_t)tile * 2 + k) * g.hbox * g.wpad + (size_t)r * g.wpad + c] =
            (__ldg(&f1[(size_t)k * g.plane + go]) - __ldg(&Q[(size_t)k * g.plane + go])) + pk;
    }
}

// One inner update of Algorithm 5 on tilde Omega_m.
__global__ void s1_update_kernel(S1Geom g, const float* __restrict__ U, const float* __restrict__ S,
                                 const float* __restrict__ W, float* V, float t) {
    const int tile = blockIdx.z;
    const Box b = tile_box(g, tile);
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r = blockIdx.y * blockDim.y + threadIdx.y;
    const int i = b.y0 + r, j = b.x0 + c;
    if (i >= b.y1 || j >= b.x1) return;
    const int my = tile / g.ax.M, mx = tile - my * g.ax.M;
    const float* ux = U + ((size_t)tile * 2 + 0) * g.hbox * g.wpad;
    const float* uy = U + ((size_t)tile * 2 + 1) * g.hbox * g.wpad;
    const float* phi = S + (size_t)tile * g.hbox * g.pitch;
    const float th = g.ay.theta(my, i) * g.ax.theta(mx, j);
    const size_t lo = (size_t)r * g.wpad + c;
    for (int k = 0; k < 2; ++k) {
        const float* w = W + ((size_t)tile * 2 + k) * g.hbox * g.wpad;
        auto zk = [&](int ii, int jj) {
            return proj_at(g, b, ux, uy, phi, k, ii, jj) - w[(size_t)(ii - b.y0) * g.wpad + (jj - b.x0)];
        };
        const float zc = zk(i, j);
        const float gx = (j + 1 < b.xp) ? zk(i, j + 1) - zc : 0.0f;
        const float gy = (i + 1 < b.yp) ? zk(i + 1, j) - zc : 0.0f;
        float* vx = tplane(V, g, tile, 4, 2 * k);
        float* vy = tplane(V, g, tile, 4, 2 * k + 1);
        const float den = th + t * sqrtf(gx * gx + gy * gy);
        if (den > 0.0f) {
            const float sc = th / den;
            vx[lo] = (vx[lo] + t * gx) * sc;
            vy[lo] = (vy[lo] + t * gy) * sc;
        } else {
            vx[lo] = 0.0f;
            vy[lo] = 0.0f;
        }
    }
}

// Q = P_K vecdiv p = vecdiv p - grad phi (global rules), phi = Delta^dagger div vecdiv p
__global__ void s1_q_kernel(S1Geom g, const float* __restrict__ p, const float* __restrict__ phi, float* Q) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.R || j >= g.C) return;
    auto ld = [&](int q, int ii, int jj) { return __ldg(&p[(size_t)q * g.plane + (size_t)ii * g.pitch + jj]); };
    const float pc = __ldg(&phi[(size_t)i * g.pitch + j]);
    for (int k = 0; k < 2; ++k) {
        const float xc = (j <= g.C - 2) ? ld(2 * k, i, j) : 0.0f;
        const float xl = (j >= 1) ? ld(2 * k, i, j - 1) : 0.0f;
        const float yc = (i <= g.R - 2) ? ld(2 * k + 1, i, j) : 0.0f;
        const float yu = (i >= 1) ? ld(2 * k + 1, i - 1, j) : 0.0f;
        const float w = (xc - xl) + (yc - yu);
        float gphi;
        if (k == 0) gphi = (j < g.C - 1) ? __ldg(&phi[(size_t)i * g.pitch + j + 1]) - pc : 0.0f;
        else gphi = (i < g.R - 1) ? __ldg(&phi[(size_t)(i + 1) * g.pitch + j]) - pc : 0.0f;
        Q[(size_t)k * g.plane + (size_t)i * g.pitch + j] = w - gphi;
    }
}

// p^{n+1} = (1 - alpha_hat) p^n + alpha_hat sum over tiles containing x of v_m(x), 4 planes
__global__ void s1_combine_kernel(S1Geom g, const float* __restrict__ pin, float* pout,
                                  const float* __restrict__ V, float ah) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= g.R || j >= g.C) return;
    const int ky = g.ay.core_of(i < g.ay.N ? i : g.ay.N - 1), kx = g.ax.core_of(j < g.ax.N ? j : g.ax.N - 1);
    float acc[4] = {0.f, 0.f, 0.f, 0.f};
    for (int a = ky - 1; a <= ky + 1; ++a) {
        if (a < 0 || a >= g.ay.M || i < g.ay.start(a) || i >= g.ay.end(a)) continue;
        for (int bb = kx - 1; bb <= kx + 1; ++bb) {
            if (bb < 0 || bb >= g.ax.M || j < g.ax.start(bb) || j >= g.ax.end(bb)) continue;
            const int tile = a * g.ax.M + bb;
            const size_t lo = (size_t)(i - g.ay.start(a)) * g.wpad + (j - g.ax.start(bb));
            for (int q = 0; q < 4; ++q) acc[q] += V[((size_t)tile * 4 + q) * g.hbox * g.wpad + lo];
        }
    }
    const size_t o = (size_t)i * g.pitch + j;
    for (int q = 0; q < 4; ++q) pout[(size_t)q * g.plane + o] = (1.0f - ah) * pin[(size_t)q * g.plane + o] + ah * acc[q];
}

// ---------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------
static S1Geom make_geom(int n2, int n1, const Schwarz1State& st, int pitch) {
    S1Geom g;
    g.ay = Axis{n2, st.m2, st.s, n2 + 1};
    g.ax = Axis{n1, st.m1, st.s, n1 + 1};
    g.R = n2 + 1;
    g.C = n1 + 1;
    g.hbox = st.hbox;
    g.wpad = st.wpad;
    g.pitch = pitch;
    g.plane = (long)g.R * pitch;
    return g;
}

static double colouring1(int m2, int m1) {
    if (m2 == 1 && m1 == 1) return 1.0;
    if (m2 == 1 || m1 == 1) return 0.5;
    return 0.25;
}

constexpr double kSchwarz1MaxBytes = 16.0e9;   // per-subdomain scratch (rows of A x grid width)

void schwarz1_carve(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch, Schwarz1State& st) {
    st.m2 = dd.m2;
    st.m1 = dd.m1;
    st.s = dd.overlap;
    st.k = dd.k_inner;
    st.alpha_hat = dd.alpha_hat > 0.0 ? dd.alpha_hat : colouring1(dd.m2, dd.m1);
    st.ntiles = dd.m2 * dd.m1;
    Axis ay{n2, dd.m2, dd.overlap, n2 + 1}, ax{n1, dd.m1, dd.overlap, n1 + 1};
    int hb = 0, wb = 0;
    for (int k = 0; k < dd.m2; ++k) hb = std::max(hb, std::min(ay.end(k) + 2, n2 + 1) - ay.start(k));
    for (int k = 0; k < dd.m1; ++k) wb = std::max(wb, std::min(ax.end(k) + 2, n1 + 1) - ax.start(k));
    st.hbox = hb;
    st.wpad = round_up(wb, 4);
    st.pitch = pitch;
    const size_t tile_floats = (size_t)st.hbox * st.wpad;
    st.V = cv.take<float>((size_t)st.ntiles * 4 * tile_floats);
    st.U = cv.take<float>((size_t)st.ntiles * 2 * tile_floats);
    st.W = cv.take<float>((size_t)st.ntiles * 2 * tile_floats);
    st.S = cv.take<float>((size_t)st.ntiles * st.hbox * pitch);
    st.Q = cv.take<float>((size_t)2 * (n2 + 1) * pitch);
    st.ranges = cv.take<int2>((size_t)st.ntiles);
}

size_t schwarz1_extend(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch) {
    Schwarz1State st;
    schwarz1_carve(cv, n2, n1, dd, pitch, st);
    return cv.used();
}

tvs_status schwarz1_check(int n2, int n1, const tvs_decomp& dd) {
    if (dd.m2 < 1 || dd.m1 < 1 || dd.overlap < 0 || dd.k_inner < 1 || dd.alpha_hat > 1.0) return TVS_ERR_ARG;
    if (dd.m2 > n2 || dd.m1 > n1) return TVS_ERR_ARG;
    const int s = dd.overlap;
    Axis ay{n2, dd.m2, s, n2 + 1}, ax{n1, dd.m1, s, n1 + 1};
    for (int k = 0; k < dd.m2; ++k)
        if (ay.core(k + 1) - ay.core(k) < (s > 1 ? s : 1)) return TVS_ERR_ARG;
    for (int k = 0; k < dd.m1; ++k)
        if (ax.core(k + 1) - ax.core(k) < (s > 1 ? s : 1)) return TVS_ERR_ARG;
    Schwarz1State st;
    Carver cv(nullptr);
    schwarz1_carve(cv, n2, n1, dd, round_up(n1 + 1, kPitchAlign), st);
    if ((double)cv.used() > kSchwarz1MaxBytes) return TVS_ERR_UNSUPPORTED;
    return TVS_OK;
}

cudaError_t schwarz1_reset(const Schwarz1State& st, int n2, int n1, cudaStream_t s) {
    S1Geom g = make_geom(n2, n1, st, st.pitch);
    std::vector<int2> h(st.ntiles);
    for (int t = 0; t < st.ntiles; ++t) {
        const Box b = tile_box(g, t);
        h[t] = make_int2(b.y0, b.ya);
    }
    cudaError_t e = cudaMemcpyAsync(st.ranges, h.data(), h.size() * sizeof(int2), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    // the copy above reads pageable memory: make sure it is done before h goes away
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(st.V, 0, (size_t)st.ntiles * 4 * st.hbox * st.wpad * sizeof(float), s);
}

// Localized projection of the tiles' u: S <- phi on the rows of A (batched).
static cudaError_t local_projection(const S1Geom& g, const Schwarz1State& st, const PoissonPlans& pp,
                                    cudaStream_t s) {
    dim3 blk(32, 8);
    dim3 grd((g.C + 31) / 32, (g.hbox + 7) / 8, st.ntiles);
    s1_s_kernel<<<grd, blk, 0, s>>>(g, st.U, st.S);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return poisson_solve_batched(st.S, st.ntiles, (long)st.hbox * g.pitch, st.ranges, st.hbox, g.R, g.C, g.pitch,
                                 pp, s);
}

cudaError_t schwarz1_iterate(float** cur, float** nxt, const float* f1, float* S_glob, int pitch, int n2, int n1,
                             const PoissonPlans& pp, const Schwarz1State& st, float t, int n_outer, unsigned* err,
                             cudaStream_t s) {
    const S1Geom g = make_geom(n2, n1, st, pitch);
    const dim3 blk(32, 8);
    const dim3 gtile((st.wpad + 31) / 32, (st.hbox + 7) / 8, st.ntiles);
    const dim3 gglob((g.C + 31) / 32, (g.R + 7) / 8);
    cudaError_t e;
    for (int n = 0; n < n_outer; ++n) {
        // Q = P_K vecdiv p^n
        if ((e = tfs_phi(*cur, S_glob, g.R, g.C, pitch, g.plane, pp, err, s)) != cudaSuccess) return e;
        s1_q_kernel<<<gglob, blk, 0, s>>>(g, *cur, S_glob, st.Q);
        // omega_m
        s1_u_kernel<true><<<gtile, blk, 0, s>>>(g, st.V, *cur, st.U);
        if ((e = local_projection(g, st, pp, s)) != cudaSuccess) return e;
        s1_omega_kernel<<<gtile, blk, 0, s>>>(g, st.U, st.S, f1, st.Q, st.W);
        // k inner updates (Algorithm 5)
        for (int it = 0; it < st.k; ++it) {
            s1_u_kernel<false><<<gtile, blk, 0, s>>>(g, st.V, *cur, st.U);
            if ((e = local_projection(g, st, pp, s)) != cudaSuccess) return e;
            ProfScope ps(kProfSchwarzTile, s);
            s1_update_kernel<<<gtile, blk, 0, s>>>(g, st.U, st.S, st.W, st.V, t);
        }
        {
            ProfScope ps(kProfSchwarzCombine, s);
            s1_combine_kernel<<<gglob, blk, 0, s>>>(g, *cur, *nxt, st.V, (float)st.alpha_hat);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        float* tmp = *cur;
        *cur = *nxt;
        *nxt = tmp;
    }
    return cudaSuccess;
}

}  // namespace tvs
