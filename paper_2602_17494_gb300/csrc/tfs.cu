// Step 1, tangent field smoothing (Section 4.2, eq. tfsdualdis, Algorithm 1):
//   tau0 = (-D^{neum-}_y d0, D^{neum-}_x d0)             (def:backdiffNeumann)
//   f1   = P_K tau0 / delta
//   per iteration: w = vecdiv p, phi = Delta^dagger div w  (dct.cu)
//                  z = P_K w - f1 = w - grad phi - f1
//                  psi_k = grad z_k, p_k <- (p_k + t psi_k) / (1 + t |psi_k|)
//   tau = P_K tau0 - delta P_K vecdiv p = -delta z
// Arrays live on the extended grid R x C = (N2+1) x (N1+1) with a padded pitch.
// The dual p may be stored as FP32 or in 16 bits (tvs_storage, Stor<S>): it
// is widened to FP32 when its box is read, the arithmetic is FP32, and 16-bit
// stores of the updated p round stochastically (seed = update number).
#include "tvs_internal.cuh"
#include "prof.h"
#include "tma.cuh"

#include <mutex>
#include <type_traits>

namespace tvs {

constexpr int kTX = 32;   // tile width (outputs)
constexpr int kTY = 32;   // tile height (outputs)
constexpr int kBY = 8;    // thread rows; each thread does kTY / kBY output rows

// The tiled stencils below receive their inputs as TMA boxes covering the
// tile plus a halo: columns j0 - 4 .. j0 + kTX + 3 are read (16-byte aligned
// start; an FP32 box carries 4 more, unused, see PBox), rows i0 - 2 ..
// i0 + kTY + 1.  Reads outside the grid come back as zeros;
// the D^- rule (x-parts zero in the last column, y-parts in the last row) is
// applied when the box is read.
constexpr int kBW = kTX + 12;     // box width (see PBox for the 4 unused columns)
constexpr int kBH = kTY + 4;      // box height
constexpr int kBoxC = 4;          // box column of grid column j0
constexpr int kBoxR = 2;          // box row of grid row i0
constexpr int kBoxFloats = kBW * kBH;

// The halo points of a phase whose main loop gives warp w the region rows
// w, w + kBY, ... go first to the warps with one row fewer (w >= rows % kBY):
// thread slots are rotated so that warp rows % kBY takes halo point 0.  The
// rotation is a bijection of 0 .. NT - 1, so every point is still done once.
__device__ __forceinline__ int halo_slot(int tid, int rows) {
    constexpr int NT = kTX * kBY;
    return (tid + NT - (rows % kBY) * kTX) % NT;
}

// Box of the dual p in storage S: columns j0 - C0 .. j0 + kTX + C0 - 1 + PAD,
// so that the box starts on a 16-byte boundary for 4- and 2-byte elements.
// In FP32 the last PAD = 4 columns (16 bytes) are never read: they make a
// box row 4 mod 8 words long (16 mod 32 bytes), so the rows of one box column
// fall into 8 groups of banks instead of 4, which halves the bank conflicts
// of the loops that walk the halo columns.  The FP32 phi and f1 boxes have
// that width too.  A 16-bit box keeps 48 columns: 16 more bytes per row would
// leave the fused step four CTAs per SM instead of five.
template <class S>
struct PBox {
    static constexpr int C0 = 16 / (int)sizeof(S);
    static constexpr int PAD = sizeof(S) == 4 ? C0 : 0;
    static constexpr int W = kTX + 2 * C0 + PAD;
    static constexpr int ELEMS = W * kBH;                        // one plane
    static constexpr int BYTES = 4 * ELEMS * (int)sizeof(S);     // four planes
    static constexpr int BYTES_AL = (BYTES + 127) / 128 * 128;
};
static_assert(PBox<float>::W == kBW, "phi and f1 boxes as wide as an FP32 p box");
static_assert((PBox<float>::W * 4) % 32 == 16, "FP32 box rows 4 mod 8 words long");
inline int pbox_width(int storage) {
    const int c0 = 16 / (int)storage_bytes(storage);
    return kTX + 2 * c0 + (storage == TVS_F32 ? c0 : 0);
}

// Cached tensor maps of one field: rebuilt only when the base, sizes, plane
// count or storage change.
template <int BH>
struct MapCache {
    const void* base = nullptr;
    int R = 0, C = 0, pitch = 0, planes = 0, st = 0;
    long plane = 0;
    CUtensorMap map;
    bool get(const void* b, int r, int c, int pt, long pl, int np, CUtensorMap* out, int storage = TVS_F32) {
        if (b != base || r != R || c != C || pt != pitch || pl != plane || np != planes || storage != st) {
            if (!make_tensor_map(&map, b, storage, r, c, pt, pl, np, pbox_width(storage), BH)) return false;
            base = b; R = r; C = c; pitch = pt; plane = pl; planes = np; st = storage;
        }
        *out = map;
        return true;
    }
};
// boxes of kTY + 4 rows (the update, div_vecdiv) and kTY + 5 rows (the fused step)
thread_local MapCache<kBH> g_map_p[4], g_map_phi[2], g_map_f1[2];
thread_local MapCache<kTY + 5> g_map5_p[4], g_map5_phi[2], g_map5_f1[2];
thread_local int g_map_next[3], g_map5_next[3];

template <class MC>
static MC* map_slot(MC* c, int n, int* next, const void* base) {
    for (int i = 0; i < n; ++i)
        if (c[i].base == base) return &c[i];
    MC* r = &c[*next];
    *next = (*next + 1) % n;
    return r;
}

static bool tile_maps(const void* p, int storage, const float* phi, const float* f1, int R, int C, int pitch,
                      long plane, CUtensorMap* mp, CUtensorMap* mphi, CUtensorMap* mf) {
    if (!map_slot(g_map_p, 4, &g_map_next[0], p)->get(p, R, C, pitch, plane, 4, mp, storage)) return false;
    if (phi && !map_slot(g_map_phi, 2, &g_map_next[1], phi)->get(phi, R, C, pitch, (long)R * pitch, 1, mphi))
        return false;
    if (f1 && !map_slot(g_map_f1, 2, &g_map_next[2], f1)->get(f1, R, C, pitch, plane, 2, mf)) return false;
    return true;
}
static bool tile_maps5(const void* p, int storage, const float* phi, const float* f1, int R, int C, int pitch,
                       long plane, CUtensorMap* mp, CUtensorMap* mphi, CUtensorMap* mf) {
    return map_slot(g_map5_p, 4, &g_map5_next[0], p)->get(p, R, C, pitch, plane, 4, mp, storage) &&
           map_slot(g_map5_phi, 2, &g_map5_next[1], phi)->get(phi, R, C, pitch, (long)R * pitch, 1, mphi) &&
           map_slot(g_map5_f1, 2, &g_map5_next[2], f1)->get(f1, R, C, pitch, plane, 2, mf);
}

// One thread issues the box loads of a tile; every thread waits (bounded).
// Returns false (after recording the error and draining) if a box never came.
__device__ __forceinline__ bool tile_load(uint64_t* bar, uint32_t bytes, void* sp, const CUtensorMap* mp, int xp,
                                          float* sphi, const CUtensorMap* mphi, float* sf, const CUtensorMap* mf,
                                          int x, int y, unsigned* err) {
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        mbar_init(bar, 1);
        mbar_init_fence();
        mbar_expect_tx(bar, bytes);
        tma_load_3d(sp, mp, xp, y, 0, bar);
        if (sphi) tma_load_2d(sphi, mphi, x, y, bar);
        if (sf) tma_load_3d(sf, mf, x, y, 0, bar);
    }
    __syncthreads();
    const bool ok = mbar_wait(bar, 0);
    if (__syncthreads_and(ok)) return true;
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        atomicOr(err, 1u);
        (void)mbar_drain(bar, 0);
    }
    return false;
}

// tile_load for the TFS update under programmatic dependent launch: the boxes
// of p and f1 (written two or more launches earlier, so complete once this
// grid may start) are issued before griddepcontrol.wait and overlap the tail
// of the previous kernel; the box of phi, which the previous launch writes,
// is issued after it.
__device__ __forceinline__ bool tile_load_early(uint64_t* bar, uint32_t bytes, void* sp, const CUtensorMap* mp,
                                                int xp, float* sphi, const CUtensorMap* mphi, float* sf,
                                                const CUtensorMap* mf, int x, int y, unsigned* err) {
    const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
    if (lead) {
        mbar_init(bar, 1);
        mbar_init_fence();
        mbar_expect_tx(bar, bytes);
        tma_load_3d(sp, mp, xp, y, 0, bar);
        tma_load_3d(sf, mf, x, y, 0, bar);
    }
    pdl_wait();
    pdl_trigger();
    if (lead) tma_load_2d(sphi, mphi, x, y, bar);
    __syncthreads();
    const bool ok = mbar_wait(bar, 0);
    if (__syncthreads_and(ok)) return true;
    if (lead) {
        atomicOr(err, 1u);
        (void)mbar_drain(bar, 0);
    }
    return false;
}

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
    ProfScope ps(kProfSetup, s);
    tau0_kernel<<<grd, blk, 0, s>>>(d0, d_pitch, n2, n1, tau, pitch, long(plane));
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// s = div(vecdiv p) on the extended grid (the source of the Poisson solve in
// every TFS iteration): p arrives as one TMA box over its four planes, then
// w = vecdiv p on a one-point halo, then s.  D^- reads its argument as zero in
// the last column (x-part) or row (y-part) and outside the grid.
// ---------------------------------------------------------------------------
template <class SP>
constexpr size_t div_smem() {
    return (size_t)PBox<SP>::BYTES_AL + (size_t)2 * (kTY + 1) * (kTX + 1) * 4 + 256;
}

template <class SP>
__global__ void __launch_bounds__(kTX * kBY)
div_vecdiv_kernel(const __grid_constant__ CUtensorMap pmap, int R, int C, int pitch, float* __restrict__ S,
                  unsigned* __restrict__ err) {
    using PB = PBox<SP>;
    pdl_wait();
    pdl_trigger();
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* base = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    const SP* sp = reinterpret_cast<const SP*>(base);   // [4][BH][PB::W]
    constexpr int WH = kTY + 1, WW = kTX + 1;      // w region: rows i0-1.., cols j0-1..
    float* sw = reinterpret_cast<float*>(base + PB::BYTES_AL);   // [2][WH][WW]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sw + 2 * WH * WW + 1) ;
    bar = reinterpret_cast<uint64_t*>((reinterpret_cast<uintptr_t>(bar) + 7) & ~static_cast<uintptr_t>(7));
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    constexpr int NT = kTX * kBY;
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;
    if (!tile_load(bar, PB::BYTES, base, &pmap, j0 - PB::C0, nullptr, nullptr, nullptr, nullptr, j0 - kBoxC,
                   i0 - kBoxR, err))
        return;
    // box value of plane q at grid (i, j) with the D^- rule
    auto P = [&](int q, int i, int j) -> float {
        const float v = Stor<SP>::ld1c(sp + (q * kBH + (i - i0 + kBoxR)) * PB::W + (j - j0 + PB::C0));
        const bool ok = (q & 1) == 0 ? j <= C - 2 : i <= R - 2;
        return ok ? v : 0.f;
    };
    // a warp takes the tile's 32 columns of one w row (no bank conflicts);
    // the halo column j0 - 1 is spread over the CTA
    auto wpoint = [&](int r, int c) {
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        float w1 = 0.f, w2 = 0.f;
        if (i >= 0 && j >= 0 && i < R && j < C) {
            w1 = (P(0, i, j) - P(0, i, j - 1)) + (P(1, i, j) - P(1, i - 1, j));
            w2 = (P(2, i, j) - P(2, i, j - 1)) + (P(3, i, j) - P(3, i - 1, j));
            if (j > C - 2) w1 = 0.f;
            if (i > R - 2) w2 = 0.f;
        }
        sw[r * WW + c] = w1;
        sw[(WH + r) * WW + c] = w2;
    };
    for (int r = ty; r < WH; r += kBY) wpoint(r, tx + 1);
    for (int r = halo_slot(tid, WH); r < WH; r += NT) wpoint(r, 0);
    __syncthreads();
#pragma unroll
    for (int rr = ty; rr < kTY; rr += kBY) {
        const int i = i0 + rr, j = j0 + tx;
        if (i < R && j < C) {
            const int r = rr + 1, c = tx + 1;
            S[(size_t)i * pitch + j] = (sw[r * WW + c] - sw[r * WW + c - 1]) + (sw[(WH + r) * WW + c] - sw[(WH + r - 1) * WW + c]);
        }
    }
}

cudaError_t launch_div_vecdiv_st(const void* p, int storage, int R, int C, int pitch, long plane, float* dst,
                                 unsigned* err, cudaStream_t s) {
    CUtensorMap mp, unused;
    if (!tile_maps(p, storage, nullptr, nullptr, R, C, pitch, plane, &mp, &unused, &unused))
        return cudaErrorInvalidValue;
    dim3 blk(kTX, kBY), grd((C + kTX - 1) / kTX, (R + kTY - 1) / kTY);
    ProfScope ps(kProfOther, s);
    cudaError_t e = cudaErrorInvalidValue;
    TVS_STORAGE_SWITCH(storage, {
        static std::once_flag once;
        std::call_once(once, [] {
            cudaFuncSetAttribute(div_vecdiv_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)div_smem<S>());
        });
        e = launch_pdl(div_vecdiv_kernel<S>, grd, blk, div_smem<S>(), s, mp, R, C, pitch, dst, err);
    })
    return e;
}

cudaError_t launch_div_vecdiv(const float* p, int R, int C, int pitch, long plane, float* S, unsigned* err,
                              cudaStream_t s) {
    return launch_div_vecdiv_st(p, TVS_F32, R, C, pitch, plane, S, err, s);
}

// ---------------------------------------------------------------------------
// out = scale * (u - grad phi) for a 2-plane field u (the last step of P_K).
// out may be u itself (each thread reads its own element of u before writing
// it), so u and out are plain pointers read with ordinary loads.
// ---------------------------------------------------------------------------
__global__ void grad_sub_kernel(const float* u, int upitch, long uplane,
                                const float* __restrict__ phi, int ppitch, int R, int C, float scale,
                                float* out, int opitch, long oplane) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y * blockDim.y + threadIdx.y;
    if (i >= R || j >= C) return;
    const float pc = __ldg(&phi[(size_t)i * ppitch + j]);
    const float gx = (j < C - 1) ? __ldg(&phi[(size_t)i * ppitch + j + 1]) - pc : 0.f;
    const float gy = (i < R - 1) ? __ldg(&phi[(size_t)(i + 1) * ppitch + j]) - pc : 0.f;
    const float ux = u[(size_t)i * upitch + j];
    const float uy = u[uplane + (size_t)i * upitch + j];
    out[(size_t)i * opitch + j] = scale * (ux - gx);
    out[oplane + (size_t)i * opitch + j] = scale * (uy - gy);
}

cudaError_t launch_grad_sub(const float* u, int upitch, long uplane, const float* phi, int ppitch, int R,
                            int C, float scale, float* out, int opitch, long oplane, cudaStream_t s) {
    dim3 blk(32, 8), grd((C + 31) / 32, (R + 7) / 8);
    ProfScope ps(kProfSetup, s);
    grad_sub_kernel<<<grd, blk, 0, s>>>(u, upitch, uplane, phi, ppitch, R, C, scale, out, opitch, oplane);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fused TFS update / check.  p (4 planes), phi and f1 (2 planes) arrive as
// TMA boxes; the tile computes z on rows i0-1..i0+TY and columns j0-1..j0+TX
// (the extra leading row/column serves div z for the residual check), psi on
// the TY x TX outputs.
// ---------------------------------------------------------------------------
constexpr int kZH = kTY + 2, kZW = kTX + 2;   // z region: rows i0-1.., cols j0-1..
// The tensor copies land on 128-byte boundaries: the phi box is padded to one.
constexpr int kPhiAl = (kBoxFloats + 31) / 32 * 32;
static_assert((kPhiAl * 4) % 128 == 0, "f1 box of the update on a 128-byte boundary");
static_assert(((kPhiAl + 2 * kBoxFloats + 2 * kZH * kZW) * 4) % 8 == 0, "mbarrier of the update 8-byte aligned");
template <class SP>
constexpr size_t upd_smem() {
    return (size_t)PBox<SP>::BYTES_AL + (size_t)(kPhiAl + 2 * kBoxFloats) * 4 + (size_t)2 * kZH * kZW * 4 + 256;
}

// SP: storage of p (in and out); TT: type of tau_out (float, or a 16-bit
// float type for tau kept inside the library).
template <class SP, bool CHECK, bool WRITE_P, bool WRITE_TAU, class TT = float>
__global__ void __launch_bounds__(kTX * kBY)
tfs_update_kernel(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap phimap,
                  const __grid_constant__ CUtensorMap fmap, SP* __restrict__ pout, int R, int C, int pitch,
                  long plane, float t, float delta, TT* __restrict__ tau_out, int tau_pitch, long tau_plane,
                  double* __restrict__ partial, uint32_t seed, unsigned* __restrict__ err) {
    // every caller launches this right after the Poisson solve that writes phi
    // (four launches that read p and write only phi's plane and the error word),
    // so p and f1 may be read before griddepcontrol.wait (tile_load_early)
    using PB = PBox<SP>;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* base = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    const SP* sp = reinterpret_cast<const SP*>(base);                  // [4][BH][PB::W]
    float* sphi = reinterpret_cast<float*>(base + PB::BYTES_AL);      // [BH][BW], padded to 128 bytes
    float* sf = sphi + kPhiAl;                     // [2][BH][BW]
    float* sz = sf + 2 * kBoxFloats;               // [2][ZH][ZW]
    uint64_t* bar = reinterpret_cast<uint64_t*>(sz + 2 * kZH * kZW);   // 8-byte aligned (even float count)
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    constexpr int NT = kTX * kBY;
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;
    if (!tile_load_early(bar, PB::BYTES + 3 * kBoxFloats * 4, base, &pmap, j0 - PB::C0, sphi, &phimap, sf, &fmap,
                         j0 - kBoxC, i0 - kBoxR, err))
        return;
    // box offsets of grid point (i, j): phi and f1, and p (widened to float)
    auto B = [&](int i, int j) -> int { return (i - i0 + kBoxR) * kBW + (j - j0 + kBoxC); };
    auto PV = [&](int q, int i, int j) -> float {
        return Stor<SP>::ld1c(sp + (q * kBH + (i - i0 + kBoxR)) * PB::W + (j - j0 + PB::C0));
    };

    // z = w - grad phi - f1 on the z region (zero outside the grid); w = vecdiv p
    // with D^- reading x-parts as zero in the last column and y-parts in the last row.
    // A warp takes the tile's 32 columns of one z row (no bank conflicts); the
    // halo columns j0 - 1 and j0 + 32 are spread over the CTA.
    auto zpoint = [&](int r, int c) {
        const int i = i0 - 1 + r, j = j0 - 1 + c;
        float z1 = 0.f, z2 = 0.f;
        if (i >= 0 && i < R && j >= 0 && j < C) {
            const int o = B(i, j);
            const float xm = (j <= C - 2) ? 1.f : 0.f;   // x-part at (i, j) read as zero in the last column
            const float ym = (i <= R - 2) ? 1.f : 0.f;   // y-part at (i, j) read as zero in the last row
            const float w1 = (PV(0, i, j) * xm - PV(0, i, j - 1)) + (PV(1, i, j) * ym - PV(1, i - 1, j));
            const float w2 = (PV(2, i, j) * xm - PV(2, i, j - 1)) + (PV(3, i, j) * ym - PV(3, i - 1, j));
            const float pc = sphi[o];
            const float gx = (j < C - 1) ? sphi[o + 1] - pc : 0.f;
            const float gy = (i < R - 1) ? sphi[o + kBW] - pc : 0.f;
            z1 = w1 - gx - sf[o];
            z2 = w2 - gy - sf[kBoxFloats + o];
        }
        sz[r * kZW + c] = z1;
        sz[(kZH + r) * kZW + c] = z2;
    };
    for (int r = ty; r < kZH; r += kBY) zpoint(r, tx + 1);
    for (int e = halo_slot(tid, kZH); e < 2 * kZH; e += NT) zpoint(e >> 1, (e & 1) ? kZW - 1 : 0);
    __syncthreads();

    // check sums: each thread adds the 8 terms of its 4 points and 2 channels
    // in FP32 (relative error of a few ulp); the block reduction carries FP32
    // pairs and the cross-block sum is FP64
    float ks[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float pmax2 = 0.0f, dmax = 0.0f;
#pragma unroll
    for (int rr = ty; rr < kTY; rr += kBY) {
        const int i = i0 + rr, j = j0 + tx;
        if (i < R && j < C) {
            const int r = rr + 1, c = tx + 1;   // position in the z region
            const int ob = B(i, j);
            const size_t o = (size_t)i * pitch + j;
            float zc[2], gx[2], gy[2], pv[4];
#pragma unroll
            for (int k = 0; k < 2; ++k) {
                const float* zk = sz + k * kZH * kZW;
                zc[k] = zk[r * kZW + c];
                gx[k] = (j < C - 1) ? zk[r * kZW + c + 1] - zc[k] : 0.f;
                gy[k] = (i < R - 1) ? zk[(r + 1) * kZW + c] - zc[k] : 0.f;
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) pv[q] = PV(q, i, j);
            if (WRITE_P) {
                // |psi_k| = s2 rsqrt(s2) (the 1e-30 keeps it finite at psi = 0, far
                // below the resolution of |psi|), one reciprocal per channel
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float s2 = fmaf(gx[k], gx[k], fmaf(gy[k], gy[k], 1e-30f));
                    const float inv = rcp_ftz(fmaf(t, s2 * rsqrt_ftz(s2), 1.0f));
                    const float vx = fmaf(t, gx[k], pv[2 * k]) * inv, vy = fmaf(t, gy[k], pv[2 * k + 1]) * inv;
                    // 16-bit dual: one hash per point, 8 random bits for each of its four planes
                    const uint32_t h = sizeof(SP) == 4 ? 0u : rkey(seed, o, 0);
                    Stor<SP>::st1r8(pout + (size_t)(2 * k) * plane + o, vx, (h >> (16 * k)) & 0xffU);
                    Stor<SP>::st1r8(pout + (size_t)(2 * k + 1) * plane + o, vy, (h >> (16 * k + 8)) & 0xffU);
                }
            }
            if (WRITE_TAU) {
                tau_out[(size_t)i * tau_pitch + j] = TT(-delta * zc[0]);
                tau_out[tau_plane + (size_t)i * tau_pitch + j] = TT(-delta * zc[1]);
            }
            if (CHECK) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float a = gx[k], b = gy[k], px = pv[2 * k], py = pv[2 * k + 1];
                    const float s2 = fmaf(a, a, fmaf(b, b, 1e-30f));
                    const float ng = s2 * rsqrt_ftz(s2);            // |grad z_k| (hardware rsqrt, ~2 ulp)
                    ks[0] += ng;
                    ks[1] += ng - fmaf(a, px, b * py);
                    ks[2] = fmaf(zc[k], zc[k], ks[2]);
                    const float zf = zc[k] + sf[k * kBoxFloats + ob];
                    ks[3] = fmaf(zf, zf, ks[3]);
                    pmax2 = fmaxf(pmax2, fmaf(px, px, py * py));
                }
                // div z with the zero-extension rule of D^- (z_1 read as zero in
                // the last column, z_2 in the last row)
                const float z1c = (j <= C - 2) ? zc[0] : 0.f;
                const float z1l = (j >= 1) ? sz[r * kZW + c - 1] : 0.f;
                const float z2c = (i <= R - 2) ? zc[1] : 0.f;
                const float z2u = (i >= 1) ? sz[(kZH + r - 1) * kZW + c] : 0.f;
                dmax = fmaxf(dmax, fabsf((z1c - z1l) + (z2c - z2u)));
            }
        }
    }
    if (CHECK)
        block_reduce_store_tfs<NT>(ks, sqrtf(pmax2), dmax,
                                   partial + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kRedSlots, tid);
}

int tfs_blocks(int R, int C) { return ((C + kTX - 1) / kTX) * ((R + kTY - 1) / kTY); }

cudaError_t tfs_set_wait_limit(long long cycles) { return set_wait_limit_here(cycles); }

template <class SP, bool CK, bool WP, bool WT, class TT>
static cudaError_t tfs_update_go(dim3 grd, dim3 blk, cudaStream_t s, const CUtensorMap& mp, const CUtensorMap& mphi,
                                 const CUtensorMap& mf, void* pout, int R, int C, int pitch, long plane, float t,
                                 float delta, void* tau_out, int tau_pitch, long tau_plane, double* partial,
                                 uint32_t seed, unsigned* err) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(tfs_update_kernel<SP, CK, WP, WT, TT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)upd_smem<SP>());
    });
    return launch_pdl(tfs_update_kernel<SP, CK, WP, WT, TT>, grd, blk, upd_smem<SP>(), s, mp, mphi, mf,
                      static_cast<SP*>(pout), R, C, pitch, plane, t, delta, static_cast<TT*>(tau_out), tau_pitch,
                      tau_plane, partial, seed, err);
}

// ---------------------------------------------------------------------------
// The TFS update fused with the source of the next Poisson solve:
//   p <- the Chambolle update of p (as tfs_update_kernel, WRITE_P), then
//   src <- div(vecdiv p) of the new p (as div_vecdiv_kernel).
// div(vecdiv .) takes backward differences twice, so s on the 32 x 32 tile
// needs the new p on the tile plus a two-point halo above and to the left;
// that needs z one row and column further than the update alone, so the
// boxes cover rows i0 - 3 .. i0 + 33 (37 rows; the columns already span
// j0 - 4 .. j0 + 35).  The new p of the 34 x 34 region overwrites the old p
// in its box slot (each point reads only its own old value), rounded exactly
// as it is stored, so s equals what div_vecdiv_kernel computes from the
// stored p; the halo points are recomputed here, not read from the CTAs that
// own them.  Reads 28 and writes 20 algorithmic bytes per point, against 28 +
// 16 for the update and 16 + 4 for a separate div_vecdiv.  src must not alias
// phi (other CTAs still read their phi halo while this one writes src).
// ---------------------------------------------------------------------------
constexpr int kBH5 = kTY + 5;               // box rows i0 - 3 .. i0 + 33
constexpr int kBoxR5 = 3;                   // box row of grid row i0
constexpr int kBoxFloats5 = kBW * kBH5;
constexpr int kZ5 = kTX + 3;                // z region: rows and columns i0 - 2 .. i0 + 32 (35)
constexpr int kU5 = kTX + 2;                // new-p region: i0 - 2 .. i0 + 31 (34)
constexpr int kW5 = kTX + 1;                // w region: i0 - 1 .. i0 + 31 (33)

template <class SP>
struct PBox5 {
    static constexpr int C0 = PBox<SP>::C0;
    static constexpr int W = PBox<SP>::W;
    static constexpr int BYTES = 4 * W * kBH5 * (int)sizeof(SP);
    static constexpr int BYTES_AL = (BYTES + 127) / 128 * 128;
};
// The tensor copies land on 128-byte boundaries: the phi box is padded to one
// (1480 floats are not a multiple of 32), so the f1 box behind it is aligned.
constexpr int kPhi5Al = (kBoxFloats5 + 31) / 32 * 32;
static_assert((kPhi5Al * 4) % 128 == 0, "f1 box of the fused step on a 128-byte boundary");
static_assert(((kPhi5Al + 2 * kBoxFloats5 + 2 * kZ5 * kZ5) * 4) % 8 == 0, "mbarrier of the fused step 8-byte aligned");
template <class SP>
constexpr size_t step_smem() {
    return (size_t)PBox5<SP>::BYTES_AL + (size_t)(kPhi5Al + 2 * kBoxFloats5) * 4 + (size_t)2 * kZ5 * kZ5 * 4 + 256;
}
static_assert(2 * kW5 * kW5 <= kPhi5Al + 2 * kBoxFloats5, "w fits over the phi and f1 boxes");

template <class SP, bool CHECK>
__global__ void __launch_bounds__(kTX * kBY)
tfs_step_kernel(const __grid_constant__ CUtensorMap pmap, const __grid_constant__ CUtensorMap phimap,
                const __grid_constant__ CUtensorMap fmap, SP* __restrict__ pout, float* __restrict__ src, int R,
                int C, int pitch, long plane, float t, double* __restrict__ partial, uint32_t seed,
                unsigned* __restrict__ err) {
    using PB = PBox5<SP>;
    extern __shared__ __align__(128) unsigned char smem_dyn[];
    unsigned char* base = smem_dyn + ((128u - (smem_u32(smem_dyn) & 127u)) & 127u);
    SP* sp = reinterpret_cast<SP*>(base);                             // [4][BH5][PB::W]
    float* sphi = reinterpret_cast<float*>(base + PB::BYTES_AL);      // [BH5][BW], padded to 128 bytes
    float* sf = sphi + kPhi5Al;                    // [2][BH5][BW]
    float* sz = sf + 2 * kBoxFloats5;              // [2][Z5][Z5]
    float* sw = sphi;                              // [2][W5][W5], over phi and f1 once z is done
    uint64_t* bar = reinterpret_cast<uint64_t*>(sz + 2 * kZ5 * kZ5);
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tid = ty * kTX + tx;
    constexpr int NT = kTX * kBY;
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;
    if (!tile_load_early(bar, PB::BYTES + 3 * kBoxFloats5 * 4, base, &pmap, j0 - PB::C0, sphi, &phimap, sf, &fmap,
                         j0 - kBoxC, i0 - kBoxR5, err))
        return;
    auto B = [&](int i, int j) -> int { return (i - i0 + kBoxR5) * kBW + (j - j0 + kBoxC); };
    auto PO = [&](int q, int i, int j) -> int { return (q * kBH5 + (i - i0 + kBoxR5)) * PB::W + (j - j0 + PB::C0); };
    auto PV = [&](int q, int i, int j) -> float { return Stor<SP>::ld1c(sp + PO(q, i, j)); };

    // Every phase works on a region a few columns wider than the tile: a warp
    // takes the tile's 32 columns of one region row (contiguous, no bank
    // conflicts), and a second loop spreads the few halo columns over the CTA.
    // Tiles whose regions lie inside the grid away from its last row and column
    // (almost all) run the phases without bounds checks and boundary masks
    // (EDGE false; the masks would all pass there, so the results are the same).
    float ks[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float pmax2 = 0.0f, dmax = 0.0f;
    const bool interior = i0 >= kTY && j0 >= kTX && i0 + kTY + 2 <= R && j0 + kTX + 2 <= C;
    auto phases = [&](auto edge_tag) {
        constexpr bool EDGE = decltype(edge_tag)::value;
        // z = vecdiv p - grad phi - f1 on rows/columns i0 - 2 .. i0 + 32 (as tfs_update_kernel)
        auto zpoint = [&](int r, int c) {
            const int i = i0 - 2 + r, j = j0 - 2 + c;
            float z1 = 0.f, z2 = 0.f;
            if (!EDGE || (i >= 0 && i < R && j >= 0 && j < C)) {
                const int o = B(i, j);
                const float xm = (!EDGE || j <= C - 2) ? 1.f : 0.f;
                const float ym = (!EDGE || i <= R - 2) ? 1.f : 0.f;
                const float w1 = (PV(0, i, j) * xm - PV(0, i, j - 1)) + (PV(1, i, j) * ym - PV(1, i - 1, j));
                const float w2 = (PV(2, i, j) * xm - PV(2, i, j - 1)) + (PV(3, i, j) * ym - PV(3, i - 1, j));
                const float pc = sphi[o];
                const float gx = (!EDGE || j < C - 1) ? sphi[o + 1] - pc : 0.f;
                const float gy = (!EDGE || i < R - 1) ? sphi[o + kBW] - pc : 0.f;
                z1 = w1 - gx - sf[o];
                z2 = w2 - gy - sf[kBoxFloats5 + o];
            }
            sz[r * kZ5 + c] = z1;
            sz[(kZ5 + r) * kZ5 + c] = z2;
        };
        for (int r = ty; r < kZ5; r += kBY) zpoint(r, tx + 2);
        for (int e = halo_slot(tid, kZ5); e < 3 * kZ5; e += NT) {   // region columns 0, 1 and 34
            const int r = e / 3, k = e - 3 * r;
            zpoint(r, k < 2 ? k : kZ5 - 1);
        }
        __syncthreads();

        // the update on rows/columns i0 - 2 .. i0 + 31, in place in the p box; the
        // tile itself also goes to pout; CHECK: the gap terms at the input p (tile only)
        auto upoint = [&](int r, int c) {                   // z region position of (i, j) is (r, c)
            const int i = i0 - 2 + r, j = j0 - 2 + c;
            const bool in_grid = !EDGE || (i >= 0 && j >= 0 && i < R && j < C);
            const bool tile = r >= 2 && c >= 2 && in_grid;
            float pv[4] = {0.f, 0.f, 0.f, 0.f};
            float vnew[4] = {0.f, 0.f, 0.f, 0.f};
            float zc[2] = {0.f, 0.f}, gx[2] = {0.f, 0.f}, gy[2] = {0.f, 0.f};
            if (in_grid) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float* zk = sz + k * kZ5 * kZ5;
                    zc[k] = zk[r * kZ5 + c];
                    gx[k] = (!EDGE || j < C - 1) ? zk[r * kZ5 + c + 1] - zc[k] : 0.f;
                    gy[k] = (!EDGE || i < R - 1) ? zk[(r + 1) * kZ5 + c] - zc[k] : 0.f;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) pv[q] = PV(q, i, j);
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float s2 = fmaf(gx[k], gx[k], fmaf(gy[k], gy[k], 1e-30f));
                    const float inv = rcp_ftz(fmaf(t, s2 * rsqrt_ftz(s2), 1.0f));
                    vnew[2 * k] = fmaf(t, gx[k], pv[2 * k]) * inv;
                    vnew[2 * k + 1] = fmaf(t, gy[k], pv[2 * k + 1]) * inv;
                }
            }
            const size_t o = (size_t)i * pitch + j;
            const uint32_t h = (sizeof(SP) == 4 || !in_grid) ? 0u : rkey(seed, o, 0);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                SP* slot = sp + PO(q, i, j);
                // the same rounding as tfs_update_kernel's store of this point (zero outside the grid)
                Stor<SP>::st1r8(slot, vnew[q], (h >> (8 * q)) & 0xffU);
                if (tile) {
                    if constexpr (sizeof(SP) == 4) pout[(size_t)q * plane + o] = vnew[q];
                    else pout[(size_t)q * plane + o] = *slot;
                }
            }
            if (CHECK && tile) {
#pragma unroll
                for (int k = 0; k < 2; ++k) {
                    const float a = gx[k], b = gy[k], px = pv[2 * k], py = pv[2 * k + 1];
                    const float s2 = fmaf(a, a, fmaf(b, b, 1e-30f));
                    const float ng = s2 * rsqrt_ftz(s2);
                    ks[0] += ng;
                    ks[1] += ng - fmaf(a, px, b * py);
                    ks[2] = fmaf(zc[k], zc[k], ks[2]);
                    const float zf = zc[k] + sf[k * kBoxFloats5 + B(i, j)];
                    ks[3] = fmaf(zf, zf, ks[3]);
                    pmax2 = fmaxf(pmax2, fmaf(px, px, py * py));
                }
                const float z1c = (!EDGE || j <= C - 2) ? zc[0] : 0.f;
                const float z1l = (!EDGE || j >= 1) ? sz[r * kZ5 + c - 1] : 0.f;
                const float z2c = (!EDGE || i <= R - 2) ? zc[1] : 0.f;
                const float z2u = (!EDGE || i >= 1) ? sz[(kZ5 + r - 1) * kZ5 + c] : 0.f;
                dmax = fmaxf(dmax, fabsf((z1c - z1l) + (z2c - z2u)));
            }
        };
        for (int r = ty; r < kU5; r += kBY) upoint(r, tx + 2);
        for (int e = halo_slot(tid, kU5); e < 2 * kU5; e += NT) upoint(e >> 1, e & 1);   // region columns 0, 1
        __syncthreads();

        // w = vecdiv p_new on rows/columns i0 - 1 .. i0 + 31, then s = div w on the
        // tile (as div_vecdiv_kernel, with the D^- rule)
        auto P = [&](int q, int i, int j) -> float {
            const float v = PV(q, i, j);
            if constexpr (!EDGE) return v;
            const bool ok = (q & 1) == 0 ? j <= C - 2 : i <= R - 2;
            return ok ? v : 0.f;
        };
        auto wpoint = [&](int r, int c) {
            const int i = i0 - 1 + r, j = j0 - 1 + c;
            float w1 = 0.f, w2 = 0.f;
            if (!EDGE || (i >= 0 && j >= 0 && i < R && j < C)) {
                w1 = (P(0, i, j) - P(0, i, j - 1)) + (P(1, i, j) - P(1, i - 1, j));
                w2 = (P(2, i, j) - P(2, i, j - 1)) + (P(3, i, j) - P(3, i - 1, j));
                if (EDGE && j > C - 2) w1 = 0.f;
                if (EDGE && i > R - 2) w2 = 0.f;
            }
            sw[r * kW5 + c] = w1;
            sw[(kW5 + r) * kW5 + c] = w2;
        };
        for (int r = ty; r < kW5; r += kBY) wpoint(r, tx + 1);
        for (int r = halo_slot(tid, kW5); r < kW5; r += NT) wpoint(r, 0);   // region column 0
        __syncthreads();
#pragma unroll
        for (int rr = ty; rr < kTY; rr += kBY) {
            const int i = i0 + rr, j = j0 + tx;
            if (!EDGE || (i < R && j < C)) {
                const int r = rr + 1, c = tx + 1;
                src[(size_t)i * pitch + j] =
                    (sw[r * kW5 + c] - sw[r * kW5 + c - 1]) + (sw[(kW5 + r) * kW5 + c] - sw[(kW5 + r - 1) * kW5 + c]);
            }
        }
    };
    if (interior) phases(std::false_type{});
    else phases(std::true_type{});
    if (CHECK)
        block_reduce_store_tfs<NT>(ks, sqrtf(pmax2), dmax,
                                   partial + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * kRedSlots, tid);
}

template <class SP, bool CK>
static cudaError_t tfs_step_go(dim3 grd, dim3 blk, cudaStream_t s, const CUtensorMap& mp, const CUtensorMap& mphi,
                               const CUtensorMap& mf, void* pout, float* src, int R, int C, int pitch, long plane,
                               float t, double* partial, uint32_t seed, unsigned* err) {
    static std::once_flag once;
    std::call_once(once, [] {
        cudaFuncSetAttribute(tfs_step_kernel<SP, CK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)step_smem<SP>());
    });
    return launch_pdl(tfs_step_kernel<SP, CK>, grd, blk, step_smem<SP>(), s, mp, mphi, mf, static_cast<SP*>(pout),
                      src, R, C, pitch, plane, t, partial, seed, err);
}

cudaError_t launch_tfs_step_st(const void* pin, void* pout, int storage, uint32_t seed, const float* phi,
                               const float* f1, float* src, int R, int C, int pitch, long plane, float t, bool check,
                               double* partial, unsigned* err, cudaStream_t s) {
    if (!pin || !pout || !phi || !f1 || !src || src == phi) return cudaErrorInvalidValue;
    CUtensorMap mp, mphi, mf;
    if (!tile_maps5(pin, storage, phi, f1, R, C, pitch, plane, &mp, &mphi, &mf)) return cudaErrorInvalidValue;
    dim3 blk(kTX, kBY), grd((C + kTX - 1) / kTX, (R + kTY - 1) / kTY);
    ProfScope ps(check ? kProfTfsCheck : kProfTfsUpdate, s);
    if (storage == TVS_F32) {
        if (check) return tfs_step_go<float, true>(grd, blk, s, mp, mphi, mf, pout, src, R, C, pitch, plane, t,
                                                   partial, seed, err);
        return tfs_step_go<float, false>(grd, blk, s, mp, mphi, mf, pout, src, R, C, pitch, plane, t, partial, seed,
                                         err);
    }
    TVS_STORAGE_SWITCH(storage, {
        if (check) return tfs_step_go<S, true>(grd, blk, s, mp, mphi, mf, pout, src, R, C, pitch, plane, t, partial,
                                               seed, err);
        return tfs_step_go<S, false>(grd, blk, s, mp, mphi, mf, pout, src, R, C, pitch, plane, t, partial, seed,
                                     err);
    })
    return cudaErrorInvalidValue;
}

cudaError_t launch_tfs_update_st(const void* pin, void* pout, int storage, uint32_t seed, const float* phi,
                                 const float* f1, int R, int C, int pitch, long plane, float t, float delta,
                                 bool check, bool write_p, void* tau_out, int tau_storage, int tau_pitch,
                                 long tau_plane, double* partial, unsigned* err, cudaStream_t s) {
    CUtensorMap mp, mphi, mf;
    if (!tile_maps(pin, storage, phi, f1, R, C, pitch, plane, &mp, &mphi, &mf)) return cudaErrorInvalidValue;
    dim3 blk(kTX, kBY), grd((C + kTX - 1) / kTX, (R + kTY - 1) / kTY);
    const bool wt = tau_out != nullptr;
    ProfScope ps((check || !write_p) ? kProfTfsCheck : kProfTfsUpdate, s);
#define TVS_TFS(SP, CK, WP, WT, TT)                                                                       \
    return tfs_update_go<SP, CK, WP, WT, TT>(grd, blk, s, mp, mphi, mf, pout, R, C, pitch, plane, t, delta,  \
                                             tau_out, tau_pitch, tau_plane, partial, seed, err)
    if (storage == TVS_F32) {
        if (wt && tau_storage != TVS_F32) return cudaErrorInvalidValue;
        if (!check && write_p && !wt) TVS_TFS(float, false, true, false, float);
        if (check && write_p && !wt) TVS_TFS(float, true, true, false, float);
        if (check && !write_p && wt) TVS_TFS(float, true, false, true, float);
        if (check && !write_p && !wt) TVS_TFS(float, true, false, false, float);
        if (!check && !write_p && wt) TVS_TFS(float, false, false, true, float);
        TVS_TFS(float, true, true, true, float);
    }
    // 16-bit duals: the plain and checked updates and the final report with tau
    TVS_STORAGE_SWITCH(storage, {
        if (!check && write_p && !wt) TVS_TFS(S, false, true, false, float);
        if (check && write_p && !wt) TVS_TFS(S, true, true, false, float);
        if (check && !write_p && wt) {
            if (tau_storage == TVS_F32) TVS_TFS(S, true, false, true, float);
            if (tau_storage == TVS_F16) TVS_TFS(S, true, false, true, __half);
            if (tau_storage == TVS_BF16) TVS_TFS(S, true, false, true, __nv_bfloat16);
        }
    })
#undef TVS_TFS
    return cudaErrorInvalidValue;
}

cudaError_t launch_tfs_update(const float* pin, float* pout, const float* phi, const float* f1, int R, int C,
                              int pitch, long plane, float t, float delta, bool check, bool write_p,
                              float* tau_out, int tau_pitch, long tau_plane, double* partial, unsigned* err,
                              cudaStream_t s) {
    return launch_tfs_update_st(pin, pout, TVS_F32, 0u, phi, f1, R, C, pitch, plane, t, delta, check, write_p,
                                tau_out, TVS_F32, tau_pitch, tau_plane, partial, err, s);
}

// ---------------------------------------------------------------------------
// Deterministic reduction of the block partials (fixed partition and order):
// CTA c of the first pass reduces the blocks [c chunk, (c + 1) chunk) into
// stage[c], then one CTA reduces the kFinCTAs stage rows in order.  (One CTA
// reading all partials took about 0.1 ms for the 66 K blocks of an 8193^2 grid.)
// ---------------------------------------------------------------------------
__global__ void finalize_red_kernel(const double* __restrict__ partial, int nblocks, double* __restrict__ stage) {
    constexpr int NT = 256;
    double acc[kRedSlots];
#pragma unroll
    for (int k = 0; k < kRedSlots; ++k) acc[k] = 0.0;
    const int chunk = (nblocks + gridDim.x - 1) / gridDim.x;
    const int b0 = blockIdx.x * chunk, b1 = min(nblocks, b0 + chunk);
    for (int b = b0 + threadIdx.x; b < b1; b += NT) {
#pragma unroll
        for (int k = 0; k < kRedSlots; ++k) {
            const double v = partial[(size_t)b * kRedSlots + k];
            acc[k] = red_is_max(k) ? fmax(acc[k], v) : acc[k] + v;
        }
    }
    block_reduce_store<NT>(acc, stage + (size_t)blockIdx.x * kRedSlots, threadIdx.x);
}

// the stage rows are loaded in parallel, then summed in their fixed order
__global__ void __launch_bounds__(256) finalize_stage_kernel(const double* __restrict__ stage,
                                                             double* __restrict__ result) {
    __shared__ double sh[kFinCTAs * kRedSlots];
    for (int i = threadIdx.x; i < kFinCTAs * kRedSlots; i += blockDim.x) sh[i] = stage[i];
    __syncthreads();
    if (threadIdx.x >= kRedSlots) return;
    const int k = threadIdx.x;
    double v = sh[k];
    for (int c = 1; c < kFinCTAs; ++c) v = red_is_max(k) ? fmax(v, sh[c * kRedSlots + k]) : v + sh[c * kRedSlots + k];
    result[k] = v;
}

void carve_red(Carver& cv, RedBuf& rb, int cap) {
    rb.cap = cap;
    rb.partial = cv.take<double>((size_t)cap * kRedSlots);
    rb.stage = cv.take<double>((size_t)kFinCTAs * kRedSlots);
    rb.result = cv.take<double>(kRedSlots);
    rb.err = cv.take<unsigned>(1);
}

cudaError_t finalize_red(const RedBuf& rb, int nblocks, cudaStream_t s) {
    ProfScope ps(kProfSetup, s, 2);
    finalize_red_kernel<<<kFinCTAs, 256, 0, s>>>(rb.partial, nblocks, rb.stage);
    finalize_stage_kernel<<<1, 256, 0, s>>>(rb.stage, rb.result);
    return cudaGetLastError();
}

}  // namespace tvs
