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
//     convolution of length M = 2^m done with two power-of-two Stockham FFTs
//     in shared memory (radix-16 passes held in registers, see below) and a
//     pointwise product with the precomputed filter spectrum.  The last input sample
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
//   (between them the column pass applies D'^{-1} Lambda D' along y as one
//    tridiagonal solve per column: tri_solve.cu)
//   dct_rows_inv  : per pair of rows, inverse DCT along x (in place)
//
// This header holds the templated device code; dct_lm_*.cu instantiate it for
// each FFT length and dct.cu holds the plans and the host dispatch.
#pragma once

#include "dct_launch.h"
#include "prof.h"

#include <mutex>
#include <utility>

namespace tvs {

// ---- shared-memory FFTs ------------------------------------------------------
//
// Stockham autosort FFT (natural order in and out) of length M = 2^m on
// shared-memory arrays.  Every pass is one radix-R step (R = 16 while at least
// 16 points remain per sub-transform, then the remaining 8, 4 or 2): thread u
// loads 16 complex values (16 / R butterflies of radix R), multiplies by the
// twiddles, runs the R-point DFTs in registers and writes the results to
// their autosorted positions.  Each pass reads and writes every element once,
// with one barrier between the reads and the writes (the transform is in
// place), so a thread must own all of its butterflies at once: launches use at
// least nfft * M / 16 threads.  Shared-memory indices are padded by one slot
// every 16 to keep the strided writes of the first passes conflict-free.
//
// Twiddle table: tw[k] = exp(-2 pi i k / M), k < M; the inverse uses conj.

__device__ __forceinline__ int pidx(int a) { return a + (a >> 4); }

// threadIdx.x read through a volatile asm: index arithmetic derived from it
// stays inside the pass that uses it instead of being hoisted (with its live
// registers) to the start of the kernel.
__device__ __forceinline__ int tid_here() {
    int t;
    asm volatile("mov.u32 %0, %%tid.x;" : "=r"(t)::"memory");
    return t;
}

template <bool INV>
__device__ __forceinline__ float2 mul_mi(float2 a) {   // a * (-i) forward, a * (+i) inverse
    return INV ? make_float2(-a.y, a.x) : make_float2(a.y, -a.x);
}

template <bool INV>
__device__ __forceinline__ void dft2(float2& a, float2& b) {
    const float2 t = a;
    a = c_add(t, b);
    b = c_sub(t, b);
}

template <bool INV>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
    const float2 t0 = c_add(a0, a2), t1 = c_sub(a0, a2);
    const float2 t2 = c_add(a1, a3), t3 = mul_mi<INV>(c_sub(a1, a3));
    a0 = c_add(t0, t2);
    a2 = c_sub(t0, t2);
    a1 = c_add(t1, t3);
    a3 = c_sub(t1, t3);
}

// exp(-+ 2 pi i m / 16) constants
template <bool INV>
__device__ __forceinline__ float2 w16(int m) {
    const float c1 = 0.92387953251128674f, s1 = 0.38268343236508977f, h = 0.70710678118654752f;
    float2 w;
    switch (m & 15) {
        case 0: w = make_float2(1.f, 0.f); break;
        case 1: w = make_float2(c1, -s1); break;
        case 2: w = make_float2(h, -h); break;
        case 3: w = make_float2(s1, -c1); break;
        case 4: w = make_float2(0.f, -1.f); break;
        case 5: w = make_float2(-s1, -c1); break;
        case 6: w = make_float2(-h, -h); break;
        case 7: w = make_float2(-c1, -s1); break;
        case 8: w = make_float2(-1.f, 0.f); break;
        case 9: w = make_float2(-c1, s1); break;
        default: w = make_float2(0.f, 0.f); break;
    }
    return INV ? c_conj(w) : w;
}

// In-register DFTs on v[OFF .. OFF + R) of a 16-entry array (natural order
// in and out); all indices are compile-time constants so v stays in registers.
template <bool INV, int OFF>
__device__ __forceinline__ void dft8_at(float2 (&v)[16]) {
    // n = 2 n1 + n2: dft4 over n1, twiddle exp(-2 pi i n2 k1 / 8), dft2 over n2
    dft4<INV>(v[OFF + 0], v[OFF + 2], v[OFF + 4], v[OFF + 6]);
    dft4<INV>(v[OFF + 1], v[OFF + 3], v[OFF + 5], v[OFF + 7]);
    v[OFF + 3] = c_mul(v[OFF + 3], w16<INV>(2));
    v[OFF + 5] = c_mul(v[OFF + 5], w16<INV>(4));
    v[OFF + 7] = c_mul(v[OFF + 7], w16<INV>(6));
    const float2 a0 = v[OFF + 0], b0 = v[OFF + 1], a1 = v[OFF + 2], b1 = v[OFF + 3];
    const float2 a2 = v[OFF + 4], b2 = v[OFF + 5], a3 = v[OFF + 6], b3 = v[OFF + 7];
    v[OFF + 0] = c_add(a0, b0);
    v[OFF + 4] = c_sub(a0, b0);
    v[OFF + 1] = c_add(a1, b1);
    v[OFF + 5] = c_sub(a1, b1);
    v[OFF + 2] = c_add(a2, b2);
    v[OFF + 6] = c_sub(a2, b2);
    v[OFF + 3] = c_add(a3, b3);
    v[OFF + 7] = c_sub(a3, b3);
}

template <bool INV>
__device__ __forceinline__ void dft16(float2 (&v)[16]) {
    // n = 4 n1 + n2: dft4 over n1 (gives A[n2][k1] at v[4 k1 + n2]), twiddle
    // exp(-2 pi i n2 k1 / 16), dft4 over n2; output X[k1 + 4 k2]
    dft4<INV>(v[0], v[4], v[8], v[12]);
    dft4<INV>(v[1], v[5], v[9], v[13]);
    dft4<INV>(v[2], v[6], v[10], v[14]);
    dft4<INV>(v[3], v[7], v[11], v[15]);
    v[5] = c_mul(v[5], w16<INV>(1));
    v[9] = c_mul(v[9], w16<INV>(2));
    v[13] = c_mul(v[13], w16<INV>(3));
    v[6] = c_mul(v[6], w16<INV>(2));
    v[10] = c_mul(v[10], w16<INV>(4));
    v[14] = c_mul(v[14], w16<INV>(6));
    v[7] = c_mul(v[7], w16<INV>(3));
    v[11] = c_mul(v[11], w16<INV>(6));
    v[15] = c_mul(v[15], w16<INV>(9));
    dft4<INV>(v[0], v[1], v[2], v[3]);       // k1 = 0 -> X[0], X[4], X[8], X[12]
    dft4<INV>(v[4], v[5], v[6], v[7]);       // k1 = 1 -> X[1], X[5], X[9], X[13]
    dft4<INV>(v[8], v[9], v[10], v[11]);     // k1 = 2
    dft4<INV>(v[12], v[13], v[14], v[15]);   // k1 = 3
    // transpose 4 x 4: X[k1 + 4 k2] sits at v[4 k1 + k2]
    float2 t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int R, bool INV>
__device__ __forceinline__ void dft_all(float2 (&v)[16]) {
    if (R == 16) {
        dft16<INV>(v);
    } else if (R == 8) {
        dft8_at<INV, 0>(v);
        dft8_at<INV, 8>(v);
    } else if (R == 4) {
        dft4<INV>(v[0], v[1], v[2], v[3]);
        dft4<INV>(v[4], v[5], v[6], v[7]);
        dft4<INV>(v[8], v[9], v[10], v[11]);
        dft4<INV>(v[12], v[13], v[14], v[15]);
    } else {
#pragma unroll
        for (int b = 0; b < 8; ++b) dft2<INV>(v[2 * b], v[2 * b + 1]);
    }
}

// Pointwise step fused into the last pass of an FFT (the outputs are then in
// natural order, output k of a line at k):
//   kEpiNone : none
//   kEpiMul  : X_k *= mul[k]                     (Bluestein's filter spectrum)
//   kEpiOut  : for k < L, X_k <- chirp_k X_k + peel_g rot_k   (Bluestein's output)
enum : int { kEpiNone = 0, kEpiMul = 1, kEpiOut = 2 };
struct FftEpi {
    const float2* mul;
    const float2* chirp;
    const float2* rot;
    const float2* peel;
    int L;
};

// Twiddle bases of a pass of radix R on sub-transforms of NS points:
// w1 = w^tstep and w4 = w^(4 tstep), tstep = M / (R NS) jm, w = exp(-2 pi i / M).
struct TwGlobal {                       // read from the plan's table tw[k] = w^k (global memory)
    const float2* __restrict__ tw;
    template <int M, int R, int NS>
    __device__ __forceinline__ float2 w1(int jm) const { return __ldg(&tw[M / (R * NS) * jm]); }
    template <int M, int R, int NS>
    __device__ __forceinline__ float2 w4(int jm) const { return __ldg(&tw[4 * (M / (R * NS)) * jm]); }
};

// One Stockham pass with everything about the shape known at compile time.
// A thread "unit" holds UV = min(16, M) points: UV / R butterflies of radix R.
// HALFIN (first pass only): the line is zero from M/2 on, so the upper half
// of every butterfly's inputs is the constant 0 and is not read.
template <int R, bool INV, int UPT, int M, int NS, int UVMAX, int EPI, bool HALFIN, class TW>
__device__ __forceinline__ void stockham_pass(float2* buf, int stride, int nfft, const TW tw, const FftEpi& ep) {
    static_assert(!HALFIN || NS == 1, "only the first pass reads the input line");
    constexpr int UV = M < UVMAX ? M : UVMAX;    // points per unit
    constexpr int B = UV / R;                    // butterflies per unit
    constexpr int U = M / UV;                    // units per transform
    constexpr int MR = M / R;
    float2 v[UPT][16];
    const int tid0 = tid_here();
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
        const int u = tid0 + q * blockDim.x;
        if (u < nfft * U) {
            const int g = u / U;
            const int uu = u - g * U;
            const float2* x = buf + (size_t)g * stride;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int j = b * U + uu;        // butterfly index in [0, M/R)
                const int jm = j & (NS - 1);
                // twiddle of input r: w^(tstep r), tstep = jm M / (NS R), as
                // w^r = (w^4)^(r/4) * w^(r%4) from two table entries (a few ulps each)
                float2 wb[4], wa[4];
                wb[0] = make_float2(1.f, 0.f);
                wb[1] = make_float2(1.f, 0.f);
                if constexpr (NS > 1) wb[1] = tw.template w1<M, R, NS>(jm);
                wb[2] = c_mul(wb[1], wb[1]);
                wb[3] = c_mul(wb[2], wb[1]);
                wa[0] = make_float2(1.f, 0.f);
                wa[1] = make_float2(1.f, 0.f);
                if constexpr (R > 4 && NS > 1) {
                    wa[1] = tw.template w4<M, R, NS>(jm);
                    wa[2] = c_mul(wa[1], wa[1]);
                    wa[3] = c_mul(wa[2], wa[1]);
                }
                // with MR a multiple of 16, pidx(j + r MR) = pidx(j) + r (MR + MR / 16)
                const float2* xj = x + pidx(j);
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float2 a = make_float2(0.f, 0.f);
                    if (!(HALFIN && r >= R / 2)) a = (MR % 16 == 0) ? xj[r * (MR + MR / 16)] : x[pidx(j + r * MR)];
                    if (r > 0 && NS > 1) {
                        float2 w = (r >> 2) == 0 ? wb[r & 3]
                                                 : ((r & 3) == 0 ? wa[r >> 2] : c_mul(wa[r >> 2], wb[r & 3]));
                        if (INV) w = c_conj(w);
                        a = c_mul(a, w);
                    }
                    v[q][b * R + r] = a;
                }
            }
        }
    }
    __syncthreads();
    const int tid1 = tid_here();
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
        const int u = tid1 + q * blockDim.x;
        if (u < nfft * U) {
            const int g = u / U;
            const int uu = u - g * U;
            float2* x = buf + (size_t)g * stride;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                if (R == 16) dft16<INV>(v[q]);
                else if (R == 8) { if (b == 0) dft8_at<INV, 0>(v[q]); else dft8_at<INV, 8>(v[q]); }
                else if (R == 4) dft4<INV>(v[q][4 * b], v[q][4 * b + 1], v[q][4 * b + 2], v[q][4 * b + 3]);
                else dft2<INV>(v[q][2 * b], v[q][2 * b + 1]);
                const int j = b * U + uu;
                const int jm = j & (NS - 1);
                const int dst = (j - jm) * R + jm;   // (j / NS) * NS * R + j % NS
                float2* xd = x + pidx(dst);           // NS a multiple of 16: slot r at r (NS + NS / 16)
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    float2 y = v[q][b * R + r];
                    if (EPI == kEpiMul) {
                        y = c_mul(y, __ldg(&ep.mul[dst + r * NS]));
                    } else if (EPI == kEpiOut) {
                        // outputs k >= L are read by no one: not stored.  In this
                        // last pass (NS R = M) every r > R/2 gives k > M/2 >= L - 1,
                        // known at compile time, so those outputs are not computed
                        if (r > R / 2) continue;
                        const int k = dst + r * NS;
                        if (k >= ep.L) continue;
                        y = c_add(c_mul(__ldg(&ep.chirp[k]), y), c_mul(ep.peel[g], __ldg(&ep.rot[k])));
                    }
                    if (NS % 16 == 0) xd[r * (NS + NS / 16)] = y;
                    else x[pidx(dst + r * NS)] = y;
                }
            }
        }
    }
    __syncthreads();
}

// The pass sequence for M = 2^LOGM: radix 16 while at least 16 points remain
// per sub-transform, then the remaining 8, 4 or 2.
template <int LOGM, int LOGNS, bool INV, int UPT, int LOGUV, int EPI, bool HALFIN, class TW>
__device__ __forceinline__ void fft_from(float2* buf, int stride, int nfft, const TW tw, const FftEpi& ep) {
    if constexpr (LOGNS < LOGM) {
        constexpr int REM = LOGM - LOGNS;
        constexpr int LR = REM >= LOGUV ? LOGUV : REM;
        constexpr bool LAST = LOGNS + LR == LOGM;
        stockham_pass<(1 << LR), INV, UPT, (1 << LOGM), (1 << LOGNS), (1 << LOGUV), LAST ? EPI : kEpiNone,
                      HALFIN && LOGNS == 0>(buf, stride, nfft, tw, ep);
        fft_from<LOGM, LOGNS + LR, INV, UPT, LOGUV, EPI, false>(buf, stride, nfft, tw, ep);
    }
}

// All passes of an FFT but the last one (the rest of fft_from's sequence).
template <int LOGM, int LOGNS, bool INV, int UPT, int LOGUV, bool HALFIN, class TW>
__device__ __forceinline__ void fft_until_last(float2* buf, int stride, int nfft, const TW tw) {
    constexpr int REM = LOGM - LOGNS;
    constexpr int LR = REM >= LOGUV ? LOGUV : REM;
    if constexpr (LOGNS + LR < LOGM) {
        stockham_pass<(1 << LR), INV, UPT, (1 << LOGM), (1 << LOGNS), (1 << LOGUV), kEpiNone, HALFIN && LOGNS == 0>(
            buf, stride, nfft, tw, FftEpi{});
        fft_until_last<LOGM, LOGNS + LR, INV, UPT, LOGUV, false>(buf, stride, nfft, tw);
    }
}

// Radix-R DFT of v[OFF .. OFF + R) (natural order in and out).
template <int R, bool INV, int OFF>
__device__ __forceinline__ void dft_slice(float2 (&v)[16]) {
    if constexpr (R == 16) {
        dft16<INV>(v);
    } else if constexpr (R == 8) {
        dft8_at<INV, OFF>(v);
    } else if constexpr (R == 4) {
        dft4<INV>(v[OFF], v[OFF + 1], v[OFF + 2], v[OFF + 3]);
    } else {
        dft2<INV>(v[OFF], v[OFF + 1]);
    }
}

template <int R, bool INV, int B, int... Bs>
__device__ __forceinline__ void dft_slices(float2 (&v)[16], std::integer_sequence<int, Bs...>) {
    (dft_slice<R, INV, Bs * R>(v), ...);
}

// The forward FFT's last pass, the product with the filter spectrum and the
// inverse FFT's first pass, in registers.  In a Stockham sequence the last
// pass of radix RF (NS RF = M) reads and writes, for unit uu, the points
// uu + U m (m < UV, U = M / UV units): butterfly b takes uu + U b + NS r,
// i.e. m = b + r (UV / RF).  The first pass of the next FFT (NS = 1, radix
// UV) reads exactly the same points in the order m.  So the forward outputs
// never go back to shared memory; the one barrier between the pass's reads
// and its writes remains (the writes go to uu UV + m').
template <int RF, int UPT, int M, int UVMAX, class TW>
__device__ __forceinline__ void fft_mid_pass(float2* buf, int stride, int nfft, const TW tw,
                                             const float2* __restrict__ mul) {
    constexpr int UV = M < UVMAX ? M : UVMAX;
    constexpr int B = UV / RF;          // forward butterflies per unit
    constexpr int U = M / UV;
    constexpr int NS = M / RF;          // the forward's last pass; MR = M / RF = NS
    static_assert(NS == U * B, "unit layout");
    float2 v[UPT][16];
    const int tid0 = tid_here();
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
        const int u = tid0 + q * blockDim.x;
        if (u < nfft * U) {
            const int g = u / U;
            const int uu = u - g * U;
            const float2* x = buf + (size_t)g * stride;
#pragma unroll
            for (int b = 0; b < B; ++b) {
                const int j = b * U + uu;            // < NS, so the twiddle of input r is w^(j r)
                float2 wb[4], wa[4];
                wb[0] = make_float2(1.f, 0.f);
                wb[1] = tw.template w1<M, RF, NS>(j);
                wb[2] = c_mul(wb[1], wb[1]);
                wb[3] = c_mul(wb[2], wb[1]);
                wa[0] = make_float2(1.f, 0.f);
                wa[1] = make_float2(1.f, 0.f);
                if constexpr (RF > 4) {
                    wa[1] = tw.template w4<M, RF, NS>(j);
                    wa[2] = c_mul(wa[1], wa[1]);
                    wa[3] = c_mul(wa[2], wa[1]);
                }
#pragma unroll
                for (int r = 0; r < RF; ++r) {
                    float2 a = x[pidx(j + r * NS)];
                    if (r > 0) {
                        const float2 w = (r >> 2) == 0 ? wb[r & 3]
                                                       : ((r & 3) == 0 ? wa[r >> 2] : c_mul(wa[r >> 2], wb[r & 3]));
                        a = c_mul(a, w);
                    }
                    v[q][b * RF + r] = a;
                }
            }
        }
    }
    __syncthreads();
    const int tid1 = tid_here();
#pragma unroll
    for (int q = 0; q < UPT; ++q) {
        const int u = tid1 + q * blockDim.x;
        if (u < nfft * U) {
            const int g = u / U;
            const int uu = u - g * U;
            float2* x = buf + (size_t)g * stride;
            dft_slices<RF, false, B>(v[q], std::make_integer_sequence<int, B>{});
            // forward output r of butterfly b is point m = b + r B; times the filter
            float2 w[16];
#pragma unroll
            for (int b = 0; b < B; ++b)
#pragma unroll
                for (int r = 0; r < RF; ++r) {
                    const int m = b + r * B;
                    w[m] = c_mul(v[q][b * RF + r], __ldg(&mul[uu + U * m]));
                }
            dft_slice<UV, true, 0>(w);
            float2* xd = x + pidx(uu * UV);
#pragma unroll
            for (int r = 0; r < UV; ++r) xd[r] = w[r];   // uu UV .. uu UV + UV - 1 lie in one 16-slot run
        }
    }
    __syncthreads();
}

// ---- in-place decimation-in-frequency FFTs (M >= 2048) ----------------------
//
// For M = 2^LOGM >= 2048 the Bluestein core runs in-place radix passes with
// one 16-point unit per thread (M / 16 threads, one line per CTA):
//   * F = (LOGM - 1) / 4 full radix-16 passes on blocks of N = M, M/16, ...
//     points (stride S = N / 16): a unit loads x[blk N + j + S m], m < 16,
//     takes the 16-point DFT and multiplies output k by w_N^(j k) (Gentleman-
//     Sande), and stores it back to x[blk N + j + S k];
//   * a last pass of radix RL = 2^(LOGM - 4F) on blocks of RL contiguous
//     points, each unit taking 16 / RL of them (the points 16 u .. 16 u + 15).
// The forward output is in digit-reversed order.  The inverse runs the same
// passes backwards (conjugate twiddles on the inputs, then the inverse DFT)
// and ends in natural order, so the filter product needs the filter spectrum
// in digit-reversed order, which is what the same forward passes produce for
// the plan.  A unit writes exactly the points it read, so a pass needs one
// barrier (before the next pass reads) instead of the two of a Stockham pass,
// and the forward last pass, the filter product and the inverse last pass
// run in registers.
template <int LOGM>
struct Dif {
    static constexpr int M = 1 << LOGM;
    static constexpr int F = (LOGM - 1) / 4;          // full radix-16 passes
    static constexpr int RL = 1 << (LOGM - 4 * F);    // radix of the last pass
    static constexpr int SMIN = (M / 16) >> (4 * (F - 1));   // stride of the last full pass
    static_assert(LOGM >= 11 && RL >= 2 && RL <= 16, "in-place passes cover M >= 2048");
};

// Twiddle bases of the in-place passes in shared memory: the pass of stride
// S (block N = 16 S) holds w1[j] = w_N^j and w4[j] = w_N^(4 j), j < S, at
// off(S).  For M = 16384 that is 2 (1024 + 64 + 4) entries (17 KB).
template <int LOGM>
struct TwDifShared {
    static constexpr int off(int S) {
        int o = 0;
        for (int st = (1 << LOGM) / 16; st > S; st /= 16) o += 2 * st;
        return o;
    }
    static constexpr int kTotal = off(Dif<LOGM>::SMIN) + 2 * Dif<LOGM>::SMIN;
    const float2* base;
    template <int M, int R, int NS>
    __device__ __forceinline__ float2 w1(int j) const { return base[off(NS) + j]; }
    template <int M, int R, int NS>
    __device__ __forceinline__ float2 w4(int j) const { return base[off(NS) + NS + j]; }
    // all threads of the CTA; the caller synchronizes before the first use
    __device__ static void fill(float2* dst, const float2* __restrict__ tw) {
        int o = 0, step = 1;   // step = M / N
        for (int st = (1 << LOGM) / 16; st >= Dif<LOGM>::SMIN; st /= 16) {
            for (int i = threadIdx.x; i < st; i += blockDim.x) {
                dst[o + i] = __ldg(&tw[step * i]);
                dst[o + st + i] = __ldg(&tw[4 * step * i]);
            }
            o += 2 * st;
            step *= 16;
        }
    }
};

// w^(j k) for k < 16 from w1 = w^j and w4 = w^(4 j): wa[k / 4] * wb[k % 4].
__device__ __forceinline__ void twiddle_powers(float2 w1, float2 w4, float2 (&wb)[4], float2 (&wa)[4]) {
    wb[0] = make_float2(1.f, 0.f);
    wb[1] = w1;
    wb[2] = c_mul(w1, w1);
    wb[3] = c_mul(wb[2], w1);
    wa[0] = make_float2(1.f, 0.f);
    wa[1] = w4;
    wa[2] = c_mul(w4, w4);
    wa[3] = c_mul(wa[2], w4);
}
__device__ __forceinline__ float2 twiddle_k(const float2 (&wb)[4], const float2 (&wa)[4], int k) {
    return (k >> 2) == 0 ? wb[k & 3] : ((k & 3) == 0 ? wa[k >> 2] : c_mul(wa[k >> 2], wb[k & 3]));
}

// One full radix-16 in-place pass on blocks of N points (S = N / 16).
// Forward: DFT, then output k times w_N^(j k).  Inverse: input m times
// w_N^(-j m), then the inverse DFT.  HALFIN: the line is zero from M/2 on
// (only the first forward pass, N = M).  EPI = kEpiOut (only the last
// inverse pass, N = M): for k < L, X_k <- chirp_k X_k + peel rot_k, and
// points k >= L are not stored (nothing reads them).
// The input of the first forward pass read straight from a pair of rows:
// point n of the line is Makhoul's reordering of the two rows (even columns
// 2n for n < (L+1)/2, odd columns 2(L-1-n)+1 after), times chirp_n, for
// n < L - 1; zero from L - 1 on (the peeled sample z_{L-1}, column 1, is
// staged separately).  a1 == nullptr: the second row is zero.
struct RowPairIn {
    const float* a0;
    const float* a1;
    const float2* chirp;
    int L;
    __device__ __forceinline__ float2 at(int n) const {
        if (n >= L - 1) return make_float2(0.f, 0.f);
        const int c = n < (L + 1) / 2 ? 2 * n : 2 * (L - 1 - n) + 1;
        return c_mul(make_float2(__ldg(a0 + c), a1 ? __ldg(a1 + c) : 0.f), __ldg(&chirp[n]));
    }
};

template <int M, int N, bool INV, bool HALFIN, int EPI, class TW>
__device__ __forceinline__ void dif_pass16(float2* x, const TW tw, const FftEpi& ep,
                                           const RowPairIn* rows = nullptr) {
    constexpr int S = N / 16;
    const int u = tid_here();
    const int j = u & (S - 1);
    const int base = (u - j) * 16 + j;                 // blk N + j, blk = u / S
    float2 v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
        if (HALFIN && m >= 8) v[m] = make_float2(0.f, 0.f);
        else if (rows) v[m] = rows->at(base + S * m);   // first forward pass only (N = M, base = u)
        else v[m] = (S % 16 == 0) ? x[pidx(base) + m * (S + S / 16)] : x[pidx(base + S * m)];
    }
    if constexpr (S > 1) {
        float2 wb[4], wa[4];
        twiddle_powers(tw.template w1<M, 16, S>(j), tw.template w4<M, 16, S>(j), wb, wa);
        if constexpr (INV) {
#pragma unroll
            for (int m = 1; m < 16; ++m) v[m] = c_mul(v[m], c_conj(twiddle_k(wb, wa, m)));
            dft16<true>(v);
        } else {
            dft16<false>(v);
#pragma unroll
            for (int k = 1; k < 16; ++k) v[k] = c_mul(v[k], twiddle_k(wb, wa, k));
        }
    } else {
        dft16<INV>(v);
    }
#pragma unroll
    for (int k = 0; k < 16; ++k) {
        float2 y = v[k];
        if constexpr (EPI == kEpiOut) {
            static_assert(N == M, "the output epilogue belongs to the last inverse pass");
            // points j + S k with k > 8 lie beyond 9 M / 16 > L - 1: never read
            if (k > 8) continue;
            const int p = base + S * k;
            if (p >= ep.L) continue;
            y = c_add(c_mul(__ldg(&ep.chirp[p]), y), c_mul(ep.peel[0], __ldg(&ep.rot[p])));
        }
        if (S % 16 == 0) x[pidx(base) + k * (S + S / 16)] = y;
        else x[pidx(base + S * k)] = y;
    }
    __syncthreads();
}

// The last pass (radix RL on contiguous blocks): unit u holds the points
// 16 u .. 16 u + 15.  MID: forward last pass, times the filter spectrum,
// inverse last pass, all in registers; the spectrum of point 16 u + i (in
// digit-reversed order) is stored at mul[i T + u], T = M / 16 units, so that
// each of the 16 loads of a warp is one contiguous run.  Otherwise the
// forward last pass alone (the plan's filter spectrum).
template <int RL, bool MID, int T>
__device__ __forceinline__ void dif_last(float2* x, const float2* __restrict__ mul) {
    const int u = tid_here();
    float2 v[16];
    float2* xu = x + 17 * u;                            // pidx(16 u + i) = 17 u + i
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = xu[i];
    dft_slices<RL, false, 16 / RL>(v, std::make_integer_sequence<int, 16 / RL>{});
    if constexpr (MID) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = c_mul(v[i], __ldg(&mul[i * T + u]));
        dft_slices<RL, true, 16 / RL>(v, std::make_integer_sequence<int, 16 / RL>{});
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) xu[i] = v[i];
    __syncthreads();
}

// Forward full passes from stride S_ (M / 16 first) down to Dif::SMIN.
template <int LOGM, int S_, bool HALFIN, class TW>
__device__ __forceinline__ void dif_passes_fwd(float2* x, const TW tw) {
    if constexpr (S_ >= Dif<LOGM>::SMIN) {
        dif_pass16<(1 << LOGM), 16 * S_, false, HALFIN, kEpiNone>(x, tw, FftEpi{});
        if constexpr (S_ / 16 >= 1) dif_passes_fwd<LOGM, S_ / 16, false>(x, tw);
    }
}
// Inverse full passes from stride S_ (Dif::SMIN first) up to M / 16; the
// last one applies Bluestein's output step.
template <int LOGM, int S_, class TW>
__device__ __forceinline__ void dif_passes_inv(float2* x, const TW tw, const FftEpi& ep) {
    if constexpr (S_ <= (1 << LOGM) / 16) {
        dif_pass16<(1 << LOGM), 16 * S_, true, false, (S_ == (1 << LOGM) / 16) ? kEpiOut : kEpiNone>(x, tw, ep);
        dif_passes_inv<LOGM, S_ * 16>(x, tw, ep);
    }
}

// Offset (log2) of the last pass in fft_from's sequence for M = 2^LOGM.
template <int LOGM, int LOGUV>
constexpr int last_pass_logns() { return (LOGM - 1) / LOGUV * LOGUV; }

// Unit size and units per thread: 8-point units (radix-8 passes) up to 1024
// points, so short transforms get twice the threads; 16-point units beyond
// (fewer passes, and so fewer barriers, on the critical path of a line pair);
// transforms of 16384 points have 1024 units for 512 threads.
template <int LOGM>
struct FftShape {
    static constexpr int M = 1 << LOGM;
    static constexpr int LOGUV = LOGM <= 10 ? 3 : 4;
    static constexpr int UV = 1 << LOGUV;
    static constexpr int UNITS = M < UV ? 1 : M / UV;
    static constexpr int THREADS = fft_threads(M);
    static constexpr int UPT = UNITS > THREADS ? 2 : 1;
};

// HALFIN: every line is zero from M/2 on.
template <int LOGM, bool INV, int EPI = kEpiNone, bool HALFIN = false, class TW>
__device__ __forceinline__ void fft_stockham(float2* buf, int stride, int nfft, const TW tw,
                                             const FftEpi& ep = FftEpi{}) {
    fft_from<LOGM, 0, INV, FftShape<LOGM>::UPT, FftShape<LOGM>::LOGUV, EPI, HALFIN>(buf, stride, nfft, tw, ep);
}

// Chirp filter spectrum: b[m] = conj(c_m) for lags m in [-(L-2), L-1] stored
// circularly, FFT'd (natural order) and scaled by 1/M.  One block.
template <int LOGM>
__global__ void __launch_bounds__(fft_threads(1 << LOGM)) plan_bhat_kernel(const __grid_constant__ DctPlan pl) {
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
        sm[pidx(m)] = v;
    }
    __syncthreads();
    if constexpr (LOGM >= 11) {
        // the in-place forward passes: the spectrum in their digit-reversed order
        dif_passes_fwd<LOGM, (1 << LOGM) / 16, false>(sm, TwGlobal{pl.tw});
        dif_last<Dif<LOGM>::RL, false, (1 << LOGM) / 16>(sm, nullptr);
    } else {
        fft_stockham<LOGM, false>(sm, padded_len(M), 1, TwGlobal{pl.tw});
    }
    const float inv = 1.0f / (float)M;
    for (int m = threadIdx.x; m < M; m += blockDim.x) {
        // in-place layout: point m = 16 u + i of the digit-reversed spectrum at i (M / 16) + u
        const int d = LOGM >= 11 ? (m & 15) * (M >> 4) + (m >> 4) : m;
        pl.bhat[d] = make_float2(sm[pidx(m)].x * inv, sm[pidx(m)].y * inv);
    }
}

// --------------------------------------------------------------------------
// Bluestein core: buf[g][0 .. L-2] holds the chirped input a_n = z_n c_n,
// buf[g][L-1 .. M) is zero and peel[g] = z_{L-1}.  On return buf[g][k] =
// Z_k = sum_n z_n exp(-2 pi i n k / L) for k < L.
// --------------------------------------------------------------------------
template <int LOGM, class TW>
__device__ __forceinline__ void bluestein(float2* buf, int stride, int G, const DctPlan& pl, const float2* peel,
                                          const TW tw) {
    const FftEpi ep{pl.bhat, pl.chirp, pl.rot, peel, pl.L};
    // FFT, times the filter spectrum (fused into the last pass), inverse FFT,
    // then the chirp and the peeled sample (fused into its last pass)
    // the chirped input occupies [0, L - 1) with L - 1 <= M / 2, so the first
    // pass reads only the lower half
    using Sh = FftShape<LOGM>;
    if constexpr (LOGM >= 11) {
        // in-place passes (one line per CTA): forward, filter, inverse
        dif_passes_fwd<LOGM, (1 << LOGM) / 16, true>(buf, tw);
        dif_last<Dif<LOGM>::RL, true, (1 << LOGM) / 16>(buf, pl.bhat);
        dif_passes_inv<LOGM, Dif<LOGM>::SMIN>(buf, tw, ep);
    } else if constexpr (LOGM > Sh::LOGUV) {
        // at least two passes each: the forward's last pass, the filter and
        // the inverse's first pass run as one (fft_mid_pass)
        constexpr int LN = last_pass_logns<LOGM, Sh::LOGUV>();
        fft_until_last<LOGM, 0, false, Sh::UPT, Sh::LOGUV, true>(buf, stride, G, tw);
        fft_mid_pass<(1 << (LOGM - LN)), Sh::UPT, (1 << LOGM), Sh::UV>(buf, stride, G, tw, pl.bhat);
        fft_from<LOGM, Sh::LOGUV, true, Sh::UPT, Sh::LOGUV, kEpiOut, false>(buf, stride, G, tw, ep);
    } else {
        fft_stockham<LOGM, false, kEpiMul, true>(buf, stride, G, tw, ep);
        fft_stockham<LOGM, true, kEpiOut>(buf, stride, G, tw, ep);
    }
}

// Bluestein core of the in-place path with the first forward pass reading a
// pair of rows directly (no staging through shared memory); the first pass
// takes its twiddles from the plan's global table, the later passes from the
// CTA's shared copy (written before, ordered by the first pass's barrier).
template <int LOGM, class TW>
__device__ __forceinline__ void bluestein_rows(float2* buf, const DctPlan& pl, float2* peel, const TW tw,
                                               const RowPairIn& rows) {
    constexpr int M = 1 << LOGM;
    if (threadIdx.x == 0) *peel = make_float2(__ldg(rows.a0 + 1), rows.a1 ? __ldg(rows.a1 + 1) : 0.f);
    const FftEpi ep{pl.bhat, pl.chirp, pl.rot, peel, pl.L};
    dif_pass16<M, M, false, true, kEpiNone>(buf, TwGlobal{pl.tw}, FftEpi{}, &rows);
    dif_passes_fwd<LOGM, M / 256, false>(buf, tw);
    dif_last<Dif<LOGM>::RL, true, M / 16>(buf, pl.bhat);
    dif_passes_inv<LOGM, Dif<LOGM>::SMIN>(buf, tw, ep);
}

// Rows start on 16-byte boundaries: base and pitch (in floats) allow float4 access.
__device__ __forceinline__ bool vec4_ok(const float* base, int pitch) {
    return ((reinterpret_cast<uintptr_t>(base) & 15) == 0) && ((pitch & 3) == 0);
}

// Makhoul's reordering: position of input sample j in the reordered line.
__device__ __forceinline__ int mk_perm(int j, int L) { return (j & 1) ? (L - 1 - (j >> 1)) : (j >> 1); }

// Stage one packed complex sample z (position n of the reordered line).
__device__ __forceinline__ void stage_sample(float2* bufg, float2* peelg, int n, int L, float2 z,
                                            const DctPlan& pl) {
    if (n == L - 1) *peelg = z;
    else bufg[pidx(n)] = c_mul(z, __ldg(&pl.chirp[n]));
}

// Zeros at [L - 1, M / 2): the part of the lower half that the staged
// samples leave free (the first pass never reads the upper half).
__device__ __forceinline__ void zero_tail(float2* buf, int stride, int G, int L, int M) {
    const int t = M / 2 - (L - 1);
    for (int b = threadIdx.x; b < G * t; b += blockDim.x) {
        const int g = b / t;
        buf[(size_t)g * stride + pidx((L - 1) + (b - g * t))] = make_float2(0.f, 0.f);
    }
}

// Separate two real lines packed as z = x1 + i x2 from Z = DFT(z) and return
// the unnormalised DCT-II values X'_k of both lines.
__device__ __forceinline__ float2 unpack_dct2(const float2* bufg, int k, int L, const DctPlan& pl) {
    const float2 zk = bufg[pidx(k)];
    const float2 zm = bufg[pidx(k == 0 ? 0 : L - k)];
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
// The transforms with in-place passes (FFT lengths of 2048 points or more)
// copy the twiddle bases of their passes into shared memory (2 to 17 KB,
// loaded while the lines are staged) instead of reading the plan's global
// table in every pass.  The shared loads cost fewer L1 wavefronts than the
// strided global ones, and cannot be moved across the passes' barriers (the
// read-only global loads were hoisted, held in registers, and spilled).
// A persistent CTA looping over line pairs would load the bases once, but
// that loop raised register pressure into spills as well.
template <int LOGM>
constexpr bool dct_tw_in_smem() { return LOGM >= 11; }
template <int LOGM>
constexpr int dct_tw_smem_entries() {
    if constexpr (dct_tw_in_smem<LOGM>()) return TwDifShared<LOGM>::kTotal;
    return 0;
}
// Dynamic shared memory of a row-transform CTA: G line buffers, G peeled
// samples, then the twiddle bases.
template <int LOGM>
constexpr size_t dct_rows_smem(int G) {
    return ((size_t)G * (padded_len(1 << LOGM) + 1) + dct_tw_smem_entries<LOGM>()) * sizeof(float2);
}

template <int LOGM>
__device__ __forceinline__ auto dct_twiddles(const DctPlan& pl, float2* smem_tw) {
    if constexpr (dct_tw_in_smem<LOGM>()) {
        TwDifShared<LOGM>::fill(smem_tw, pl.tw);   // ordered before the first pass by the barrier after staging
        return TwDifShared<LOGM>{smem_tw};
    } else {
        return TwGlobal{pl.tw};
    }
}

// Launch bounds: at most 64 registers per thread (as many CTAs as make 1024
// threads per SM), so that registers never limit residency below what the
// shared memory of a line pair allows.
template <RowSource SRC, int LOGM>
__global__ void __launch_bounds__(fft_threads(1 << LOGM), 1024 / fft_threads(1 << LOGM))
dct_rows_fwd_kernel(float* __restrict__ out, int rows, int cols, int pitch, const __grid_constant__ DctPlan pl,
                    RowSrcArgs sa, int G, const __grid_constant__ BatchArgs ba) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const int L = cols, M = pl.M, stride = padded_len(M);
    float2* buf = sm;
    float2* peel = sm + (size_t)G * stride;
    const int2 rr = batch_rows(ba, rows);
    out += (size_t)blockIdx.y * ba.bstride;
    sa.a += (size_t)blockIdx.y * ba.bstride;
    const int npairs = (rr.y - rr.x + 1) >> 1;
    {
        const int base = blockIdx.x * G;
        if (base >= npairs) return;
        const int gc = min(G, npairs - base);
        const auto tw = dct_twiddles<LOGM>(pl, peel + G);
        if constexpr (LOGM >= 11 && SRC == RowSource::Plain) {
            // in-place path: the first pass reads the rows itself (one line pair per CTA)
            const int r0 = rr.x + 2 * base, r1 = r0 + 1;
            const RowPairIn rows{sa.a + row_off(ba, rr, r0, sa.pitch),
                                 r1 < rr.y ? sa.a + row_off(ba, rr, r1, sa.pitch) : nullptr, pl.chirp, L};
            bluestein_rows<LOGM>(buf, pl, peel, tw, rows);
        } else {
        if (SRC == RowSource::Plain && vec4_ok(sa.a, sa.pitch) && vec4_ok(out, pitch)) {
            // groups of four samples, one 16-byte load per row
            const int ng = (L + 3) >> 2;
            for (int b = threadIdx.x; b < gc * ng; b += blockDim.x) {
                const int g = b / ng;
                const int j0 = (b - g * ng) << 2;
                const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
                const float* a0 = sa.a + row_off(ba, rr, r0, sa.pitch) + j0;
                const float* a1 = sa.a + row_off(ba, rr, r1, sa.pitch) + j0;
                float v0[4] = {0.f, 0.f, 0.f, 0.f}, v1[4] = {0.f, 0.f, 0.f, 0.f};
                if (j0 + 3 < L) {
                    const float4 u = __ldg(reinterpret_cast<const float4*>(a0));
                    v0[0] = u.x; v0[1] = u.y; v0[2] = u.z; v0[3] = u.w;
                    if (r1 < rr.y) {
                        const float4 w = __ldg(reinterpret_cast<const float4*>(a1));
                        v1[0] = w.x; v1[1] = w.y; v1[2] = w.z; v1[3] = w.w;
                    }
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (j0 + e < L) {
                            v0[e] = __ldg(a0 + e);
                            if (r1 < rr.y) v1[e] = __ldg(a1 + e);
                        }
                }
#pragma unroll
                for (int e = 0; e < 4; ++e)
                    if (j0 + e < L)
                        stage_sample(buf + (size_t)g * stride, peel + g, mk_perm(j0 + e, L), L,
                                     make_float2(v0[e], v1[e]), pl);
            }
        } else {
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
        }
        zero_tail(buf, stride, gc, L, M);
        __syncthreads();
        bluestein<LOGM>(buf, stride, gc, pl, peel, tw);
        }
        if (vec4_ok(out, pitch)) {
            // groups of four outputs, one 16-byte store per row
            const int ng = (L + 3) >> 2;
            for (int b = threadIdx.x; b < gc * ng; b += blockDim.x) {
                const int g = b / ng;
                const int k0 = (b - g * ng) << 2;
                const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
                float v0[4], v1[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 X = k0 + e < L ? unpack_dct2(buf + (size_t)g * stride, k0 + e, L, pl)
                                                : make_float2(0.f, 0.f);
                    v0[e] = X.x;
                    v1[e] = X.y;
                }
                float* o0 = out + row_off(ba, rr, r0, pitch) + k0;
                float* o1 = out + row_off(ba, rr, r1, pitch) + k0;
                if (k0 + 3 < L) {
                    *reinterpret_cast<float4*>(o0) = make_float4(v0[0], v0[1], v0[2], v0[3]);
                    if (r1 < rr.y) *reinterpret_cast<float4*>(o1) = make_float4(v1[0], v1[1], v1[2], v1[3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (k0 + e < L) {
                            o0[e] = v0[e];
                            if (r1 < rr.y) o1[e] = v1[e];
                        }
                }
            }
        } else {
            for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
                const int g = b / L;
                const int k = b - g * L;
                const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
                const float2 X = unpack_dct2(buf + (size_t)g * stride, k, L, pl);
                out[row_off(ba, rr, r0, pitch) + k] = X.x;
                if (r1 < rr.y) out[row_off(ba, rr, r1, pitch) + k] = X.y;
            }
        }
        __syncthreads();
    }
}

template <int LOGM>
__global__ void __launch_bounds__(fft_threads(1 << LOGM), 1024 / fft_threads(1 << LOGM))
dct_rows_inv_kernel(float* __restrict__ S, int rows, int cols, int pitch, const __grid_constant__ DctPlan pl, int G,
                    const __grid_constant__ BatchArgs ba) {
    extern __shared__ float2 sm[];
    pdl_wait();
    pdl_trigger();
    const int L = cols, M = pl.M, stride = padded_len(M);
    float2* buf = sm;
    float2* peel = sm + (size_t)G * stride;
    const int2 rr = batch_rows(ba, rows);
    S += (size_t)blockIdx.y * ba.bstride;
    const int npairs = (rr.y - rr.x + 1) >> 1;
    const float invL = 1.0f / (float)L;
    {
        const int base = blockIdx.x * G;
        if (base >= npairs) return;
        const int gc = min(G, npairs - base);
        const auto tw = dct_twiddles<LOGM>(pl, peel + G);
        // one thread per pair (k, L - k): the same four loads stage both samples
        const int half = L / 2 + 1;
        for (int b = threadIdx.x; b < gc * half; b += blockDim.x) {
            const int g = b / half;
            const int k = b - g * half;
            const int km = k == 0 ? 0 : L - k;
            if (k > km) continue;                            // each pair once
            const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
            const float* a0 = S + row_off(ba, rr, r0, pitch);
            const float x1k = a0[k], x1m = k ? a0[km] : 0.f;
            float x2k = 0.f, x2m = 0.f;
            if (r1 < rr.y) {
                const float* a1 = S + row_off(ba, rr, r1, pitch);
                x2k = a1[k];
                x2m = k ? a1[km] : 0.f;
            }
            float2* bufg = buf + (size_t)g * stride;
            stage_sample(bufg, peel + g, k, L, pack_dct3(x1k, x1m, x2k, x2m, k, pl), pl);
            if (k != 0 && km != k) stage_sample(bufg, peel + g, km, L, pack_dct3(x1m, x1k, x2m, x2k, km, pl), pl);
        }
        zero_tail(buf, stride, gc, L, M);
        __syncthreads();
        bluestein<LOGM>(buf, stride, gc, pl, peel, tw);
        if (vec4_ok(S, pitch)) {
            // groups of four outputs, one 16-byte store per row
            const int ng = (L + 3) >> 2;
            for (int b = threadIdx.x; b < gc * ng; b += blockDim.x) {
                const int g = b / ng;
                const int j0 = (b - g * ng) << 2;
                const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
                float v0[4], v1[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    const float2 Y = j0 + e < L ? buf[(size_t)g * stride + pidx(mk_perm(j0 + e, L))]
                                                : make_float2(0.f, 0.f);
                    v0[e] = Y.x * invL;
                    v1[e] = -Y.y * invL;
                }
                float* o0 = S + row_off(ba, rr, r0, pitch) + j0;
                float* o1 = S + row_off(ba, rr, r1, pitch) + j0;
                if (j0 + 3 < L) {
                    *reinterpret_cast<float4*>(o0) = make_float4(v0[0], v0[1], v0[2], v0[3]);
                    if (r1 < rr.y) *reinterpret_cast<float4*>(o1) = make_float4(v1[0], v1[1], v1[2], v1[3]);
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e)
                        if (j0 + e < L) {
                            o0[e] = v0[e];
                            if (r1 < rr.y) o1[e] = v1[e];
                        }
                }
            }
        } else {
            for (int b = threadIdx.x; b < gc * L; b += blockDim.x) {
                const int g = b / L;
                const int j = b - g * L;
                const int r0 = rr.x + 2 * (base + g), r1 = r0 + 1;
                const float2 Y = buf[(size_t)g * stride + pidx(mk_perm(j, L))];
                S[row_off(ba, rr, r0, pitch) + j] = Y.x * invL;
                if (r1 < rr.y) S[row_off(ba, rr, r1, pitch) + j] = -Y.y * invL;
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Launchers for one FFT length
// ---------------------------------------------------------------------------
// Shared-memory limit and carve-out of a DCT kernel.  The plan tables (twiddles,
// filter spectrum, chirp, Makhoul twiddles: about 28 M bytes) are read by every
// CTA through L1; the carve-out is sized for at most four CTAs per SM (fewer
// when fewer fit at all: one for the 16384-point transforms) so that the rest
// of the unified L1/shared storage can keep them resident.
template <class K>
inline void allow_dct_smem(K kernel, size_t smem_per_cta = 0) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemBudget + 16 * 1024);
    if (smem_per_cta) {
        const size_t per_sm = 228 * 1024;
        size_t ctas = per_sm / (smem_per_cta + 1024);
        ctas = ctas < 1 ? 1 : (ctas > 4 ? 4 : ctas);
        int pct = (int)((ctas * (smem_per_cta + 1024) * 100 + per_sm - 1) / per_sm);
        pct = pct < 1 ? 1 : (pct > 100 ? 100 : pct);
        cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, pct);
    }
}

template <int LM>
cudaError_t launch_bhat_lm(const DctPlan& pl, cudaStream_t s) {
    static std::once_flag once;
    std::call_once(once, [] { allow_dct_smem(plan_bhat_kernel<LM>); });
    const size_t smem = (size_t)padded_len(pl.M) * sizeof(float2);
    plan_bhat_kernel<LM><<<1, fft_threads(1 << LM), smem, s>>>(pl);
    return cudaGetLastError();
}

template <int LM>
cudaError_t launch_rows_fwd_lm(RowSource src, float* S, int rows, int cols, int pitch, const DctPlan& pl,
                               const RowSrcArgs& sa, const BatchArgs& ba, int nbatch, int maxrows, cudaStream_t s) {
    static std::once_flag once;
    const size_t smem = dct_rows_smem<LM>(1);
    std::call_once(once, [smem] {
        allow_dct_smem(dct_rows_fwd_kernel<RowSource::Plain, LM>, smem);
        allow_dct_smem(dct_rows_fwd_kernel<RowSource::DivField, LM>, smem);
    });
    const dim3 grid((maxrows + 1) / 2, nbatch);
    const int nt = fft_threads(pl.M);
    if (src == RowSource::Plain)
        return launch_pdl(dct_rows_fwd_kernel<RowSource::Plain, LM>, grid, dim3(nt), smem, s, S, rows, cols, pitch, pl,
                          sa, 1, ba);
    if (src == RowSource::DivField)
        return launch_pdl(dct_rows_fwd_kernel<RowSource::DivField, LM>, grid, dim3(nt), smem, s, S, rows, cols, pitch,
                          pl, sa, 1, ba);
    return cudaErrorInvalidValue;
}

template <int LM>
cudaError_t launch_rows_inv_lm(float* S, int rows, int cols, int pitch, const DctPlan& pl, const BatchArgs& ba,
                               int nbatch, int maxrows, cudaStream_t s) {
    static std::once_flag once;
    const size_t smem = dct_rows_smem<LM>(1);
    std::call_once(once, [smem] { allow_dct_smem(dct_rows_inv_kernel<LM>, smem); });
    const dim3 grid((maxrows + 1) / 2, nbatch);
    return launch_pdl(dct_rows_inv_kernel<LM>, grid, dim3(fft_threads(pl.M)), smem, s, S, rows, cols, pitch, pl, 1,
                      ba);
}

#define TVS_DCT_INSTANTIATE(LM)                                                                                   \
    template cudaError_t launch_bhat_lm<LM>(const DctPlan&, cudaStream_t);                                        \
    template cudaError_t launch_rows_fwd_lm<LM>(RowSource, float*, int, int, int, const DctPlan&,                  \
                                                const RowSrcArgs&, const BatchArgs&, int, int, cudaStream_t);      \
    template cudaError_t launch_rows_inv_lm<LM>(float*, int, int, int, const DctPlan&, const BatchArgs&, int, int, \
                                                cudaStream_t);

}  // namespace tvs
