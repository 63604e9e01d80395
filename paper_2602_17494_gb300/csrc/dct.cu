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
//   tri_cols_solve: per column pair, D'^{-1} Lambda(., k_x) D' along y, which
//                   is a Neumann tridiagonal solve (tri_solve.cu; in place);
//                   long columns go through the chunked form of the same
//                   solve (tri_chunk_* kernels, coalesced rows)
//   dct_rows_inv  : per pair of rows, inverse DCT along x (in place)
#include "dct_launch.h"
#include "prof.h"

#include <cmath>

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
    pl.tw = cv.take<float2>(pl.M);
    pl.bhat = cv.take<float2>(pl.M);
    pl.sig2 = cv.take<float>(L);
}

__global__ void plan_tables_kernel(DctPlan pl) {
    const int L = pl.L, M = pl.M;
    const int n = L > M ? L : M;
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
            pl.sig2[i] = (float)(4.0 * s * s);
        }
        if (i < M) {
            sincospi(2.0 * (double)i / (double)M, &s, &c);
            pl.tw[i] = make_float2((float)c, (float)-s);
        }
    }
}

cudaError_t build_plan(const DctPlan& pl, cudaStream_t s) {
    const int n = pl.L > pl.M ? pl.L : pl.M;
    plan_tables_kernel<<<(n + 255) / 256, 256, 0, s>>>(pl);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = cudaErrorInvalidValue;
    TVS_LOGM_SWITCH(pl.logM, (e = launch_bhat_lm<LM>(pl, s)));
    return e;
}

void carve_poisson(Carver& cv, PoissonPlans& pp, int rows, int cols) {
    carve_plan(cv, pp.row, cols);
    pp.rows = rows;
    pp.tri = cv.take<float4>(2 * (size_t)cols);
    if (rows >= kTriChunkRows) {
        pp.tnch = tri_chunks(rows);
        pp.tsum = cv.take<float>(tri_chunk_floats(rows, cols));
    } else {
        pp.tnch = 0;
        pp.tsum = nullptr;
    }
}

cudaError_t build_poisson(const PoissonPlans& pp, cudaStream_t s) {
    ProfScope ps(kProfSetup, s, 3);
    const cudaError_t e = build_plan(pp.row, s);
    if (e != cudaSuccess) return e;
    return build_tri_table(pp.tri, pp.rows, pp.row.L, s);
}

// --------------------------------------------------------------------------
// Poisson solve: row transforms, tridiagonal column solve, inverse row transforms.
// One pair of lines per CTA (the kernels are latency-bound, so resident warps
// matter more than batching).
// --------------------------------------------------------------------------
static cudaError_t poisson_launch(float* S, int rows, int cols, int pitch, const PoissonPlans& pp, RowSource src,
                                  const RowSrcArgs& sa, int nbatch, const int2* ranges, long bstride, int maxrows,
                                  int packed, cudaStream_t s) {
    if (pp.row.logM < kMinLogM || pp.row.logM > kMaxLogM || rows != pp.rows || cols != pp.row.L)
        return cudaErrorInvalidValue;
    const BatchArgs ba{ranges, bstride, packed};
    cudaError_t e = cudaErrorInvalidValue;
    {
        ProfScope ps(kProfRowsFwd, s);
        TVS_LOGM_SWITCH(pp.row.logM,
                        (e = launch_rows_fwd_lm<LM>(src, S, rows, cols, pitch, pp.row, sa, ba, nbatch, maxrows, s)));
    }
    if (e != cudaSuccess) return e;
    e = cudaErrorInvalidValue;
    {
        const bool chunked = pp.tsum && nbatch == 1 && !ranges;
        ProfScope ps(kProfCols, s, chunked ? 3 : 1);
        if (chunked) e = launch_tri_cols_chunked(S, rows, cols, pitch, pp, s);
        else e = launch_tri_cols(S, rows, cols, pitch, pp.tri, ba, nbatch, s);
    }
    if (e != cudaSuccess) return e;
    e = cudaErrorInvalidValue;
    {
        ProfScope ps(kProfRowsInv, s);
        TVS_LOGM_SWITCH(pp.row.logM,
                        (e = launch_rows_inv_lm<LM>(S, rows, cols, pitch, pp.row, ba, nbatch, maxrows, s)));
    }
    return e;
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
