// Launchers of the DCT kernels, one explicit instantiation per FFT length
// M = 2^LM (dct_lm_*.cu); dct.cu dispatches on the runtime length.
#pragma once

#include "tvs_internal.cuh"

namespace tvs {

constexpr int kDctThreads = 512;             // threads per DCT CTA up to 8192-point FFTs
constexpr int kDctThreadsMax = 1024;         // threads per DCT CTA (at most)
constexpr int kMinLogM = 2, kMaxLogM = 14;   // FFT lengths 4 .. 16384 (transform lengths 3 .. 8193)

// Shared-memory FFT arrays are padded by one slot every 16 entries.
__host__ __device__ __forceinline__ int padded_len(int M) { return M + (M >> 4) + 4; }

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

// Row range [x, y) of this CTA's array (blockIdx.y) and the storage offset of row r.
__device__ __forceinline__ int2 batch_rows(const BatchArgs& ba, int rows) {
    return ba.ranges ? ba.ranges[blockIdx.y] : make_int2(0, rows);
}
__device__ __forceinline__ size_t row_off(const BatchArgs& ba, int2 rr, int r, int pitch) {
    return (size_t)(ba.packed ? r - rr.x : r) * pitch;
}


template <int LM>
cudaError_t launch_bhat_lm(const DctPlan& pl, cudaStream_t s);
template <int LM>
cudaError_t launch_rows_fwd_lm(RowSource src, float* S, int rows, int cols, int pitch, const DctPlan& pl,
                               const RowSrcArgs& sa, const BatchArgs& ba, int nbatch, int maxrows, cudaStream_t s);
template <int LM>
cudaError_t launch_rows_inv_lm(float* S, int rows, int cols, int pitch, const DctPlan& pl, const BatchArgs& ba,
                               int nbatch, int maxrows, cudaStream_t s);

// Column pass of the Poisson pseudo-inverse as Neumann tridiagonal solves along
// y (tri_solve.cu): S holds the row-transformed planes; tab the per-column
// coefficients written by build_tri_table for the same rows and cols.
cudaError_t launch_tri_cols(float* S, int rows, int cols, int pitch, const float4* tab, const BatchArgs& ba,
                            int nbatch, cudaStream_t s);
cudaError_t build_tri_table(float4* tab, int rows, int cols, cudaStream_t s);
// The same solve for one unbatched problem with long columns (pp.tsum set):
// chunks of kTriChunk rows, three kernels with coalesced row accesses.
cudaError_t launch_tri_cols_chunked(float* S, int rows, int cols, int pitch, const PoissonPlans& pp,
                                    cudaStream_t s);

// Threads for a transform of length M: one per FFT unit (8 points up to 1024,
// 16 beyond); the 16384-point transforms have 1024 units and 1024 threads.
__host__ __device__ constexpr int fft_threads(int M) {
    const int uv = M <= 1024 ? 8 : 16;
    const int units = M < uv ? 1 : M / uv;
    const int t = (units + 31) / 32 * 32;
    return t < 64 ? 64 : (t > kDctThreadsMax ? kDctThreadsMax : t);
}

// Runs STMT with the compile-time constant LM equal to the runtime value v.
#define TVS_LOGM_CASE(N, STMT) \
    case N: {                  \
        constexpr int LM = N;  \
        STMT;                  \
    } break;
#define TVS_LOGM_SWITCH(v, STMT)                                                                   \
    switch (v) {                                                                                   \
        TVS_LOGM_CASE(2, STMT) TVS_LOGM_CASE(3, STMT) TVS_LOGM_CASE(4, STMT) TVS_LOGM_CASE(5, STMT)  \
        TVS_LOGM_CASE(6, STMT) TVS_LOGM_CASE(7, STMT) TVS_LOGM_CASE(8, STMT) TVS_LOGM_CASE(9, STMT)  \
        TVS_LOGM_CASE(10, STMT) TVS_LOGM_CASE(11, STMT) TVS_LOGM_CASE(12, STMT)                     \
        TVS_LOGM_CASE(13, STMT) TVS_LOGM_CASE(14, STMT)                                            \
        default: break;                                                                            \
    }

}  // namespace tvs
