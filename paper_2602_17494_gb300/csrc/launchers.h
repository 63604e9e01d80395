// Host-side launchers of the kernels in dct.cu, tfs.cu, irv.cu, schwarz.cu.
#pragma once

#include "tvs_internal.cuh"

namespace tvs {

// tfs.cu
cudaError_t launch_tau0(const float* d0, int d_pitch, int n2, int n1, float* tau, int pitch, long plane,
                        cudaStream_t s);
cudaError_t launch_grad_sub(const float* u, int upitch, long uplane, const float* phi, int ppitch, int R, int C,
                            float scale, float* out, int opitch, long oplane, cudaStream_t s);
cudaError_t launch_tfs_update(const float* pin, float* pout, const float* phi, const float* f1, int R, int C,
                              int pitch, long plane, float t, float delta, bool check, bool write_p, float* tau_out,
                              int tau_pitch, long tau_plane, double* partial, cudaStream_t s);
int tfs_blocks(int R, int C);

// irv.cu
cudaError_t launch_xi_f2(const float* d0, int d0_pitch, const float* tau, long tplane, int tpitch, int R, int C,
                         float alpha, float eps, float* f2, int fpitch, cudaStream_t s);
cudaError_t launch_irv1_update(const float* pin, float* pout, const float* f2, int R, int C, int pitch, long plane,
                               float t, float alpha, bool check, bool write_p, float* d_out, int d_pitch,
                               double* partial, cudaStream_t s);
int irv1_blocks(int R, int C);

// schwarz.cu -- Algorithm 2 with Algorithm 3 for IRV1 on the image grid
struct Schwarz2State {
    int m2, m1, s, k;
    double alpha_hat;
    int hmax, wmax, wpad;   // largest subdomain extent, padded width of q storage
    int ncl, band;          // CTAs per subdomain (cluster size) and rows per CTA
    size_t smem;            // dynamic shared memory per CTA
    float* q;               // per-subdomain warm starts, [m2*m1][2][hmax][wpad]
};
tvs_status schwarz2_check(int n2, int n1, const tvs_decomp& dd);
size_t schwarz2_extend(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch);
void schwarz2_carve(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch, Schwarz2State& st);
// Zero the warm starts q_m (Algorithm 3 starts every subdomain from 0).
cudaError_t schwarz2_reset(const Schwarz2State& st, cudaStream_t s);
// n_outer outer iterations of Algorithm 2: p^{n+1} from p^n = *cur, swapping
// *cur and *nxt after each iteration.
cudaError_t schwarz2_iterate(float** cur, float** nxt, const float* f2, int pitch, long plane, int n2, int n1,
                             const Schwarz2State& st, float t, int n_outer, cudaStream_t s);

}  // namespace tvs
