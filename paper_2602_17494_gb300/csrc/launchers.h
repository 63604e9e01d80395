// Host-side launchers of the kernels in dct.cu, tfs.cu, irv.cu, schwarz.cu.
#pragma once

#include "tvs_internal.cuh"
#include "decomp.cuh"

namespace tvs {

// tfs.cu
cudaError_t launch_tau0(const float* d0, int d_pitch, int n2, int n1, float* tau, int pitch, long plane,
                        cudaStream_t s);
cudaError_t launch_grad_sub(const float* u, int upitch, long uplane, const float* phi, int ppitch, int R, int C,
                            float scale, float* out, int opitch, long oplane, cudaStream_t s);
cudaError_t launch_tfs_update(const float* pin, float* pout, const float* phi, const float* f1, int R, int C,
                              int pitch, long plane, float t, float delta, bool check, bool write_p,
                              float* tau_out, int tau_pitch, long tau_plane, double* partial, unsigned* err,
                              cudaStream_t s);
// The same for a dual p stored as `storage` (tvs_storage; pin and pout in that
// format, 16-bit stores rounded stochastically with `seed`), tau_out in
// `tau_storage` (TVS_F32, or TVS_F16 / TVS_BF16 for a 16-bit dual).
cudaError_t launch_tfs_update_st(const void* pin, void* pout, int storage, uint32_t seed, const float* phi,
                                 const float* f1, int R, int C, int pitch, long plane, float t, float delta,
                                 bool check, bool write_p, void* tau_out, int tau_storage, int tau_pitch,
                                 long tau_plane, double* partial, unsigned* err, cudaStream_t s);
// The update (as launch_tfs_update_st with write_p, no tau) fused with the
// source of the next Poisson solve: src <- div(vecdiv pout).  src must not be
// phi.  Partial sums (check) are the gap terms at pin, as launch_tfs_update_st.
cudaError_t launch_tfs_step_st(const void* pin, void* pout, int storage, uint32_t seed, const float* phi,
                               const float* f1, float* src, int R, int C, int pitch, long plane, float t, bool check,
                               double* partial, unsigned* err, cudaStream_t s);
int tfs_blocks(int R, int C);
// Limit of the bounded TMA waits of the kernels in tfs.cu / irv.cu (SM cycles).
cudaError_t tfs_set_wait_limit(long long cycles);
cudaError_t irv_set_wait_limit(long long cycles);
// err: device word whose bit 0 is set if a bounded wait on the TMA boxes gave up
cudaError_t launch_div_vecdiv(const float* p, int R, int C, int pitch, long plane, float* S, unsigned* err,
                              cudaStream_t s);
cudaError_t launch_div_vecdiv_st(const void* p, int storage, int R, int C, int pitch, long plane, float* dst,
                                 unsigned* err, cudaStream_t s);
// S <- Delta^dagger div(vecdiv p) on the extended grid (phi of the TFS iteration);
// p stored as `storage`
inline cudaError_t tfs_phi_st(const void* p, int storage, float* S, int R, int C, int pitch, long plane,
                              const PoissonPlans& pp, unsigned* err, cudaStream_t s) {
    cudaError_t e = launch_div_vecdiv_st(p, storage, R, C, pitch, plane, S, err, s);
    if (e != cudaSuccess) return e;
    RowSrcArgs sa{S, 0, pitch};
    return poisson_solve(S, R, C, pitch, pp, RowSource::Plain, sa, s);
}
inline cudaError_t tfs_phi(const float* p, float* S, int R, int C, int pitch, long plane, const PoissonPlans& pp,
                           unsigned* err, cudaStream_t s) {
    cudaError_t e = launch_div_vecdiv(p, R, C, pitch, plane, S, err, s);
    if (e != cudaSuccess) return e;
    RowSrcArgs sa{S, 0, pitch};
    return poisson_solve(S, R, C, pitch, pp, RowSource::Plain, sa, s);
}

// irv.cu
cudaError_t launch_xi_f2(const float* d0, int d0_pitch, const float* tau, long tplane, int tpitch, int R, int C,
                         float alpha, float eps, float* f2, int fpitch, cudaStream_t s);
// the same with tau stored as tau_storage (TVS_F32, TVS_F16 or TVS_BF16)
cudaError_t launch_xi_f2_st(const float* d0, int d0_pitch, const void* tau, int tau_storage, long tplane,
                            int tpitch, int R, int C, float alpha, float eps, float* f2, int fpitch, cudaStream_t s);
// p (pin, pout) is stored as `storage` (tvs_storage); everything else is float.
// seed: update counter for the stochastic rounding of 16-bit stores; err:
// device word that gets bit 0 set if a bounded wait inside the kernel gave up.
cudaError_t launch_irv1_update(const void* pin, void* pout, const float* f2, int R, int C, int pitch, long plane,
                               float t, float alpha, bool check, bool write_p, float* d_out, int d_pitch,
                               double* partial, int storage, uint32_t seed, unsigned* err, cudaStream_t s);
int irv1_blocks(int R, int C);
// IRV2 (eq. ir2dualdis): S <- div v, the source of the potential g of tau_perp
// on the n2 x n1 image grid (g = Delta^dagger S); f = alpha (d0 - g); d += g.
cudaError_t launch_potential_src(const float* tau, long tplane, int tpitch, int n2, int n1, float* S, int spitch,
                                 cudaStream_t s);
cudaError_t launch_irv2_f(const float* d0, int d0_pitch, const float* g, int gpitch, int n2, int n1, float alpha,
                          float* f, int fpitch, cudaStream_t s);
cudaError_t launch_add_plane(float* d, int dpitch, const float* g, int gpitch, int n2, int n1, cudaStream_t s);
// W^{1,1} dual (eq. IRW11:dual): p += sign * xi on a dense two-plane n2 x n1 field
cudaError_t launch_shift_xi(float* p, int n2, int n1, const float* tau, long tplane, int tpitch, float eps,
                            float sign, cudaStream_t s);
// Copy `planes` planes of rows x cols between layouts and storage formats
// (element pitches and plane strides in elements of each side's format).
cudaError_t convert_planes(void* dst, int dst_storage, int dpitch, long dplane, const void* src, int src_storage,
                           int spitch, long splane, int rows, int cols, int planes, cudaStream_t s);

// schwarz.cu -- Algorithm 2 with Algorithm 3 for IRV1 on the image grid
struct Schwarz2State {
    int m2, m1, s, k;
    double alpha_hat;
    int hmax, wmax, wpad;   // largest subdomain extent, padded shared-memory row of the cluster kernel
    int qp;                 // row pitch of q; a subdomain's row starts at column start & ~3
    int small, tx, ty;      // 1: whole subdomain in one CTA of tx x ty threads (4 x 4 pixels each);
                            // 2: a cluster of ncl such CTAs, band = 4 ty rows each; 0: band kernel
    int ncl, band;          // otherwise: CTAs per subdomain (cluster size) and rows per CTA
    size_t smem;            // dynamic shared memory per CTA
    int stor;               // tvs_storage of p and q
    void* q;                // per-subdomain warm starts, [m2*m1][2][hmax][qp]
};
tvs_status schwarz2_check(int n2, int n1, const tvs_decomp& dd);
size_t schwarz2_extend(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch, int storage);
void schwarz2_carve(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch, int storage, Schwarz2State& st);
// Zero the warm starts q_m (Algorithm 3 starts every subdomain from 0).
cudaError_t schwarz2_reset(const Schwarz2State& st, cudaStream_t s);
// One image of a small-subdomain Schwarz step-2 launch.  A launch covers the
// subdomains of one image or of several images (sorted by `first`): CTA b
// runs subdomain b - first of the image with the largest first <= b.
struct TileImg {
    const void* p;    // p^n, 2 planes (storage of the launch)
    void* pnext;      // p^{n+1}, written on the exclusive part of the core
    const float* f2;
    void* q;          // [sub][2][hmax][qp], columns from start & ~3
    int pitch;
    long plane;
    int hmax, qp;
    Axis ay, ax;
    float ahat;       // damping of Algorithm 2
    int first;        // launch-wide index of the image's first subdomain
};
// n_outer outer iterations over several images, small subdomains only: per
// outer iteration one small-tile launch and one strip launch over all
// subdomains.  imgs_dev holds 2 * nimg descriptors in device memory: [0, nimg)
// for even outer iterations, [nimg, 2 nimg) for odd ones (p and pnext
// swapped).  tx, ty: thread block covering the largest subdomain.
cudaError_t schwarz2_iterate_multi(int storage, const TileImg* imgs_dev, int nimg, int nsub_total, int tx, int ty,
                                   int k, float t, int n_outer, uint32_t seed0, cudaStream_t s);
// The same n_outer outer iterations as one persistent cooperative launch (grid
// barriers between the tile and strip phases); bar: 2 device words (zeroed by
// the call), err: bit 1 set if a barrier wait gave up, seed_ctr: device
// counter of the 16-bit rounding seeds (advanced by n_outer).  Capturable in
// a CUDA graph.
cudaError_t schwarz2_persist_multi(int storage, const TileImg* imgs_dev, int nimg, int nsub_total, int tx, int ty,
                                   int k, float t, int n_outer, unsigned* bar, unsigned* err, uint32_t* seed_ctr,
                                   cudaStream_t s);
// Block shape of the small-subdomain kernel for subdomains up to hmax x wmax
// (0 if they need the cluster kernel); q row pitch and shared memory bytes.
int small_tile_shape(int hmax, int wmax, int* tx, int* ty, int* qp, size_t* smem);
// n_outer outer iterations of Algorithm 2: p^{n+1} from p^n = *cur, swapping
// *cur and *nxt after each iteration.  seed0: outer iterations done so far
// (seeds the stochastic rounding of 16-bit stores).
cudaError_t schwarz2_iterate(void** cur, void** nxt, const float* f2, int pitch, long plane, int n2, int n1,
                             const Schwarz2State& st, float t, int n_outer, uint32_t seed0, cudaStream_t s);

// schwarz1.cu -- Algorithm 2 with the localized Algorithm 5 for TFS on the extended grid
struct Schwarz1State {
    int m2, m1, s, k, ntiles;
    double alpha_hat;
    int hbox, wpad, pitch;   // per-subdomain storage covers A = (tilde Omega_{m,+})_+
    float *V, *U, *W;        // inner dual v (4 planes), u = vecdiv v (2), omega (2), per subdomain
    float* S;                // packed Poisson rows of A, per subdomain (rows of A x pitch)
    float* Q;                // P_K vecdiv p^n on the whole grid (2 planes)
    int2* ranges;            // rows of A per subdomain (device)
};
tvs_status schwarz1_check(int n2, int n1, const tvs_decomp& dd);
size_t schwarz1_extend(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch);
void schwarz1_carve(Carver& cv, int n2, int n1, const tvs_decomp& dd, int pitch, Schwarz1State& st);
cudaError_t schwarz1_reset(const Schwarz1State& st, int n2, int n1, cudaStream_t s);
cudaError_t schwarz1_iterate(float** cur, float** nxt, const float* f1, float* S_glob, int pitch, int n2, int n1,
                             const PoissonPlans& pp, const Schwarz1State& st, float t, int n_outer, unsigned* err,
                             cudaStream_t s);

}  // namespace tvs
