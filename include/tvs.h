/*
 * tvs.h -- C ABI of the GB300 TV-Stokes library (libtvs.so).
 *
 * The TV-Stokes model (Langer, Runft, Rahman, Tai, Wu, "Functional Analysis
 * and Parallel Domain Decomposition for the TV-Stokes Model") denoises an
 * image d0 in two steps:
 *   step 1 (tangent field smoothing, TFS): the dual problem eq. tfsdualdis on
 *          the extended grid, solved by Chambolle's semi-implicit iteration
 *          (Algorithm 1) with the divergence-free projection P_K
 *          (eq. formula:PKh; Delta^dagger of eq. form:DiscInvLapl evaluated as a
 *          DCT along x and one Neumann tridiagonal solve per x frequency along y,
 *          the same operator up to rounding);
 *   step 2 (image reconstruction IRV1): the dual problem eq. ir1dualdis on the
 *          image grid with the normal field xi of eq. defXi2:discrete.
 * Both may also run under the overlapping Schwarz decomposition of
 * Section 6 (Algorithm 2 with Algorithm 3, resp. Algorithms 4/5).
 *
 * Conventions shared by every entry point
 *  - All array arguments are CUDA DEVICE pointers owned by the caller.  The
 *    library never frees or keeps them after the call returns.
 *  - Arrays are dense, row-major float32: element (i, j) of a plane with
 *    `cols` columns is base[i * cols + j]; i = row = y, j = column = x.
 *    Vector fields are consecutive planes.
 *      image grid Omega        : n2 rows x n1 cols
 *      extended grid ~Omega    : (n2+1) rows x (n1+1) cols
 *      step-1 dual p           : 4 planes on ~Omega, order p1x, p1y, p2x, p2y
 *      step-2 dual p           : 2 planes on Omega,  order px, py
 *      tangent field tau       : 2 planes on ~Omega, order tau1, tau2
 *  - Scratch memory comes from the caller: `ws` is a device buffer of at
 *    least tvs_workspace_bytes(...) bytes, 256-byte aligned.  The calls do
 *    not allocate device memory for data.  Runs of unchecked iterations of
 *    tvs_step1, tvs_step2 (FP32 dual), tvs_schwarz (step 2, FP32 dual) and
 *    tvs_denoise are replayed from a cache of at most 32 instantiated CUDA
 *    graphs (driver-owned objects, keyed by every pointer and size they
 *    use); tvs_set_graphs(0) turns this off.
 *  - All device work is enqueued on `stream`.  Calls that fill a tvs_report
 *    synchronize `stream` before returning.
 *  - Argument errors return TVS_ERR_ARG before any work is enqueued.  CUDA
 *    errors return TVS_ERR_CUDA; tvs_last_error() names the failing call.
 *  - The grid spacing is h = 1 (Section 5.2).
 */
#ifndef TVS_H
#define TVS_H

#include <stddef.h>
#include <cuda_runtime.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    TVS_OK = 0,
    TVS_ERR_ARG = 1,            /* invalid argument, nothing enqueued          */
    TVS_ERR_WORKSPACE = 2,      /* ws NULL, misaligned or smaller than needed   */
    TVS_ERR_CUDA = 3,           /* a CUDA runtime call failed                   */
    TVS_ERR_TIMEOUT = 4,        /* a bounded device-side wait gave up           */
    TVS_ERR_NOT_CONVERGED = 5,  /* max_iter reached before rel_gap_tol; outputs valid */
    TVS_ERR_UNSUPPORTED = 6     /* size or option not supported by this build   */
} tvs_status;

/* Storage of the step-2 dual between updates (arithmetic is always FP32).
 * TVS_S16 is 16-bit fixed point on [-1, 1] (code / 32767): every component
 * of a feasible dual lies there (|p| <= 1), so it spends all 16 bits on that
 * range.  16-bit formats round stochastically on store (reproducibly). */
typedef enum { TVS_F32 = 0, TVS_BF16 = 1, TVS_F16 = 2, TVS_S16 = 3 } tvs_storage;

/* Iteration control of one dual solve (Sections 4.2 and 5.2). */
typedef struct {
    int    max_iter;     /* dual updates (global) or outer iterations (Schwarz), >= 0 */
    double t;            /* Chambolle step, 0 < t <= 1/8 (convergence theorem, Sec. 4.2) */
    double rel_gap_tol;  /* stop once gap/E <= tol (checked every check_every); 0 = never */
    int    check_every;  /* updates between gap checks; <= 0 means only at the end      */
    int    storage;      /* tvs_storage of the dual fields kept between updates:
                          * TVS_F32 everywhere; TVS_BF16, TVS_F16 or TVS_S16 for
                          * the global step 1 (tvs_step1, tvs_denoise it1) and
                          * for step 2 (tvs_step2, tvs_schwarz step 2,
                          * tvs_denoise it2, tvs_irv2, tvs_step2_w11), where p
                          * and the Schwarz warm starts q are stored in 16 bits
                          * and widened to FP32 for every update.  The caller's
                          * p stays FP32.  tvs_denoise keeps tau, when the
                          * caller passes none, as FP16 (it1 FP16 or fixed
                          * point) or BF16 (it1 BF16).  Schwarz step 1 and the
                          * engine's step 1 with a 16-bit storage:
                          * TVS_ERR_UNSUPPORTED; any other value: TVS_ERR_ARG. */
} tvs_iter;

/* Values at the returned dual iterate p (duality gap per Appendix A):
 *   dual_D   = ||Lambda p - f||^2                     (eq. opt_dual_discrete)
 *   primal_E = TV(u) + (beta/2)||u - g||^2, u recovered from p
 *   gap      = sum_k sum_ij (|grad u_k| + grad u_k . p_k) >= 0
 *   rel_gap  = gap / primal_E
 *   div_res_max = max |div tau| (step 1; 0 for step 2)
 *   max_p    = max over pixels and channels of |p_k| (<= 1 when feasible) */
typedef struct {
    int    iters;
    double dual_D, primal_E, gap, rel_gap, div_res_max, max_p;
} tvs_report;

/* Overlapping Schwarz decomposition (Section 6.1): m2 x m1 subdomains whose
 * cores split each axis evenly; neighbours share a strip of `overlap` pixels;
 * k_inner Chambolle updates per subdomain and outer iteration; alpha_hat <= 0
 * selects the colouring rule (1, 1/2 or 1/4). */
typedef struct {
    int    m2, m1;
    int    overlap;
    int    k_inner;
    double alpha_hat;
} tvs_decomp;

/* Library version (major*10000 + minor*100 + patch). */
int tvs_version(void);

/* Human-readable text of a status code (static storage). */
const char* tvs_status_string(tvs_status st);

/* Text of the last CUDA error recorded on the calling thread ("" if none). */
const char* tvs_last_error(void);

/* Bytes of scratch needed by a call.
 *   step = 1: tvs_step1 / tvs_schwarz(step=1); step = 2: tvs_step2 /
 *   tvs_schwarz(step=2) / tvs_step2_w11; step = 0: tvs_denoise (covers
 *   both); step = 3: tvs_project; step = 4: tvs_quality; step = 5: tvs_irv2.
 *   dd = NULL means the global iteration.  storage: the tvs_iter.storage of
 *   the call (for step 0: of it2; the size covers an FP32 step-1 dual and
 *   tau, which a 16-bit it1 also fits).  Returns 0 for invalid sizes or a
 *   storage the step does not support. */
size_t tvs_workspace_bytes(int step, int n2, int n1, const tvs_decomp* dd, int storage);

/* Divergence-free projection P_K = I - grad Delta^dagger div on a grid of
 * `rows` x `cols` points (eq. formula:PKh, Appendix B), with Delta^dagger of
 * eqs. form:DiscInvLapl, form:DiscInvLaplTild (DCT along x, tridiagonal solves
 * along y).
 *   in   : 2 planes rows x cols (x-part, y-part); out: same layout; in == out allowed.
 *   rows, cols >= 3.  ws: tvs_workspace_bytes(3, rows-1, cols-1, NULL, 0). */
tvs_status tvs_project(const float* in, float* out, int rows, int cols,
                       void* ws, size_t ws_bytes, cudaStream_t stream);

/* Divergence-free projection for callers that cannot allocate device memory.
 * The paper has no counterpart: this is tvs_project without a workspace, for
 * code that must not call cudaMalloc or take memory from a caching allocator
 * (for example a plug-in running inside another framework's allocator or a
 * host callback where allocation is forbidden).
 *   in, out : 2 planes rows x cols each, as in tvs_project (in == out allowed).
 *   Maximum : rows and cols at most 1025 each (images up to 1024 x 1024).  The
 *             scratch is one fixed 5 MiB device array inside the library, held
 *             on every GPU that loads the library until the process exits.
 *             Larger grids return TVS_ERR_UNSUPPORTED with a message in
 *             tvs_last_error().
 *   Every call looks up that array's device address on the current device
 *   (a host-side query; the first one on a device loads the library's device
 *   code there, so make that first call before any stream capture).  All
 *   calls share the one array, so calls whose GPU work overlaps (other
 *   streams, other host threads) race; serialize them on one stream.
 *   Allocates nothing. */
tvs_status tvs_project_noalloc(const float* in, float* out, int rows, int cols, cudaStream_t stream);

/* Step 1, TFS (Section 4.2, eq. tfsdualdis, Algorithm 1 with the projected
 * data term f1 = P_K tau0 / delta).
 *   d0   : n2 x n1 noisy image.            n2, n1 >= 2.   delta > 0.
 *   tau  : out, 2 planes on ~Omega, tau = P_K tau0 - delta P_K vecdiv p.
 *   p    : in/out warm start (4 planes on ~Omega) or NULL to start from 0.
 *   rep  : filled at the returned p (may be NULL). */
tvs_status tvs_step1(const float* d0, int n2, int n1, double delta, const tvs_iter* it,
                     float* tau, float* p, void* ws, size_t ws_bytes,
                     cudaStream_t stream, tvs_report* rep);

/* Step 2, IRV1 (Section 4.2, eq. ir1dualdis): xi = tau_perp/|tau_perp|_eps
 * from the first n2 rows and n1 columns of tau (eq. defXi2:discrete),
 * f2 = alpha d0 - div xi, Chambolle's iteration, d = (f2 - div p)/alpha.
 *   tau  : 2 planes on ~Omega (from tvs_step1).   alpha > 0, eps > 0.
 *   d    : out, n2 x n1.   p: in/out (2 planes on Omega) or NULL. */
tvs_status tvs_step2(const float* d0, const float* tau, int n2, int n1, double alpha, double eps,
                     const tvs_iter* it, float* d, float* p, void* ws, size_t ws_bytes,
                     cudaStream_t stream, tvs_report* rep);

/* W^{1,1} variant of step 2 (Remark IRPW11, eq. IRW11:dual): the dual
 *   min ||div p - alpha d0||^2 over |p - xi| <= 1,  d = d0 - div p / alpha,
 * with xi of eq. defXi2:discrete as in tvs_step2.  With q = p - xi this is the
 * IRV1 dual (eq. IRPXi_dual over |q| <= 1), so the same iteration runs on q
 * and the call returns p = q + xi; d equals tvs_step2's d.
 *   p  : out, 2 planes on Omega, the W^{1,1} dual.
 *   p0 : warm start of p (2 planes, may equal p) or NULL to start from p = xi.
 *   Other arguments and ws as for tvs_step2 (tvs_workspace_bytes(2, ...)). */
tvs_status tvs_step2_w11(const float* d0, const float* tau, int n2, int n1, double alpha, double eps,
                         const tvs_iter* it, float* d, float* p, const float* p0, void* ws, size_t ws_bytes,
                         cudaStream_t stream, tvs_report* rep);

/* Image reconstruction variant 2 (IRV2, Section 3.3: eqs. modifiedStep2,
 * modifiedStep2_2, modifiedStep2_2_dual; discrete eq. ir2dualdis).
 *   g   : potential of tau_perp = R_Omega(tau_2, -tau_1) on the image grid.
 *         The paper asks for (D^-_x g, D^-_y g) = tau_perp; those equations
 *         between neighbouring pixels are consistent exactly when div tau = 0
 *         inside the extended grid, while the zero-extension rows of D^- are
 *         not in general.  g is therefore the least-squares solution of the
 *         neighbour differences (g = Delta^dagger div v on the n2 x n1 grid,
 *         v the forward-edge field of tau_perp; DCT along x, tridiagonal
 *         solves along y), with mean zero.  Where an exact potential exists
 *         this is it; a constant in g does not change d.
 *   Then Chambolle's iteration for ||div p - alpha (d0 - g)||^2 over |p| <= 1
 *   (globally, or under the Schwarz decomposition dd when dd != NULL, as
 *   tvs_schwarz step 2), u = d0 - g - div p / alpha and d = u + g.
 *   tau  : 2 planes on ~Omega (from tvs_step1).   n2, n1 >= 3.   alpha > 0.
 *   d    : out, n2 x n1.   p: in/out (2 planes on Omega) or NULL.
 *   g_out: out, n2 x n1, or NULL.
 *   rep  : the ROF problem in u (beta = alpha, data d0 - g).
 *   ws   : tvs_workspace_bytes(5, n2, n1, dd, it->storage). */
tvs_status tvs_irv2(const float* d0, const float* tau, int n2, int n1, double alpha, const tvs_iter* it,
                    const tvs_decomp* dd, float* d, float* p, float* g_out, void* ws, size_t ws_bytes,
                    cudaStream_t stream, tvs_report* rep);

/* Both steps: d0 -> tau -> xi, f2 -> d.  Step 2 runs under the Schwarz
 * decomposition dd2 when dd2 != NULL, else globally.  tau may be NULL (kept
 * in ws).  rep[0] reports step 1, rep[1] step 2 (rep may be NULL). */
tvs_status tvs_denoise(const float* d0, int n2, int n1, double delta, double alpha, double eps,
                       const tvs_iter* it1, const tvs_iter* it2, const tvs_decomp* dd2,
                       float* tau, float* d, void* ws, size_t ws_bytes,
                       cudaStream_t stream, tvs_report* rep);

/* Overlapping Schwarz iteration (Algorithm 2) of one step.
 *   step = 2: inner Algorithm 3 for eq. ir1dualdis; `tau` and `eps` as in
 *             tvs_step2, `weight` = alpha, `out` = d (n2 x n1), p 2 planes.
 *   step = 1: inner Algorithm 5 for eq. tfsdualdis; `tau` unused, `weight` =
 *             delta, `out` = tau (2 planes on ~Omega), p 4 planes.
 *   outer->max_iter outer iterations; dd->k_inner inner updates each.
 *   p: in/out or NULL (zero start; the per-subdomain warm starts q_m always
 *   start at 0). */
tvs_status tvs_schwarz(int step, const float* d0, const float* tau, int n2, int n1,
                       double weight, double eps, const tvs_decomp* dd, const tvs_iter* outer,
                       float* out, float* p, void* ws, size_t ws_bytes,
                       cudaStream_t stream, tvs_report* rep);

/* Kernel timing, for measurement.  tvs_profile_enable(1) clears the
 * accumulators and starts bracketing every launch of the hot-path kernels
 * with CUDA events on the launching stream; (0) stops.  tvs_profile_read()
 * waits for the recorded events and writes one entry per kernel class
 * (launch count, summed device milliseconds) into out[0..cap); it returns the
 * number of entries written.  Not a numerical operation of the paper. */
typedef struct {
    char   name[32];
    int    launches;
    double ms;
} tvs_kernel_time;
int tvs_profile_enable(int on);
int tvs_profile_read(tvs_kernel_time* out, int cap);

/* Limit of the bounded device-side waits (the TMA tile and row loads of the
 * step-1 stencils and the step-2 update), in SM cycles; cycles <= 0 restores
 * the default of about two seconds.  A diagnostic, not an operation of the
 * paper: with a limit of a few cycles the first wait of a launch gives up
 * before its copy lands, the kernel records that in the call's error word,
 * waits (with the default limit) for its copies still in flight and
 * returns, and the call reports TVS_ERR_TIMEOUT.  Applies to launches
 * enqueued after it returns; call it while no work of the library runs. */
tvs_status tvs_set_wait_limit(long long cycles);

/* Graph replay of the iteration runs (see the conventions above): on (1, the
 * default) or off (0).  Returns the previous setting.  While profiling is
 * enabled every launch is made directly. */
int tvs_set_graphs(int on);

/* Quality of a reconstruction d against a ground truth gt (Section 5.3),
 * both n2 x n1 dense float with intensities in [0, 1] (largest value R = 1):
 *   psnr  = -10 log10(mean (d - gt)^2)          (+infinity if d == gt)
 *   mssim = single-window structural similarity over the whole image with
 *           population moments and c1 = (0.01 R)^2, c2 = (0.03 R)^2.
 * Sums are formed in FP32 per thread (compensated) and reduced in FP64.
 * ws: tvs_workspace_bytes(4, n2, n1, NULL, 0) bytes.  Synchronizes stream. */
tvs_status tvs_quality(const float* d, const float* gt, int n2, int n1, void* ws, size_t ws_bytes,
                       cudaStream_t stream, double* psnr, double* mssim);

/* ---------------------------------------------------------------------------
 * Batching and serving engine.  The paper has no counterpart (it denoises one
 * image at a time); this is the request loop around the two steps above.
 *   - Requests of any size (n2, n1 in [2, 8192]) are queued by
 *     tvs_engine_submit and admitted first-in first-out while their state
 *     (tvs_engine_request_bytes) fits the free part of the caller's device
 *     pool and fewer than max_live requests are resident.
 *   - Each tvs_engine_step advances every resident request: step 1 (TFS) by
 *     it1.check_every updates per request, step 2 (IRV1 under the Schwarz
 *     decomposition with cores of at most `tile` pixels, overlap `overlap`,
 *     k_inner inner updates) by it2.check_every outer iterations in launches
 *     shared by all resident step-2 requests.  It then synchronizes `stream`
 *     once, moves requests whose relative duality gap reached the step's
 *     rel_gap_tol (or whose max_iter passed; a chunk may pass it by less than
 *     check_every) to the next step, writes d of finished requests and
 *     releases their pool blocks.
 *   - All request state stays on the device between steps.  d0 and d are the
 *     caller's device buffers (n2 x n1 dense float); d0 must stay valid until
 *     the request is returned as done.
 *   - The pool is a caller-owned 256-byte-aligned device buffer; the engine
 *     allocates no device memory itself (pinned host memory and CUDA streams
 *     are created at tvs_engine_create).  Not thread-safe: one host thread
 *     drives an engine.
 * ------------------------------------------------------------------------- */
typedef struct tvs_engine tvs_engine;
typedef struct {
    double   delta, alpha, eps;   /* model weights, as for tvs_denoise                    */
    tvs_iter it1;                 /* step 1: t, rel_gap_tol, max_iter, check_every >= 1  */
    tvs_iter it2;                 /* step 2 (outer iterations), storage as for tvs_step2 */
    int      tile, overlap, k_inner;   /* step-2 subdomains; tile >= 16, 2 overlap < tile */
    int      max_live;            /* requests resident at once                           */
} tvs_engine_config;

/* Pool bytes one request of n2 x n1 needs (0: invalid size or config). */
size_t tvs_engine_request_bytes(const tvs_engine_config* cfg, int n2, int n1);
/* Pool bytes the engine keeps for itself (descriptor arrays). */
size_t tvs_engine_pool_overhead(const tvs_engine_config* cfg);
/* TVS_ERR_UNSUPPORTED: tile + overlap too large for one CTA per subdomain. */
tvs_status tvs_engine_create(const tvs_engine_config* cfg, void* pool, size_t pool_bytes,
                             cudaStream_t stream, tvs_engine** out);
/* Queue a request.  TVS_ERR_UNSUPPORTED if it could never fit the pool. */
tvs_status tvs_engine_submit(tvs_engine* e, long long id, const float* d0, int n2, int n1, float* d);
/* One engine step (see above).  Up to `cap` finished requests are returned
 * in done_ids (and, if done_reports is not NULL, their step-1 and step-2
 * reports at done_reports[2k], done_reports[2k+1]); more wait for the next
 * call. */
tvs_status tvs_engine_step(tvs_engine* e, long long* done_ids, tvs_report* done_reports, int cap,
                           int* n_done);
/* Requests queued, resident or finished but not yet returned. */
int tvs_engine_pending(const tvs_engine* e);
void tvs_engine_destroy(tvs_engine* e);

/* ---------------------------------------------------------------------------
 * Autotuner of the step-2 Schwarz decomposition.  The paper leaves the
 * subdomain size, the overlap and the number of inner updates free
 * (Sec. 6.1-6.3); this measures them.  Every candidate (core size tiles[a]:
 * m = ceil(n / tile) subdomains per axis, overlap overlaps[b], k = ks[c]) runs
 * tvs_schwarz step 2 on (d0, tau) from a zero dual until it->rel_gap_tol
 * (> 0, checked every it->check_every >= 1 outer iterations, at most
 * it->max_iter), timed with CUDA events on `stream` (the call synchronizes
 * it).  Candidates whose cores are narrower than the overlap are skipped.
 *   best    : out, {tile, overlap, k} of the fastest candidate that reached the
 *             tolerance; best_ms (may be NULL) its time in milliseconds.
 *   returns : TVS_ERR_NOT_CONVERGED if no candidate reached the tolerance.
 *   ws      : tvs_tune_workspace_bytes(...) bytes. */
size_t tvs_tune_workspace_bytes(int n2, int n1, const int* tiles, int ntiles, const int* overlaps,
                                int noverlaps, int storage);
tvs_status tvs_tune_schwarz2(const float* d0, const float* tau, int n2, int n1, double alpha, double eps,
                             const tvs_iter* it, const int* tiles, int ntiles, const int* overlaps,
                             int noverlaps, const int* ks, int nks, void* ws, size_t ws_bytes,
                             cudaStream_t stream, int* best, float* best_ms);

#ifdef __cplusplus
}
#endif
#endif /* TVS_H */
