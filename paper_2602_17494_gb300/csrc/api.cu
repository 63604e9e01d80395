// C ABI of libtvs (declared in include/tvs.h): argument checks, workspace
// layout and the host-side iteration drivers.  All arithmetic of the method
// runs in the kernels of dct.cu, tfs.cu, irv.cu and schwarz.cu.
#include "drivers.h"
#include "graphs.h"
#include "tma.cuh"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>

namespace tvs {

static thread_local std::string g_last_error;

void set_error(const char* what, cudaError_t e) {
    char buf[256];
    std::snprintf(buf, sizeof buf, "%s: %s", what, cudaGetErrorString(e));
    g_last_error = buf;
}

void set_error_text(const char* msg) { g_last_error = msg; }

size_t layout_step1(Carver& cv, int n2, int n1, Step1Layout& L, int storage) {
    L.R = n2 + 1;
    L.C = n1 + 1;
    L.P = round_up(L.C, kPitchAlign);
    L.plane = (long)L.R * L.P;
    L.st = storage;
    carve_poisson(cv, L.pp, L.R, L.C);
    // the dual in its storage format (4 planes, element pitch L.P)
    L.pa = reinterpret_cast<float*>(cv.take<char>(4 * (size_t)L.plane * storage_bytes(storage)));
    L.pb = reinterpret_cast<float*>(cv.take<char>(4 * (size_t)L.plane * storage_bytes(storage)));
    L.f1 = cv.take<float>(2 * (size_t)L.plane);
    L.S = cv.take<float>((size_t)L.plane);
    L.src = cv.take<float>((size_t)L.plane);
    carve_red(cv, L.red, tfs_blocks(L.R, L.C));
    return cv.used();
}


size_t layout_step2(Carver& cv, int n2, int n1, Step2Layout& L, int storage) {
    L.R = n2;
    L.C = n1;
    L.P = round_up(L.C, kPitchAlign);
    L.plane = (long)L.R * L.P;
    L.st = storage;
    L.pa = cv.take<char>(2 * (size_t)L.plane * storage_bytes(storage));
    L.pb = cv.take<char>(2 * (size_t)L.plane * storage_bytes(storage));
    L.f2 = cv.take<float>((size_t)L.plane);
    carve_red(cv, L.red, irv1_blocks(L.R, L.C));
    return cv.used();
}


// IRV2: Poisson plans on the n2 x n1 image grid and the potential g, then the
// step-2 state (and, with a decomposition, the Schwarz warm starts).
static size_t layout_irv2(Carver& cv, int n2, int n1, int storage, Step2Layout& L, PoissonPlans& pp, float** g) {
    carve_poisson(cv, pp, n2, n1);
    *g = cv.take<float>((size_t)n2 * round_up(n1, kPitchAlign));
    return layout_step2(cv, n2, n1, L, storage);
}

size_t layout_project(Carver& cv, int rows, int cols, ProjLayout& L) {
    L.P = round_up(cols, kPitchAlign);
    L.plane = (long)rows * L.P;
    carve_poisson(cv, L.pp, rows, cols);
    L.u = cv.take<float>(2 * (size_t)L.plane);
    L.S = cv.take<float>((size_t)L.plane);
    return cv.used();
}

// ---------------------------------------------------------------------------
// Checks
// ---------------------------------------------------------------------------
bool side_ok(int n) { return n >= 2 && n <= kMaxSide; }

// step 1 keeps its dual in FP32; step 2 also stores it as bf16 or fp16
tvs_status check_iter(const tvs_iter* it, bool narrow_ok) {
    if (!it) return TVS_ERR_ARG;
    if (it->max_iter < 0 || !(it->t > 0.0) || it->t > 0.125 || it->rel_gap_tol < 0.0) return TVS_ERR_ARG;
    if (storage_bytes(it->storage) == 0) return TVS_ERR_ARG;
    if (it->storage != TVS_F32 && !narrow_ok) return TVS_ERR_UNSUPPORTED;
    return TVS_OK;
}

tvs_status check_ws(void* ws, size_t ws_bytes, size_t need) {
    if (!ws || (reinterpret_cast<uintptr_t>(ws) & 255u) || ws_bytes < need) return TVS_ERR_WORKSPACE;
    return TVS_OK;
}

tvs_status read_result(const RedBuf& rb, int nblocks, cudaStream_t s, double out[kRedSlots]) {
    unsigned err = 0;
    TVS_CUDA(finalize_red(rb, nblocks, s));
    TVS_CUDA(cudaMemcpyAsync(out, rb.result, kRedSlots * sizeof(double), cudaMemcpyDeviceToHost, s));
    TVS_CUDA(cudaMemcpyAsync(&err, rb.err, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
    TVS_CUDA(cudaStreamSynchronize(s));
    if (err) {
        set_error_text("a bounded device-side wait gave up (TMA row load)");
        return TVS_ERR_TIMEOUT;
    }
    return TVS_OK;
}

void report_tfs(const double r[kRedSlots], double delta, int iters, tvs_report* rep) {
    const double tv = delta * r[0];
    const double e = tv + 0.5 * delta * r[3];
    const double gap = delta * r[1];
    rep->iters = iters;
    rep->dual_D = r[2];
    rep->primal_E = e;
    rep->gap = gap;
    rep->rel_gap = e > 0 ? gap / e : 0.0;
    rep->div_res_max = delta * r[5];
    rep->max_p = r[4];
}

void report_irv1(const double r[kRedSlots], double alpha, int iters, tvs_report* rep) {
    const double tv = r[0] / alpha;
    const double e = tv + r[3] / (2.0 * alpha);
    const double gap = r[1] / alpha;
    rep->iters = iters;
    rep->dual_D = r[2];
    rep->primal_E = e;
    rep->gap = gap;
    rep->rel_gap = e > 0 ? gap / e : 0.0;
    rep->div_res_max = 0.0;
    rep->max_p = r[4];
}

// Copy `planes` dense planes of rows x cols into / out of pitched storage.
cudaError_t to_pitched(float* dst, int dpitch, const float* src, int rows, int cols, int planes,
                             cudaStream_t s) {
    return cudaMemcpy2DAsync(dst, (size_t)dpitch * sizeof(float), src, (size_t)cols * sizeof(float),
                             (size_t)cols * sizeof(float), (size_t)rows * planes, cudaMemcpyDeviceToDevice, s);
}
cudaError_t from_pitched(float* dst, const float* src, int spitch, int rows, int cols, int planes,
                               cudaStream_t s) {
    return cudaMemcpy2DAsync(dst, (size_t)cols * sizeof(float), src, (size_t)spitch * sizeof(float),
                             (size_t)cols * sizeof(float), (size_t)rows * planes, cudaMemcpyDeviceToDevice, s);
}
// The caller's dense float dual into / out of the step-2 state (any storage).
cudaError_t p2_in(const Step2Layout& L, const float* src, cudaStream_t s) {
    if (L.st == TVS_F32) return to_pitched(static_cast<float*>(L.pa), L.P, src, L.R, L.C, 2, s);
    return convert_planes(L.pa, L.st, L.P, L.plane, src, TVS_F32, L.C, (long)L.R * L.C, L.R, L.C, 2, s);
}
cudaError_t p2_out(const Step2Layout& L, float* dst, const void* cur, cudaStream_t s) {
    if (L.st == TVS_F32) return from_pitched(dst, static_cast<const float*>(cur), L.P, L.R, L.C, 2, s);
    return convert_planes(dst, TVS_F32, L.C, (long)L.R * L.C, cur, L.st, L.P, L.plane, L.R, L.C, 2, s);
}
cudaError_t p2_zero(const Step2Layout& L, cudaStream_t s) {
    return cudaMemsetAsync(L.pa, 0, 2 * (size_t)L.plane * storage_bytes(L.st), s);
}

// ---------------------------------------------------------------------------
// Drivers
// ---------------------------------------------------------------------------
// f1 = P_K tau0 / delta into L.f1 (uses L.S as scratch).
tvs_status tfs_setup(const Step1Layout& L, const float* d0, int n2, int n1, double delta, cudaStream_t s) {
    TVS_CUDA(cudaMemsetAsync(L.red.err, 0, sizeof(unsigned), s));
    TVS_CUDA(build_poisson(L.pp, s));
    TVS_CUDA(launch_tau0(d0, n1, n2, n1, L.f1, L.P, L.plane, s));
    RowSrcArgs sa{L.f1, L.plane, L.P};
    TVS_CUDA(poisson_solve(L.S, L.R, L.C, L.P, L.pp, RowSource::DivField, sa, s));
    TVS_CUDA(launch_grad_sub(L.f1, L.P, L.plane, L.S, L.P, L.R, L.C, (float)(1.0 / delta), L.f1, L.P, L.plane, s));
    return TVS_OK;
}

// Runs of plain (unchecked) iterations between two convergence checks are
// replayed as cached CUDA graphs (graphs.h), at most kGraphRun iterations per
// graph and always an even number, so that p^n is back in the same buffer.
constexpr int kGraphRun = 64;

static int plain_run(bool check_loop, int n, const tvs_iter& it) {
    const int stop = check_loop ? std::min(it.max_iter, (n / it.check_every + 1) * it.check_every) : it.max_iter;
    return std::min(stop - n, kGraphRun) & ~1;
}

static void key_plan(GraphKey& k, const DctPlan& pl) {
    k.add((uint64_t)pl.L).add((uint64_t)pl.M).ptr(pl.chirp).ptr(pl.rot).ptr(pl.post).ptr(pl.tw).ptr(pl.bhat).ptr(pl.sig2);
}

// `count` plain TFS iterations from cur on stream st (cur and nxt alternate; FP32 dual).
// One update of the global TFS loop.  On entry L.src holds div(vecdiv cur);
// phi = Delta^dagger of it goes to L.S, then the fused step writes nxt and
// div(vecdiv nxt) into L.src, so the invariant holds for the next update.
static cudaError_t tfs_one(const Step1Layout& L, const float* cur, float* nxt, uint32_t seed, float t, bool check,
                           cudaStream_t st) {
    RowSrcArgs sa{L.src, 0, L.P};
    cudaError_t e = poisson_solve(L.S, L.R, L.C, L.P, L.pp, RowSource::Plain, sa, st);
    if (e != cudaSuccess) return e;
    return launch_tfs_step_st(cur, nxt, L.st, seed, L.S, L.f1, L.src, L.R, L.C, L.P, L.plane, t, check,
                              L.red.partial, L.red.err, st);
}

static cudaError_t tfs_iters(const Step1Layout& L, float* cur, float* nxt, int count, float t, float fd,
                             cudaStream_t st) {
    (void)fd;
    for (int i = 0; i < count; ++i) {
        const cudaError_t e = tfs_one(L, cur, nxt, 0u, t, false, st);
        if (e != cudaSuccess) return e;
        std::swap(cur, nxt);
    }
    return cudaSuccess;
}

// The caller's dense FP32 step-1 dual into / out of the state (any storage).
static cudaError_t p1_in(const Step1Layout& L, const float* src, cudaStream_t s) {
    if (L.st == TVS_F32) return to_pitched(L.pa, L.P, src, L.R, L.C, 4, s);
    return convert_planes(L.pa, L.st, L.P, L.plane, src, TVS_F32, L.C, (long)L.R * L.C, L.R, L.C, 4, s);
}
static cudaError_t p1_out(const Step1Layout& L, float* dst, const float* cur, cudaStream_t s) {
    if (L.st == TVS_F32) return from_pitched(dst, cur, L.P, L.R, L.C, 4, s);
    return convert_planes(dst, TVS_F32, L.C, (long)L.R * L.C, cur, L.st, L.P, L.plane, L.R, L.C, 4, s);
}

// tau (2 planes on the extended grid, pitch tau_pitch) is written as
// tau_storage: TVS_F32, or TVS_F16 / TVS_BF16 for tau kept in the workspace
// with a 16-bit dual.
static tvs_status run_tfs(const Step1Layout& L, const float* d0, int n2, int n1, double delta, const tvs_iter& it,
                          void* tau, int tau_storage, int tau_pitch, long tau_plane, float* p_user, cudaStream_t s,
                          tvs_report* rep) {
    tvs_status st = tfs_setup(L, d0, n2, n1, delta, s);
    if (st != TVS_OK) return st;
    if (p_user) TVS_CUDA(p1_in(L, p_user, s));
    else TVS_CUDA(cudaMemsetAsync(L.pa, 0, 4 * (size_t)L.plane * storage_bytes(L.st), s));
    float* cur = L.pa;
    float* nxt = L.pb;
    const int nb = tfs_blocks(L.R, L.C);
    const bool check_loop = it.rel_gap_tol > 0.0 && it.check_every > 0;
    const float t = (float)it.t, fd = (float)delta;
    int n = 0;
    bool converged = !check_loop;
    double r[kRedSlots];
    // the loop keeps L.src = div(vecdiv cur) (tfs_one)
    TVS_CUDA(launch_div_vecdiv_st(cur, L.st, L.R, L.C, L.P, L.plane, L.src, L.red.err, s));
    while (n < it.max_iter) {
        const bool ck = check_loop && n > 0 && (n % it.check_every) == 0;
        // FP32 dual only: 16-bit stores draw their rounding bits from the update
        // number, which a replayed graph would repeat
        const int run = (ck || L.st != TVS_F32) ? 0 : plain_run(check_loop, n, it);
        if (run >= 4) {
            GraphKey key;
            key.add(1).add((uint64_t)run).ptr(cur).ptr(nxt).ptr(L.S).ptr(L.src).ptr(L.f1).add((uint64_t)L.R).add((uint64_t)L.C)
                .add((uint64_t)L.P).add((uint64_t)L.plane).num(t).num(fd).ptr(L.red.partial).ptr(L.red.err);
            key_plan(key, L.pp.row);
            key.add((uint64_t)L.pp.rows).ptr(L.pp.tri);
            TVS_CUDA(graph_run(key, s, [&](cudaStream_t st) { return tfs_iters(L, cur, nxt, run, t, fd, st); }));
            n += run;
            continue;
        }
        TVS_CUDA(tfs_one(L, cur, nxt, (uint32_t)n + 1u, t, ck, s));
        std::swap(cur, nxt);
        ++n;
        if (ck) {
            st = read_result(L.red, nb, s, r);
            if (st != TVS_OK) return st;
            tvs_report tmp;
            report_tfs(r, delta, n - 1, &tmp);
            if (tmp.rel_gap <= it.rel_gap_tol) {
                converged = true;
                break;
            }
        }
    }
    {
        RowSrcArgs sa{L.src, 0, L.P};
        TVS_CUDA(poisson_solve(L.S, L.R, L.C, L.P, L.pp, RowSource::Plain, sa, s));
    }
    TVS_CUDA(launch_tfs_update_st(cur, nullptr, L.st, 0u, L.S, L.f1, L.R, L.C, L.P, L.plane, t, fd, true, false, tau,
                                  tau_storage, tau_pitch, tau_plane, L.red.partial, L.red.err, s));
    st = read_result(L.red, nb, s, r);
    if (st != TVS_OK) return st;
    tvs_report fin;
    report_tfs(r, delta, n, &fin);
    if (rep) *rep = fin;
    if (p_user) TVS_CUDA(p1_out(L, p_user, cur, s));
    if (check_loop && !converged && fin.rel_gap > it.rel_gap_tol) return TVS_ERR_NOT_CONVERGED;
    return TVS_OK;
}

// Chambolle's iteration for ||div p - f2||^2 over |p| <= 1 with f2 already in
// L.f2 (IRV1: alpha d0 - div xi; IRV2: alpha (d0 - g)); d = (f2 - div p) / alpha.
static tvs_status run_irv1_loop(const Step2Layout& L, int n1, double alpha, const tvs_iter& it, float* d,
                                float* p_user, cudaStream_t s, tvs_report* rep) {
    if (p_user) TVS_CUDA(p2_in(L, p_user, s));
    else TVS_CUDA(p2_zero(L, s));
    TVS_CUDA(cudaMemsetAsync(L.red.err, 0, sizeof(unsigned), s));
    void* cur = L.pa;
    void* nxt = L.pb;
    const int nb = irv1_blocks(L.R, L.C);
    const bool check_loop = it.rel_gap_tol > 0.0 && it.check_every > 0;
    const float t = (float)it.t, fa = (float)alpha;
    int n = 0;
    bool converged = !check_loop;
    double r[kRedSlots];
    tvs_status st;
    while (n < it.max_iter) {
        const bool ck = check_loop && n > 0 && (n % it.check_every) == 0;
        // FP32 dual only: 16-bit stores draw their rounding bits from the
        // iteration number, which a replayed graph would repeat
        const int run = (ck || L.st != TVS_F32) ? 0 : plain_run(check_loop, n, it);
        if (run >= 4) {
            GraphKey key;
            key.add(2).add((uint64_t)run).ptr(cur).ptr(nxt).ptr(L.f2).add((uint64_t)L.R).add((uint64_t)L.C)
                .add((uint64_t)L.P).add((uint64_t)L.plane).num(t).num(fa).ptr(L.red.partial).ptr(L.red.err);
            TVS_CUDA(graph_run(key, s, [&](cudaStream_t st) {
                void* a = cur;
                void* b = nxt;
                for (int i = 0; i < run; ++i) {
                    const cudaError_t e = launch_irv1_update(a, b, L.f2, L.R, L.C, L.P, L.plane, t, fa, false, true,
                                                             nullptr, 0, L.red.partial, L.st, 0u, L.red.err, st);
                    if (e != cudaSuccess) return e;
                    std::swap(a, b);
                }
                return cudaSuccess;
            }));
            n += run;
            continue;
        }
        TVS_CUDA(launch_irv1_update(cur, nxt, L.f2, L.R, L.C, L.P, L.plane, t, fa, ck, true, nullptr, 0,
                                    L.red.partial, L.st, (uint32_t)n + 1u, L.red.err, s));
        std::swap(cur, nxt);
        ++n;
        if (ck) {
            st = read_result(L.red, nb, s, r);
            if (st != TVS_OK) return st;
            tvs_report tmp;
            report_irv1(r, alpha, n - 1, &tmp);
            if (tmp.rel_gap <= it.rel_gap_tol) {
                converged = true;
                break;
            }
        }
    }
    TVS_CUDA(launch_irv1_update(cur, nullptr, L.f2, L.R, L.C, L.P, L.plane, t, fa, true, false, d, n1,
                                L.red.partial, L.st, 0u, L.red.err, s));
    st = read_result(L.red, nb, s, r);
    if (st != TVS_OK) return st;
    tvs_report fin;
    report_irv1(r, alpha, n, &fin);
    if (rep) *rep = fin;
    if (p_user) TVS_CUDA(p2_out(L, p_user, cur, s));
    if (check_loop && !converged && fin.rel_gap > it.rel_gap_tol) return TVS_ERR_NOT_CONVERGED;
    return TVS_OK;
}

static tvs_status run_irv1(const Step2Layout& L, const float* d0, const void* tau, int n2, int n1, double alpha,
                           double eps, const tvs_iter& it, float* d, float* p_user, cudaStream_t s,
                           tvs_report* rep, int tau_storage = TVS_F32) {
    const int R = n2 + 1, C = n1 + 1;
    TVS_CUDA(launch_xi_f2_st(d0, n1, tau, tau_storage, (long)R * C, C, n2, n1, (float)alpha, (float)eps, L.f2, L.P,
                             s));
    return run_irv1_loop(L, n1, alpha, it, d, p_user, s, rep);
}

tvs_status run_schwarz2(const Step2Layout& L, Schwarz2State& S2, int n2, int n1, double alpha,
                               const tvs_iter& it, float* d, float* p_user, cudaStream_t s, tvs_report* rep) {
    if (p_user) TVS_CUDA(p2_in(L, p_user, s));
    else TVS_CUDA(p2_zero(L, s));
    TVS_CUDA(cudaMemsetAsync(L.red.err, 0, sizeof(unsigned), s));
    TVS_CUDA(schwarz2_reset(S2, s));
    void* cur = L.pa;
    void* nxt = L.pb;
    const int nb = irv1_blocks(L.R, L.C);
    const bool check_loop = it.rel_gap_tol > 0.0 && it.check_every > 0;
    const float t = (float)it.t, fa = (float)alpha;
    const int chunk = check_loop ? it.check_every : (it.max_iter > 0 ? it.max_iter : 1);
    int n = 0;
    bool converged = !check_loop;
    double r[kRedSlots];
    tvs_status st;
    while (n < it.max_iter) {
        const int step = chunk < it.max_iter - n ? chunk : it.max_iter - n;
        if (S2.stor == TVS_F32 && step >= 2) {
            // even runs of outer iterations as cached graphs (FP32 dual: the
            // rounding seed of 16-bit stores would repeat in a replay)
            const int run = std::min(step, kGraphRun) & ~1;
            GraphKey key;
            key.add(3).add((uint64_t)run).ptr(cur).ptr(nxt).ptr(L.f2).add((uint64_t)L.P).add((uint64_t)L.plane)
                .add((uint64_t)n2).add((uint64_t)n1).num(t).ptr(S2.q).add((uint64_t)S2.m2).add((uint64_t)S2.m1)
                .add((uint64_t)S2.s).add((uint64_t)S2.k).num(S2.alpha_hat).add((uint64_t)S2.small)
                .add((uint64_t)S2.tx).add((uint64_t)S2.ty).add((uint64_t)S2.ncl).add((uint64_t)S2.band)
                .add((uint64_t)S2.smem).add((uint64_t)S2.hmax).add((uint64_t)S2.wpad).add((uint64_t)S2.qp);
            TVS_CUDA(graph_run(key, s, [&](cudaStream_t st) {
                void* a = cur;
                void* b = nxt;
                return schwarz2_iterate(&a, &b, L.f2, L.P, L.plane, n2, n1, S2, t, run, 0u, st);
            }));
            if (step > run)
                TVS_CUDA(schwarz2_iterate(&cur, &nxt, L.f2, L.P, L.plane, n2, n1, S2, t, step - run, (uint32_t)(n + run), s));
        } else {
            TVS_CUDA(schwarz2_iterate(&cur, &nxt, L.f2, L.P, L.plane, n2, n1, S2, t, step, (uint32_t)n, s));
        }
        n += step;
        if (check_loop && n < it.max_iter) {
            TVS_CUDA(launch_irv1_update(cur, nullptr, L.f2, L.R, L.C, L.P, L.plane, t, fa, true, false, nullptr, 0,
                                        L.red.partial, L.st, 0u, L.red.err, s));
            st = read_result(L.red, nb, s, r);
            if (st != TVS_OK) return st;
            tvs_report tmp;
            report_irv1(r, alpha, n, &tmp);
            if (tmp.rel_gap <= it.rel_gap_tol) {
                converged = true;
                break;
            }
        }
    }
    TVS_CUDA(launch_irv1_update(cur, nullptr, L.f2, L.R, L.C, L.P, L.plane, t, fa, true, false, d, n1,
                                L.red.partial, L.st, 0u, L.red.err, s));
    st = read_result(L.red, nb, s, r);
    if (st != TVS_OK) return st;
    tvs_report fin;
    report_irv1(r, alpha, n, &fin);
    if (rep) *rep = fin;
    if (p_user) TVS_CUDA(p2_out(L, p_user, cur, s));
    if (check_loop && !converged && fin.rel_gap > it.rel_gap_tol) return TVS_ERR_NOT_CONVERGED;
    return TVS_OK;
}

static tvs_status run_schwarz1(const Step1Layout& L, Schwarz1State& S1, const float* d0, int n2, int n1,
                               double delta, const tvs_iter& it, float* tau, float* p_user, cudaStream_t s,
                               tvs_report* rep) {
    tvs_status st = tfs_setup(L, d0, n2, n1, delta, s);
    if (st != TVS_OK) return st;
    if (p_user) TVS_CUDA(to_pitched(L.pa, L.P, p_user, L.R, L.C, 4, s));
    else TVS_CUDA(cudaMemsetAsync(L.pa, 0, 4 * (size_t)L.plane * sizeof(float), s));
    TVS_CUDA(schwarz1_reset(S1, n2, n1, s));
    float* cur = L.pa;
    float* nxt = L.pb;
    const int nb = tfs_blocks(L.R, L.C);
    const bool check_loop = it.rel_gap_tol > 0.0 && it.check_every > 0;
    const float t = (float)it.t, fd = (float)delta;
    const int chunk = check_loop ? it.check_every : (it.max_iter > 0 ? it.max_iter : 1);
    int n = 0;
    bool converged = !check_loop;
    double r[kRedSlots];
    while (n < it.max_iter) {
        const int step = chunk < it.max_iter - n ? chunk : it.max_iter - n;
        TVS_CUDA(schwarz1_iterate(&cur, &nxt, L.f1, L.S, L.P, n2, n1, L.pp, S1, t, step, L.red.err, s));
        n += step;
        if (check_loop && n < it.max_iter) {
            TVS_CUDA(tfs_phi(cur, L.S, L.R, L.C, L.P, L.plane, L.pp, L.red.err, s));
            TVS_CUDA(launch_tfs_update(cur, nullptr, L.S, L.f1, L.R, L.C, L.P, L.plane, t, fd, true, false, nullptr,
                                       0, 0, L.red.partial, L.red.err, s));
            st = read_result(L.red, nb, s, r);
            if (st != TVS_OK) return st;
            tvs_report tmp;
            report_tfs(r, delta, n, &tmp);
            if (tmp.rel_gap <= it.rel_gap_tol) {
                converged = true;
                break;
            }
        }
    }
    TVS_CUDA(tfs_phi(cur, L.S, L.R, L.C, L.P, L.plane, L.pp, L.red.err, s));
    TVS_CUDA(launch_tfs_update(cur, nullptr, L.S, L.f1, L.R, L.C, L.P, L.plane, t, fd, true, false, tau, n1 + 1,
                               (long)(n2 + 1) * (n1 + 1), L.red.partial, L.red.err, s));
    st = read_result(L.red, nb, s, r);
    if (st != TVS_OK) return st;
    tvs_report fin;
    report_tfs(r, delta, n, &fin);
    if (rep) *rep = fin;
    if (p_user) TVS_CUDA(from_pitched(p_user, cur, L.P, L.R, L.C, 4, s));
    if (check_loop && !converged && fin.rel_gap > it.rel_gap_tol) return TVS_ERR_NOT_CONVERGED;
    return TVS_OK;
}

}  // namespace tvs

using namespace tvs;

extern "C" {

int tvs_version(void) { return 100; }

const char* tvs_status_string(tvs_status st) {
    switch (st) {
        case TVS_OK: return "ok";
        case TVS_ERR_ARG: return "invalid argument";
        case TVS_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
        case TVS_ERR_CUDA: return "CUDA error";
        case TVS_ERR_TIMEOUT: return "device-side wait timed out";
        case TVS_ERR_NOT_CONVERGED: return "iteration limit reached before the gap tolerance";
        case TVS_ERR_UNSUPPORTED: return "unsupported size or option";
    }
    return "unknown status";
}

const char* tvs_last_error(void) { return g_last_error.c_str(); }

tvs_status tvs_set_wait_limit(long long cycles) {
    const long long v = cycles > 0 && cycles < kWaitCycles ? cycles : kWaitCycles;
    TVS_CUDA(tfs_set_wait_limit(v));
    TVS_CUDA(irv_set_wait_limit(v));
    return TVS_OK;
}

size_t tvs_workspace_bytes(int step, int n2, int n1, const tvs_decomp* dd, int storage) {
    if (storage_bytes(storage) == 0) return 0;
    if (storage != TVS_F32 && (step == 3 || (step == 1 && dd))) return 0;   // Schwarz step 1 keeps an FP32 dual
    Carver cv(nullptr);
    if (step == 3) {
        if (n2 < 2 || n1 < 2 || n2 + 1 > kMaxSide + 1 || n1 + 1 > kMaxSide + 1) return 0;
        ProjLayout L;
        return layout_project(cv, n2 + 1, n1 + 1, L);
    }
    if (!side_ok(n2) || !side_ok(n1)) return 0;
    if (step == 1) {
        Step1Layout L;
        size_t b = layout_step1(cv, n2, n1, L, storage);
        if (dd) {
            if (schwarz1_check(n2, n1, *dd) != TVS_OK) return 0;
            b = schwarz1_extend(cv, n2, n1, *dd, L.P);
        }
        return b;
    }
    if (step == 2) {
        Step2Layout L;
        size_t b = layout_step2(cv, n2, n1, L, storage);
        if (dd) b = schwarz2_extend(cv, n2, n1, *dd, L.P, storage);
        return b;
    }
    if (step == 4) {
        RedBuf rb;
        return quality_layout(cv, rb);
    }
    if (step == 5) {
        if (n2 < 3 || n1 < 3) return 0;
        Step2Layout L;
        PoissonPlans pp;
        float* g;
        size_t b = layout_irv2(cv, n2, n1, storage, L, pp, &g);
        if (dd) b = schwarz2_extend(cv, n2, n1, *dd, L.P, storage);
        return b;
    }
    if (step == 0) {
        Step1Layout L1;
        layout_step1(cv, n2, n1, L1);
        cv.take<float>(2 * (size_t)(n2 + 1) * (n1 + 1));
        Step2Layout L2;
        size_t b = layout_step2(cv, n2, n1, L2, storage);
        if (dd) b = schwarz2_extend(cv, n2, n1, *dd, L2.P, storage);
        return b;
    }
    return 0;
}

tvs_status tvs_project(const float* in, float* out, int rows, int cols, void* ws, size_t ws_bytes,
                       cudaStream_t stream) {
    if (!in || !out || rows < 3 || cols < 3 || rows > kMaxSide + 1 || cols > kMaxSide + 1) return TVS_ERR_ARG;
    Carver cv0(nullptr);
    ProjLayout L0;
    tvs_status st = check_ws(ws, ws_bytes, layout_project(cv0, rows, cols, L0));
    if (st != TVS_OK) return st;
    Carver cv(ws);
    ProjLayout L;
    layout_project(cv, rows, cols, L);
    TVS_CUDA(build_poisson(L.pp, stream));
    TVS_CUDA(to_pitched(L.u, L.P, in, rows, cols, 2, stream));
    RowSrcArgs sa{L.u, L.plane, L.P};
    TVS_CUDA(poisson_solve(L.S, rows, cols, L.P, L.pp, RowSource::DivField, sa, stream));
    TVS_CUDA(launch_grad_sub(L.u, L.P, L.plane, L.S, L.P, rows, cols, 1.0f, out, cols, (long)rows * cols, stream));
    return TVS_OK;
}

tvs_status tvs_step1(const float* d0, int n2, int n1, double delta, const tvs_iter* it, float* tau, float* p,
                     void* ws, size_t ws_bytes, cudaStream_t stream, tvs_report* rep) {
    if (!d0 || !tau || !side_ok(n2) || !side_ok(n1) || !(delta > 0.0)) return TVS_ERR_ARG;
    tvs_status st = check_iter(it, true);
    if (st != TVS_OK) return st;
    Carver cv0(nullptr);
    Step1Layout L;
    st = check_ws(ws, ws_bytes, layout_step1(cv0, n2, n1, L, it->storage));
    if (st != TVS_OK) return st;
    Carver cv(ws);
    layout_step1(cv, n2, n1, L, it->storage);
    return run_tfs(L, d0, n2, n1, delta, *it, tau, TVS_F32, n1 + 1, (long)(n2 + 1) * (n1 + 1), p, stream, rep);
}

tvs_status tvs_step2(const float* d0, const float* tau, int n2, int n1, double alpha, double eps,
                     const tvs_iter* it, float* d, float* p, void* ws, size_t ws_bytes, cudaStream_t stream,
                     tvs_report* rep) {
    if (!d0 || !tau || !d || !side_ok(n2) || !side_ok(n1) || !(alpha > 0.0) || !(eps > 0.0)) return TVS_ERR_ARG;
    tvs_status st = check_iter(it, true);
    if (st != TVS_OK) return st;
    Carver cv0(nullptr);
    Step2Layout L;
    st = check_ws(ws, ws_bytes, layout_step2(cv0, n2, n1, L, it->storage));
    if (st != TVS_OK) return st;
    Carver cv(ws);
    layout_step2(cv, n2, n1, L, it->storage);
    return run_irv1(L, d0, tau, n2, n1, alpha, eps, *it, d, p, stream, rep);
}

tvs_status tvs_schwarz(int step, const float* d0, const float* tau, int n2, int n1, double weight, double eps,
                       const tvs_decomp* dd, const tvs_iter* outer, float* out, float* p, void* ws,
                       size_t ws_bytes, cudaStream_t stream, tvs_report* rep) {
    if (step == 1) {
        if (!dd || !d0 || !out || !side_ok(n2) || !side_ok(n1) || !(weight > 0.0)) return TVS_ERR_ARG;
        tvs_status st = check_iter(outer, false);
        if (st != TVS_OK) return st;
        st = schwarz1_check(n2, n1, *dd);
        if (st != TVS_OK) return st;
        st = check_ws(ws, ws_bytes, tvs_workspace_bytes(1, n2, n1, dd, TVS_F32));
        if (st != TVS_OK) return st;
        Carver cv(ws);
        Step1Layout L;
        layout_step1(cv, n2, n1, L);
        Schwarz1State S1;
        schwarz1_carve(cv, n2, n1, *dd, L.P, S1);
        return run_schwarz1(L, S1, d0, n2, n1, weight, *outer, out, p, stream, rep);
    }
    if (step != 2 || !dd || !d0 || !tau || !out || !side_ok(n2) || !side_ok(n1) || !(weight > 0.0) ||
        !(eps > 0.0))
        return TVS_ERR_ARG;
    tvs_status st = check_iter(outer, true);
    if (st != TVS_OK) return st;
    st = schwarz2_check(n2, n1, *dd);
    if (st != TVS_OK) return st;
    Carver cv0(nullptr);
    Step2Layout L;
    layout_step2(cv0, n2, n1, L, outer->storage);
    st = check_ws(ws, ws_bytes, schwarz2_extend(cv0, n2, n1, *dd, L.P, outer->storage));
    if (st != TVS_OK) return st;
    Carver cv(ws);
    layout_step2(cv, n2, n1, L, outer->storage);
    Schwarz2State S2;
    schwarz2_carve(cv, n2, n1, *dd, L.P, outer->storage, S2);
    const int R = n2 + 1, C = n1 + 1;
    TVS_CUDA(launch_xi_f2(d0, n1, tau, (long)R * C, C, n2, n1, (float)weight, (float)eps, L.f2, L.P, stream));
    return run_schwarz2(L, S2, n2, n1, weight, *outer, out, p, stream, rep);
}

tvs_status tvs_step2_w11(const float* d0, const float* tau, int n2, int n1, double alpha, double eps,
                         const tvs_iter* it, float* d, float* p, const float* p0, void* ws, size_t ws_bytes,
                         cudaStream_t stream, tvs_report* rep) {
    if (!d0 || !tau || !d || !p || !side_ok(n2) || !side_ok(n1) || !(alpha > 0.0) || !(eps > 0.0))
        return TVS_ERR_ARG;
    tvs_status st = check_iter(it, true);
    if (st != TVS_OK) return st;
    Carver cv0(nullptr);
    Step2Layout L;
    st = check_ws(ws, ws_bytes, layout_step2(cv0, n2, n1, L, it->storage));
    if (st != TVS_OK) return st;
    Carver cv(ws);
    layout_step2(cv, n2, n1, L, it->storage);
    const long tplane = (long)(n2 + 1) * (n1 + 1);
    const size_t pbytes = 2 * (size_t)n2 * n1 * sizeof(float);
    // q = p - xi is the IRV1 dual (eq. IRPXi_dual); start from q0 = p0 - xi, or 0
    if (p0) {
        if (p0 != p) TVS_CUDA(cudaMemcpyAsync(p, p0, pbytes, cudaMemcpyDeviceToDevice, stream));
        TVS_CUDA(launch_shift_xi(p, n2, n1, tau, tplane, n1 + 1, (float)eps, -1.0f, stream));
    } else {
        TVS_CUDA(cudaMemsetAsync(p, 0, pbytes, stream));
    }
    st = run_irv1(L, d0, tau, n2, n1, alpha, eps, *it, d, p, stream, rep);
    if (st != TVS_OK && st != TVS_ERR_NOT_CONVERGED) return st;
    TVS_CUDA(launch_shift_xi(p, n2, n1, tau, tplane, n1 + 1, (float)eps, 1.0f, stream));
    return st;
}

tvs_status tvs_irv2(const float* d0, const float* tau, int n2, int n1, double alpha, const tvs_iter* it,
                    const tvs_decomp* dd, float* d, float* p, float* g_out, void* ws, size_t ws_bytes,
                    cudaStream_t stream, tvs_report* rep) {
    if (!d0 || !tau || !d || n2 < 3 || n1 < 3 || !side_ok(n2) || !side_ok(n1) || !(alpha > 0.0)) return TVS_ERR_ARG;
    tvs_status st = check_iter(it, true);
    if (st != TVS_OK) return st;
    if (dd) {
        st = schwarz2_check(n2, n1, *dd);
        if (st != TVS_OK) return st;
    }
    st = check_ws(ws, ws_bytes, tvs_workspace_bytes(5, n2, n1, dd, it->storage));
    if (st != TVS_OK) return st;
    Carver cv(ws);
    Step2Layout L;
    PoissonPlans pp;
    float* g = nullptr;
    layout_irv2(cv, n2, n1, it->storage, L, pp, &g);
    // g = Delta^dagger div v on the image grid, then f = alpha (d0 - g)
    TVS_CUDA(build_poisson(pp, stream));
    TVS_CUDA(launch_potential_src(tau, (long)(n2 + 1) * (n1 + 1), n1 + 1, n2, n1, g, L.P, stream));
    RowSrcArgs sa{g, 0, L.P};
    TVS_CUDA(poisson_solve(g, n2, n1, L.P, pp, RowSource::Plain, sa, stream));
    TVS_CUDA(launch_irv2_f(d0, n1, g, L.P, n2, n1, (float)alpha, L.f2, L.P, stream));
    TVS_CUDA(cudaMemsetAsync(L.red.err, 0, sizeof(unsigned), stream));
    if (dd) {
        Schwarz2State S2;
        schwarz2_carve(cv, n2, n1, *dd, L.P, it->storage, S2);
        st = run_schwarz2(L, S2, n2, n1, alpha, *it, d, p, stream, rep);
    } else {
        st = run_irv1_loop(L, n1, alpha, *it, d, p, stream, rep);
    }
    if (st != TVS_OK && st != TVS_ERR_NOT_CONVERGED) return st;
    // d = u + g (eq. modifiedStep2_2 solved for u = d - g)
    TVS_CUDA(launch_add_plane(d, n1, g, L.P, n2, n1, stream));
    if (g_out) TVS_CUDA(from_pitched(g_out, g, L.P, n2, n1, 1, stream));
    return st;
}

tvs_status tvs_denoise(const float* d0, int n2, int n1, double delta, double alpha, double eps, const tvs_iter* it1,
                       const tvs_iter* it2, const tvs_decomp* dd2, float* tau, float* d, void* ws, size_t ws_bytes,
                       cudaStream_t stream, tvs_report* rep) {
    if (!d0 || !d || !side_ok(n2) || !side_ok(n1) || !(delta > 0.0) || !(alpha > 0.0) || !(eps > 0.0))
        return TVS_ERR_ARG;
    tvs_status st = check_iter(it1, true);
    if (st != TVS_OK) return st;
    st = check_iter(it2, true);
    if (st != TVS_OK) return st;
    if (dd2) {
        st = schwarz2_check(n2, n1, *dd2);
        if (st != TVS_OK) return st;
    }
    const size_t need = tvs_workspace_bytes(0, n2, n1, dd2, it2->storage);
    st = check_ws(ws, ws_bytes, need);
    if (st != TVS_OK) return st;
    // the workspace is laid out for an FP32 step-1 dual and tau (tvs_workspace_bytes
    // step 0); a 16-bit step-1 dual uses the front part of its slots
    Carver cv(ws);
    Step1Layout L1;
    layout_step1(cv, n2, n1, L1);
    L1.st = it1->storage;
    float* tau_ws = cv.take<float>(2 * (size_t)(n2 + 1) * (n1 + 1));
    // tau kept in the workspace follows the step-1 dual: FP16 for an FP16 or
    // fixed-point dual (tau is not bounded by 1), BF16 for a BF16 dual
    const int tau_st = tau ? TVS_F32 : (it1->storage == TVS_BF16 ? TVS_BF16 : (it1->storage == TVS_F32 ? TVS_F32 : TVS_F16));
    void* tau_use = tau ? static_cast<void*>(tau) : static_cast<void*>(tau_ws);
    Step2Layout L2;
    layout_step2(cv, n2, n1, L2, it2->storage);
    tvs_report r1{}, r2{};
    tvs_status s1 = run_tfs(L1, d0, n2, n1, delta, *it1, tau_use, tau_st, n1 + 1, (long)(n2 + 1) * (n1 + 1), nullptr,
                            stream, &r1);
    if (s1 != TVS_OK && s1 != TVS_ERR_NOT_CONVERGED) return s1;
    tvs_status s2;
    if (dd2) {
        Schwarz2State S2;
        schwarz2_carve(cv, n2, n1, *dd2, L2.P, it2->storage, S2);
        const int R = n2 + 1, C = n1 + 1;
        TVS_CUDA(launch_xi_f2_st(d0, n1, tau_use, tau_st, (long)R * C, C, n2, n1, (float)alpha, (float)eps, L2.f2,
                                 L2.P, stream));
        s2 = run_schwarz2(L2, S2, n2, n1, alpha, *it2, d, nullptr, stream, &r2);
    } else {
        s2 = run_irv1(L2, d0, tau_use, n2, n1, alpha, eps, *it2, d, nullptr, stream, &r2, tau_st);
    }
    if (rep) {
        rep[0] = r1;
        rep[1] = r2;
    }
    if (s2 != TVS_OK) return s2;
    return s1;
}

}  // extern "C"
