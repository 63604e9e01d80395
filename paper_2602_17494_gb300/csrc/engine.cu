// Batching and serving engine (include/tvs.h, tvs_engine_*).  The paper
// denoises one image at a time; this host runtime keeps many requests of
// different sizes resident on the device and advances them together:
//   * admission: FIFO, a request is admitted when its state fits the free
//     part of the caller's device pool and a slot is free;
//   * step 1 (TFS, Algorithm 1): each request runs its own chunk of updates,
//     spread over a few side streams so that small images overlap;
//   * step 2 (IRV1 under Algorithm 2 with Algorithm 3): all live step-2
//     requests share one persistent cooperative launch per engine step that
//     sweeps the subdomain tiles of all of them for check_every outer
//     iterations (grid barriers between the tile and strip phases); with an
//     even check_every that launch and every request's check are captured
//     once per set of resident step-2 requests into a CUDA graph, replayed
//     while the set is unchanged;
//   * every engine step ends with one stream synchronization; requests whose
//     relative duality gap reached the tolerance move on (or finish: d is
//     written to the caller's buffer and the pool block is released).
// All state stays on the device between steps; the host keeps only indices
// and the per-request reduction results.
#include "drivers.h"
#include "graphs.h"

#include <algorithm>
#include <cmath>
#include <deque>
#include <map>
#include <vector>

namespace tvs {

namespace {

constexpr int kSideStreams = 16;
constexpr int kCapStreams = 8;    // private streams of the captured step-2 checks

// First-fit allocator over [0, size) of the caller's pool (256-byte units).
class PoolAlloc {
public:
    explicit PoolAlloc(size_t size) { free_[0] = size; }
    bool alloc(size_t bytes, size_t* off) {
        bytes = round_up_sz(bytes, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t at = it->first + bytes;
                free_.erase(it);
                if (rest) free_[at] = rest;
                used_[*off] = bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off) {
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t start = off, len = u->second;
        used_.erase(u);
        auto next = free_.lower_bound(start);
        if (next != free_.end() && next->first == start + len) {
            len += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == start) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        free_[start] = len;
    }

private:
    std::map<size_t, size_t> free_, used_;
};

struct Request {
    long long id;
    int n2, n1;
    const float* d0;
    float* d;
    size_t off = 0;
    int stage = 0;          // 1: step 1, 2: step 2
    int it1 = 0, it2 = 0;   // updates / outer iterations done
    Step1Layout L1;
    Step2Layout L2;
    Schwarz2State S2;
    float* tau = nullptr;
    float *cur1 = nullptr, *nxt1 = nullptr;
    void *cur2 = nullptr, *nxt2 = nullptr;
    int side = 0;           // side stream of the step-1 chunks and the step-2 checks
    int slot = 0;           // row of the pinned result array
    bool checked = false;   // a check was enqueued this engine step
    tvs_report rep[2] = {};
    cudaGraphExec_t g1 = nullptr;   // captured full step-1 chunk (check_every even), replayed each engine step
    Request() = default;
    Request(const Request&) = delete;
    Request& operator=(const Request&) = delete;
    ~Request() {
        if (g1) cudaGraphExecDestroy(g1);
    }
};

// Step-2 decomposition of an image under the engine's tile policy.
tvs_decomp tile_decomp(const tvs_engine_config& c, int n2, int n1) {
    tvs_decomp dd{};
    dd.m2 = std::max(1, (n2 + c.tile - 1) / c.tile);   // cores of at most tile pixels
    dd.m1 = std::max(1, (n1 + c.tile - 1) / c.tile);
    dd.overlap = c.overlap;
    dd.k_inner = c.k_inner;
    dd.alpha_hat = 0.0;
    return dd;
}

// Carves a request's state: the tvs_denoise layout (step 1, tau, step 2 with
// its Schwarz warm starts).  Returns the bytes used.
size_t carve_request(Carver& cv, const tvs_engine_config& c, int n2, int n1, Request* r) {
    Step1Layout L1;
    layout_step1(cv, n2, n1, L1);
    float* tau = cv.take<float>(2 * (size_t)(n2 + 1) * (n1 + 1));
    Step2Layout L2;
    layout_step2(cv, n2, n1, L2, c.it2.storage);
    Schwarz2State S2;
    const tvs_decomp dd = tile_decomp(c, n2, n1);
    schwarz2_carve(cv, n2, n1, dd, L2.P, c.it2.storage, S2);
    if (r) {
        r->L1 = L1;
        r->tau = tau;
        r->L2 = L2;
        r->S2 = S2;
    }
    return cv.used();
}

}  // namespace

struct EngineImpl {
    tvs_engine_config cfg;
    char* pool;
    size_t pool_bytes;
    PoolAlloc alloc;
    cudaStream_t stream;
    cudaStream_t side[kSideStreams];
    cudaEvent_t ev_main, ev_s2, ev_side[kSideStreams];   // ev_s2: the shared step-2 launches are enqueued
    std::deque<Request*> queue;
    std::vector<Request*> live;
    std::vector<Request*> done;
    double* host_red = nullptr;       // pinned [max_live][kRedSlots]
    TileImg* host_imgs = nullptr;     // pinned [2 * max_live]
    TileImg* dev_imgs = nullptr;      // head of the pool
    unsigned* dev_sync = nullptr;     // pool head: [0, 2) grid barrier, [2] error word, [3] rounding-seed counter
    unsigned* host_err = nullptr;     // pinned copy of the error word
    cudaStream_t cap[kCapStreams] = {};
    cudaStream_t gcap = nullptr;      // private stream the step-2 chunk is captured on
    cudaEvent_t ev_cap[kCapStreams] = {};
    cudaGraphExec_t g2 = nullptr;     // captured step-2 chunk of the set g2_set
    std::vector<uintptr_t> g2_set;    // per request: id, both dual buffers, result slot
    std::vector<int> free_slots;
    int next_side = 0;

    explicit EngineImpl(size_t n) : alloc(n) {}
};

}  // namespace tvs

struct tvs_engine {
    tvs::EngineImpl* impl;
};

using namespace tvs;

static tvs_status engine_check_cfg(const tvs_engine_config* c) {
    if (!c || !(c->delta > 0.0) || !(c->alpha > 0.0) || !(c->eps > 0.0)) return TVS_ERR_ARG;
    tvs_status st = check_iter(&c->it1, false);
    if (st != TVS_OK) return st;
    st = check_iter(&c->it2, true);
    if (st != TVS_OK) return st;
    if (c->it1.check_every < 1 || c->it2.check_every < 1 || c->it1.max_iter < 1 || c->it2.max_iter < 1)
        return TVS_ERR_ARG;
    if (c->tile < 16 || c->overlap < 0 || 2 * c->overlap >= c->tile || c->k_inner < 1 || c->max_live < 1)
        return TVS_ERR_ARG;
    int tx, ty, qp;
    size_t smem;
    if (!small_tile_shape(c->tile + c->overlap, c->tile + c->overlap, &tx, &ty, &qp, &smem))
        return TVS_ERR_UNSUPPORTED;   // subdomains must fit the one-CTA-per-subdomain kernel
    return TVS_OK;
}

static size_t engine_header_bytes(const tvs_engine_config* c) {
    return round_up_sz(2 * (size_t)c->max_live * sizeof(TileImg), 256) + 256;   // descriptors, sync words
}

extern "C" {

size_t tvs_engine_request_bytes(const tvs_engine_config* cfg, int n2, int n1) {
    if (engine_check_cfg(cfg) != TVS_OK || !side_ok(n2) || !side_ok(n1)) return 0;
    const tvs_decomp dd = tile_decomp(*cfg, n2, n1);
    if (schwarz2_check(n2, n1, dd) != TVS_OK) return 0;
    Carver cv(nullptr);
    return carve_request(cv, *cfg, n2, n1, nullptr);
}

size_t tvs_engine_pool_overhead(const tvs_engine_config* cfg) {
    if (engine_check_cfg(cfg) != TVS_OK) return 0;
    return engine_header_bytes(cfg);
}

tvs_status tvs_engine_create(const tvs_engine_config* cfg, void* pool, size_t pool_bytes, cudaStream_t stream,
                             tvs_engine** out) {
    if (!out) return TVS_ERR_ARG;
    *out = nullptr;
    tvs_status st = engine_check_cfg(cfg);
    if (st != TVS_OK) return st;
    const size_t head = engine_header_bytes(cfg);
    if (!pool || (reinterpret_cast<uintptr_t>(pool) & 255u) || pool_bytes <= head) return TVS_ERR_WORKSPACE;
    auto* e = new EngineImpl(pool_bytes - head);
    e->cfg = *cfg;
    e->pool = static_cast<char*>(pool) + head;
    e->pool_bytes = pool_bytes - head;
    e->stream = stream;
    e->dev_imgs = static_cast<TileImg*>(pool);
    e->dev_sync = reinterpret_cast<unsigned*>(static_cast<char*>(pool) +
                                              round_up_sz(2 * (size_t)cfg->max_live * sizeof(TileImg), 256));
    bool ok = cudaHostAlloc(reinterpret_cast<void**>(&e->host_red), (size_t)cfg->max_live * kRedSlots * sizeof(double),
                            cudaHostAllocDefault) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&e->host_imgs), 2 * (size_t)cfg->max_live * sizeof(TileImg),
                            cudaHostAllocDefault) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->ev_main, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->ev_s2, cudaEventDisableTiming) == cudaSuccess &&
              cudaHostAlloc(reinterpret_cast<void**>(&e->host_err), sizeof(unsigned), cudaHostAllocDefault) ==
                  cudaSuccess &&
              cudaMemsetAsync(e->dev_sync, 0, 4 * sizeof(unsigned), stream) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&e->gcap, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < kCapStreams; ++i)
        ok = cudaStreamCreateWithFlags(&e->cap[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->ev_cap[i], cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < kSideStreams; ++i)
        ok = cudaStreamCreateWithFlags(&e->side[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->ev_side[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        set_error_text("tvs_engine_create: host allocation or stream creation failed");
        auto* h = new tvs_engine{e};
        tvs_engine_destroy(h);
        return TVS_ERR_CUDA;
    }
    for (int i = cfg->max_live - 1; i >= 0; --i) e->free_slots.push_back(i);
    *out = new tvs_engine{e};
    return TVS_OK;
}

tvs_status tvs_engine_submit(tvs_engine* h, long long id, const float* d0, int n2, int n1, float* d) {
    if (!h || !d0 || !d || !side_ok(n2) || !side_ok(n1)) return TVS_ERR_ARG;
    EngineImpl* e = h->impl;
    const size_t need = tvs_engine_request_bytes(&e->cfg, n2, n1);
    if (need == 0) return TVS_ERR_UNSUPPORTED;
    if (need > e->pool_bytes) return TVS_ERR_UNSUPPORTED;   // could never be admitted
    auto* r = new Request();
    r->id = id;
    r->n2 = n2;
    r->n1 = n1;
    r->d0 = d0;
    r->d = d;
    e->queue.push_back(r);
    return TVS_OK;
}

int tvs_engine_pending(const tvs_engine* h) {
    if (!h) return 0;
    return (int)(h->impl->queue.size() + h->impl->live.size() + h->impl->done.size());
}

void tvs_engine_destroy(tvs_engine* h) {
    if (!h) return;
    EngineImpl* e = h->impl;
    if (e) {
        cudaStreamSynchronize(e->stream);
        for (int i = 0; i < kSideStreams; ++i) {
            if (e->side[i]) {
                cudaStreamSynchronize(e->side[i]);
                cudaStreamDestroy(e->side[i]);
            }
            if (e->ev_side[i]) cudaEventDestroy(e->ev_side[i]);
        }
        if (e->g2) cudaGraphExecDestroy(e->g2);
        for (int i = 0; i < kCapStreams; ++i) {
            if (e->cap[i]) {
                cudaStreamSynchronize(e->cap[i]);
                cudaStreamDestroy(e->cap[i]);
            }
            if (e->ev_cap[i]) cudaEventDestroy(e->ev_cap[i]);
        }
        if (e->gcap) cudaStreamDestroy(e->gcap);
        if (e->host_err) cudaFreeHost(e->host_err);
        if (e->ev_main) cudaEventDestroy(e->ev_main);
        if (e->ev_s2) cudaEventDestroy(e->ev_s2);
        if (e->host_red) cudaFreeHost(e->host_red);
        if (e->host_imgs) cudaFreeHost(e->host_imgs);
        for (Request* r : e->queue) delete r;
        for (Request* r : e->live) delete r;
        for (Request* r : e->done) delete r;
        delete e;
    }
    delete h;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// One engine step
// ---------------------------------------------------------------------------
static tvs_status admit(EngineImpl* e) {
    while (!e->queue.empty() && !e->free_slots.empty()) {
        Request* r = e->queue.front();
        Carver cv0(nullptr);
        const size_t need = carve_request(cv0, e->cfg, r->n2, r->n1, nullptr);
        size_t off;
        if (!e->alloc.alloc(need, &off)) break;   // FIFO: wait until the head fits
        e->queue.pop_front();
        r->off = off;
        Carver cv(e->pool + off);
        carve_request(cv, e->cfg, r->n2, r->n1, r);
        r->slot = e->free_slots.back();
        e->free_slots.pop_back();
        r->side = e->next_side;
        e->next_side = (e->next_side + 1) % kSideStreams;
        cudaStream_t s = e->side[r->side];
        tvs_status st = tfs_setup(r->L1, r->d0, r->n2, r->n1, e->cfg.delta, s);
        if (st != TVS_OK) return st;
        TVS_CUDA(cudaMemsetAsync(r->L1.pa, 0, 4 * (size_t)r->L1.plane * sizeof(float), s));
        r->cur1 = r->L1.pa;
        r->nxt1 = r->L1.pb;
        r->stage = 1;
        e->live.push_back(r);
    }
    return TVS_OK;
}

// Step-1 chunk of one request on its side stream; the last update of the
// chunk also evaluates the gap at its input iterate.
// n TFS updates (the last with the check sums), the reduction and its copy
// to the request's row of the pinned result array, on stream s; cur1/nxt1
// alternate from *cur, *nxt.
// The updates are the fused step of the global loop: div(vecdiv p) of the
// chunk's first iterate, then per update the Poisson solve of the current
// source and the update that also writes the next source.
static cudaError_t step1_launches(EngineImpl* e, Request* r, int n, float** cur, float** nxt, cudaStream_t s) {
    const Step1Layout& L = r->L1;
    const float t = (float)e->cfg.it1.t;
    cudaError_t err = launch_div_vecdiv_st(*cur, TVS_F32, L.R, L.C, L.P, L.plane, L.src, L.red.err, s);
    if (err != cudaSuccess) return err;
    for (int j = 0; j < n; ++j) {
        const bool ck = j == n - 1;
        RowSrcArgs sa{L.src, 0, L.P};
        err = poisson_solve(L.S, L.R, L.C, L.P, L.pp, RowSource::Plain, sa, s);
        if (err != cudaSuccess) return err;
        err = launch_tfs_step_st(*cur, *nxt, TVS_F32, 0u, L.S, L.f1, L.src, L.R, L.C, L.P, L.plane, t, ck,
                                 L.red.partial, L.red.err, s);
        if (err != cudaSuccess) return err;
        std::swap(*cur, *nxt);
    }
    err = finalize_red(L.red, tfs_blocks(L.R, L.C), s);
    if (err != cudaSuccess) return err;
    return cudaMemcpyAsync(e->host_red + (size_t)r->slot * kRedSlots, L.red.result, kRedSlots * sizeof(double),
                           cudaMemcpyDeviceToHost, s);
}

static tvs_status step1_chunk(EngineImpl* e, Request* r) {
    cudaStream_t s = e->side[r->side];
    const int n = std::min(e->cfg.it1.check_every, e->cfg.it1.max_iter - r->it1);
    // a full chunk of an even number of updates leaves p in the buffer it
    // started from, so one captured graph per request serves every such chunk
    if (n == e->cfg.it1.check_every && n % 2 == 0 && graphs_enabled()) {
        if (!r->g1) {
            float* c0 = r->cur1;
            float* c1 = r->nxt1;
            graph_capture([&](cudaStream_t cs) { return step1_launches(e, r, n, &c0, &c1, cs); }, &r->g1);
        }
        if (r->g1) {
            TVS_CUDA(cudaGraphLaunch(r->g1, s));
            r->it1 += n;
            r->checked = true;
            return TVS_OK;
        }
    }
    TVS_CUDA(step1_launches(e, r, n, &r->cur1, &r->nxt1, s));
    r->it1 += n;
    r->checked = true;
    return TVS_OK;
}

// tau of the finished step 1, then the step-2 data f2 and a zero dual (on the
// main stream, which runs the request's step 2 from the next engine step on).
static tvs_status step1_to_step2(EngineImpl* e, Request* r) {
    const Step1Layout& L = r->L1;
    cudaStream_t s = e->stream;
    if (r->g1) {   // step 1 is over; its graph is not replayed again
        cudaGraphExecDestroy(r->g1);
        r->g1 = nullptr;
    }
    unsigned err = 0;   // step 1 finished on a side stream that the last synchronization covered
    TVS_CUDA(cudaMemcpy(&err, L.red.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
    if (err) {
        set_error_text("a bounded device-side wait gave up (TMA tile load)");
        return TVS_ERR_TIMEOUT;
    }
    const int n2 = r->n2, n1 = r->n1, R = n2 + 1, C = n1 + 1;
    TVS_CUDA(tfs_phi(r->cur1, L.S, L.R, L.C, L.P, L.plane, L.pp, L.red.err, s));
    TVS_CUDA(launch_tfs_update(r->cur1, nullptr, L.S, L.f1, L.R, L.C, L.P, L.plane, (float)e->cfg.it1.t,
                               (float)e->cfg.delta, false, false, r->tau, C, (long)R * C, L.red.partial, L.red.err, s));
    TVS_CUDA(launch_xi_f2(r->d0, n1, r->tau, (long)R * C, C, n2, n1, (float)e->cfg.alpha, (float)e->cfg.eps,
                          r->L2.f2, r->L2.P, s));
    TVS_CUDA(p2_zero(r->L2, s));
    TVS_CUDA(cudaMemsetAsync(r->L2.red.err, 0, sizeof(unsigned), s));
    TVS_CUDA(schwarz2_reset(r->S2, s));
    r->cur2 = r->L2.pa;
    r->nxt2 = r->L2.pb;
    r->stage = 2;
    return TVS_OK;
}

// Enqueues one step-2 chunk of the requests rs: the persistent sweep of n
// outer iterations on the main stream, then each request's check (update
// kernel in check mode, reduction, copy of the result row to pinned memory)
// on a side stream (cap: the private capture streams, joined back into the
// main stream).  The checks read p where the chunk leaves it (cur2 after an
// even n, nxt2 after an odd one).
static tvs_status step2_enqueue(EngineImpl* e, const std::vector<Request*>& rs, int nsub, int tx, int ty, int n,
                                bool cap, cudaStream_t ms) {
    const tvs_engine_config& c = e->cfg;
    const int nimg = (int)rs.size();
    TVS_CUDA(schwarz2_persist_multi(c.it2.storage, e->dev_imgs, nimg, nsub, tx, ty, c.k_inner, (float)c.it2.t, n,
                                    e->dev_sync, e->dev_sync + 2, e->dev_sync + 3, ms));
    TVS_CUDA(cudaEventRecord(e->ev_s2, ms));
    bool waited[kSideStreams] = {};
    for (int i = 0; i < nimg; ++i) {
        Request* r = rs[i];
        const Step2Layout& L = r->L2;
        const int si = cap ? i % kCapStreams : r->side;
        cudaStream_t ss = cap ? e->cap[si] : e->side[si];
        if (!waited[si]) {
            TVS_CUDA(cudaStreamWaitEvent(ss, e->ev_s2, 0));
            waited[si] = true;
        }
        void* p = (n & 1) ? r->nxt2 : r->cur2;
        TVS_CUDA(launch_irv1_update(p, nullptr, L.f2, L.R, L.C, L.P, L.plane, (float)c.it2.t, (float)c.alpha, true,
                                    false, nullptr, 0, L.red.partial, L.st, 0u, L.red.err, ss));
        TVS_CUDA(finalize_red(L.red, irv1_blocks(L.R, L.C), ss));
        TVS_CUDA(cudaMemcpyAsync(e->host_red + (size_t)r->slot * kRedSlots, L.red.result, kRedSlots * sizeof(double),
                                 cudaMemcpyDeviceToHost, ss));
    }
    if (cap)
        for (int si = 0; si < kCapStreams; ++si)
            if (waited[si]) {
                TVS_CUDA(cudaEventRecord(e->ev_cap[si], e->cap[si]));
                TVS_CUDA(cudaStreamWaitEvent(ms, e->ev_cap[si], 0));
            }
    return TVS_OK;
}

// All live step-2 requests: check_every outer iterations in one persistent
// launch, then one check per request.  With an even check_every the
// descriptors of a set of requests do not change from step to step, so the
// chunk is captured into a CUDA graph the second time the same set comes
// round and replayed while the set lasts.
static tvs_status step2_chunk(EngineImpl* e, std::vector<Request*>& rs) {
    if (rs.empty()) {
        if (e->g2) TVS_CUDA(cudaGraphExecDestroy(e->g2));
        e->g2 = nullptr;
        e->g2_set.clear();
        return TVS_OK;
    }
    const tvs_engine_config& c = e->cfg;
    std::vector<uintptr_t> key;
    for (Request* r : rs) {
        key.push_back((uintptr_t)r->id);
        key.push_back(reinterpret_cast<uintptr_t>(r->cur2));
        key.push_back(reinterpret_cast<uintptr_t>(r->nxt2));
        key.push_back((uintptr_t)r->slot);
    }
    const int nimg = (int)rs.size();
    int nsub = 0, tx = 1, ty = 1;
    // every request advances check_every outer iterations (its cap may be
    // passed by less than one chunk)
    const int n = c.it2.check_every;
    for (int i = 0; i < nimg; ++i) {
        Request* r = rs[i];
        const Schwarz2State& S2 = r->S2;
        Axis ay{r->n2, S2.m2, S2.s, r->n2}, ax{r->n1, S2.m1, S2.s, r->n1};
        TileImg a{r->cur2, r->nxt2, r->L2.f2, S2.q, r->L2.P, r->L2.plane, S2.hmax, S2.qp, ay, ax,
                  (float)S2.alpha_hat, nsub};
        TileImg b = a;                        // odd outer iterations: buffers swapped
        b.p = r->nxt2;
        b.pnext = r->cur2;
        e->host_imgs[i] = a;
        e->host_imgs[nimg + i] = b;
        nsub += S2.m2 * S2.m1;
        tx = std::max(tx, S2.tx);
        ty = std::max(ty, S2.ty);
    }
    const bool graph_ok = graphs_enabled() && (n & 1) == 0;
    if (graph_ok && e->g2 && e->g2_set == key) {
        TVS_CUDA(cudaGraphLaunch(e->g2, e->stream));       // descriptors already in place for this set
    } else {
        const bool capture = graph_ok && e->g2_set == key;  // the same set a second time: capture it
        if (e->g2) {
            TVS_CUDA(cudaGraphExecDestroy(e->g2));
            e->g2 = nullptr;
        }
        // the host array is rewritten next step, after this step's synchronization
        TVS_CUDA(cudaMemcpyAsync(e->dev_imgs, e->host_imgs, 2 * (size_t)nimg * sizeof(TileImg),
                                 cudaMemcpyHostToDevice, e->stream));
        if (capture) {
            // captured on a private stream (the caller's may be the legacy
            // default stream, which cannot be captured), launched on the caller's
            cudaGraph_t g = nullptr;
            TVS_CUDA(cudaStreamBeginCapture(e->gcap, cudaStreamCaptureModeThreadLocal));
            const tvs_status st = step2_enqueue(e, rs, nsub, tx, ty, n, true, e->gcap);
            const cudaError_t ce = cudaStreamEndCapture(e->gcap, &g);
            if (st != TVS_OK) {
                if (g) cudaGraphDestroy(g);
                return st;
            }
            TVS_CUDA(ce);
            const cudaError_t ie = cudaGraphInstantiate(&e->g2, g, 0);
            cudaGraphDestroy(g);
            TVS_CUDA(ie);
            TVS_CUDA(cudaGraphLaunch(e->g2, e->stream));
        } else {
            const tvs_status st = step2_enqueue(e, rs, nsub, tx, ty, n, false, e->stream);
            if (st != TVS_OK) return st;
        }
        e->g2_set = key;
    }
    TVS_CUDA(cudaMemcpyAsync(e->host_err, e->dev_sync + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, e->stream));
    for (Request* r : rs) {
        if (n & 1) std::swap(r->cur2, r->nxt2);
        r->it2 += n;
        r->checked = true;
    }
    return TVS_OK;
}

extern "C" tvs_status tvs_engine_step(tvs_engine* h, long long* done_ids, tvs_report* done_reports, int cap,
                                      int* n_done) {
    if (!h || !n_done || cap < 0 || (cap > 0 && !done_ids)) return TVS_ERR_ARG;
    EngineImpl* e = h->impl;
    const tvs_engine_config& c = e->cfg;
    *n_done = 0;
    // side streams start after everything already on the main stream
    TVS_CUDA(cudaEventRecord(e->ev_main, e->stream));
    for (int i = 0; i < kSideStreams; ++i) TVS_CUDA(cudaStreamWaitEvent(e->side[i], e->ev_main, 0));
    tvs_status st = admit(e);
    if (st != TVS_OK) return st;
    std::vector<Request*> s2;
    for (Request* r : e->live) {
        r->checked = false;
        if (r->stage == 1) {
            st = step1_chunk(e, r);
            if (st != TVS_OK) return st;
        } else if (r->stage == 2) {
            s2.push_back(r);
        }
    }
    // all live step-2 requests share the launches of this engine step
    st = step2_chunk(e, s2);
    if (st != TVS_OK) return st;
    for (int i = 0; i < kSideStreams; ++i) {
        TVS_CUDA(cudaEventRecord(e->ev_side[i], e->side[i]));
        TVS_CUDA(cudaStreamWaitEvent(e->stream, e->ev_side[i], 0));
    }
    TVS_CUDA(cudaStreamSynchronize(e->stream));
    if (!s2.empty() && *e->host_err) {
        set_error_text("a grid barrier of the persistent Schwarz sweep gave up");
        return TVS_ERR_TIMEOUT;
    }
    // transitions
    std::vector<Request*> finished;
    for (Request* r : e->live) {
        if (!r->checked) continue;
        const double* red = e->host_red + (size_t)r->slot * kRedSlots;
        if (r->stage == 1) {
            report_tfs(red, c.delta, r->it1 - 1, &r->rep[0]);
            if (r->rep[0].rel_gap <= c.it1.rel_gap_tol || r->it1 >= c.it1.max_iter) {
                st = step1_to_step2(e, r);
                if (st != TVS_OK) return st;
            }
        } else {
            report_irv1(red, c.alpha, r->it2, &r->rep[1]);
            if (r->rep[1].rel_gap <= c.it2.rel_gap_tol || r->it2 >= c.it2.max_iter) finished.push_back(r);
        }
    }
    if (!finished.empty()) {
        for (Request* r : finished) {
            const Step2Layout& L = r->L2;
            TVS_CUDA(launch_irv1_update(r->cur2, nullptr, L.f2, L.R, L.C, L.P, L.plane, (float)c.it2.t,
                                        (float)c.alpha, true, false, r->d, r->n1, L.red.partial, L.st, 0u, L.red.err,
                                        e->stream));
        }
        TVS_CUDA(cudaStreamSynchronize(e->stream));
        for (Request* r : finished) {
            unsigned err = 0;
            TVS_CUDA(cudaMemcpy(&err, r->L2.red.err, sizeof(unsigned), cudaMemcpyDeviceToHost));
            if (err) {
                set_error_text("a bounded device-side wait gave up (TMA row load)");
                return TVS_ERR_TIMEOUT;
            }
            e->alloc.release(r->off);
            e->free_slots.push_back(r->slot);
            e->live.erase(std::find(e->live.begin(), e->live.end(), r));
            e->done.push_back(r);
        }
    }
    // hand back finished requests
    int k = 0;
    while (k < cap && !e->done.empty()) {
        Request* r = e->done.front();
        e->done.erase(e->done.begin());
        done_ids[k] = r->id;
        if (done_reports) {
            done_reports[2 * k] = r->rep[0];
            done_reports[2 * k + 1] = r->rep[1];
        }
        delete r;
        ++k;
    }
    *n_done = k;
    return TVS_OK;
}
