// Cache of instantiated CUDA graphs for the iteration drivers (graphs.h).
#include "graphs.h"
#include "prof.h"

#include <atomic>
#include <mutex>
#include <vector>

namespace tvs {

namespace {
constexpr size_t kMaxGraphs = 32;   // least recently used beyond this are destroyed

struct Entry {
    GraphKey key;
    int device;
    cudaGraphExec_t exec;
    uint64_t last;
};

std::mutex g_mu;
std::vector<Entry> g_cache;
uint64_t g_tick = 0;
thread_local int g_off = 0;
std::atomic<int> g_global_on{1};

// The capture stream of this thread on the current device.
cudaStream_t capture_stream(int device) {
    thread_local cudaStream_t cs = nullptr;
    thread_local int cs_dev = -1;
    if (!cs || cs_dev != device) {
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
            cs = nullptr;
            return nullptr;
        }
        cs_dev = device;
    }
    return cs;
}
}  // namespace

bool graphs_enabled() { return g_off == 0 && g_global_on.load(std::memory_order_relaxed) != 0 && !prof_enabled(); }

GraphsOff::GraphsOff() { ++g_off; }
GraphsOff::~GraphsOff() { --g_off; }

bool graph_capture(const std::function<cudaError_t(cudaStream_t)>& enqueue, cudaGraphExec_t* out) {
    *out = nullptr;
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    cudaStream_t cs = capture_stream(device);
    if (!cs || cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const cudaError_t launched = enqueue(cs);
    cudaGraph_t graph = nullptr;
    const cudaError_t ended = cudaStreamEndCapture(cs, &graph);
    if (launched != cudaSuccess || ended != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return false;
    }
    const cudaError_t inst = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (inst != cudaSuccess) {
        *out = nullptr;
        cudaGetLastError();
        return false;
    }
    return true;
}

cudaError_t graph_run(const GraphKey& key, cudaStream_t s, const std::function<cudaError_t(cudaStream_t)>& enqueue) {
    if (!graphs_enabled() || !key.valid()) return enqueue(s);
    int device = 0;
    if (cudaGetDevice(&device) != cudaSuccess) return enqueue(s);
    cudaGraphExec_t exec = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        for (Entry& e : g_cache)
            if (e.device == device && e.key == key) {
                e.last = ++g_tick;
                exec = e.exec;
                break;
            }
    }
    if (exec) return cudaGraphLaunch(exec, s);

    if (!graph_capture(enqueue, &exec)) return enqueue(s);
    {
        std::lock_guard<std::mutex> lk(g_mu);
        if (g_cache.size() >= kMaxGraphs) {
            size_t lru = 0;
            for (size_t i = 1; i < g_cache.size(); ++i)
                if (g_cache[i].last < g_cache[lru].last) lru = i;
            cudaGraphExecDestroy(g_cache[lru].exec);
            g_cache.erase(g_cache.begin() + (long)lru);
        }
        g_cache.push_back(Entry{key, device, exec, ++g_tick});
    }
    return cudaGraphLaunch(exec, s);
}


}  // namespace tvs

extern "C" int tvs_set_graphs(int on) { return tvs::g_global_on.exchange(on ? 1 : 0); }
