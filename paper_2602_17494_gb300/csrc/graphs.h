// Replay of fixed launch sequences through instantiated CUDA graphs.
//
// The iteration drivers enqueue runs of identical iterations (between two
// convergence checks) through graph_run: the first run with a given key is
// captured on a private stream and instantiated; later runs with the same key
// are a single cudaGraphLaunch on the caller's stream.  The key holds every
// pointer and scalar the captured kernels receive, so a hit replays exactly
// the launches the caller would have made.  The programmatic dependencies
// between the captured kernels are kept as graph edges.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <functional>

namespace tvs {

struct GraphKey {
    static constexpr int kMax = 40;
    uint64_t w[kMax];
    int n = 0;
    GraphKey& add(uint64_t x) {
        if (n < kMax) w[n] = x;
        ++n;
        return *this;
    }
    GraphKey& ptr(const void* p) { return add(static_cast<uint64_t>(reinterpret_cast<uintptr_t>(p))); }
    GraphKey& num(double x) {
        uint64_t u;
        std::memcpy(&u, &x, sizeof(u));
        return add(u);
    }
    bool valid() const { return n <= kMax; }
    bool operator==(const GraphKey& o) const { return n == o.n && std::memcmp(w, o.w, sizeof(uint64_t) * n) == 0; }
};

// False while kernel profiling is on or inside a GraphsOff scope (the
// drivers then launch directly).
bool graphs_enabled();

// Scope on the calling thread in which graph_run launches directly (used by
// the autotuner, whose timings must not include capture).
struct GraphsOff {
    GraphsOff();
    ~GraphsOff();
    GraphsOff(const GraphsOff&) = delete;
    GraphsOff& operator=(const GraphsOff&) = delete;
};

// Captures enqueue(stream) on a private stream into an instantiated graph
// (*out, owned by the caller, cudaGraphExecDestroy).  Returns false (and
// leaves no error pending) if capture or instantiation fails.
bool graph_capture(const std::function<cudaError_t(cudaStream_t)>& enqueue, cudaGraphExec_t* out);

// Runs enqueue(stream) on s: through the cached graph of `key` (capturing it
// on first use) when graphs are enabled, else directly.  Capture or
// instantiation failures fall back to the direct launches.
cudaError_t graph_run(const GraphKey& key, cudaStream_t s, const std::function<cudaError_t(cudaStream_t)>& enqueue);

}  // namespace tvs
