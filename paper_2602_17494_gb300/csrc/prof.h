// Opt-in per-kernel-class timing with CUDA events (see prof.cu).
#pragma once

#include <cuda_runtime.h>

#include "../../include/tvs.h"

namespace tvs {

enum ProfClass : int {
    kProfRowsFwd = 0,
    kProfCols = 1,
    kProfRowsInv = 2,
    kProfTfsUpdate = 3,
    kProfIrv1Update = 4,
    kProfSchwarzTile = 5,
    kProfSchwarzCombine = 6,
    kProfOther = 7,
    kProfTfsCheck = 8,
    kProfIrv1Check = 9,
    kProfSetup = 10,        // once-per-call kernels: tables, tau0, xi and f2, the last P_K step, reductions
    kProfClasses = 11
};

// True while per-kernel profiling is on.
bool prof_enabled();

// Records an event on `s` at construction and at destruction when profiling
// is enabled; a no-op otherwise.  `kernels` is the number of kernel launches
// the scope covers (the launch count of its class grows by that much).
class ProfScope {
public:
    ProfScope(ProfClass cls, cudaStream_t s, int kernels = 1);
    ~ProfScope();
    ProfScope(const ProfScope&) = delete;
    ProfScope& operator=(const ProfScope&) = delete;

private:
    ProfClass cls_;
    int kernels_;
    cudaStream_t s_;
    cudaEvent_t a_;
};

}  // namespace tvs
