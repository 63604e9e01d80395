// Tensor-memory-accelerator (TMA) loads and mbarrier waits for the streaming
// stencil kernels (sm_100-family PTX: cp.async.bulk.tensor, mbarrier with
// transaction counts).  Every wait is bounded: after kWaitCycles SM cycles
// the caller gets `false`, records an error and drains its own copies.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cstdint>

namespace tvs {

constexpr long long kWaitCycles = 4000000000LL;   // about two seconds of SM clock before a wait gives up

// Limit of the first wait on a phase, in SM cycles.  Each translation unit
// that waits has its own copy; tvs_set_wait_limit sets all of them (a
// diagnostic: a short limit makes waits give up on copies still in flight,
// so the timeout path can be tested without a stuck copy).  The drain after
// a wait gave up always uses kWaitCycles.
static __constant__ long long c_wait_limit = kWaitCycles;
static inline cudaError_t set_wait_limit_here(long long cycles) {
    return cudaMemcpyToSymbol(c_wait_limit, &cycles, sizeof cycles);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Make initialised barriers visible to the async (TMA) proxy.
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) writes to it.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// One poll; the thread may sleep in hardware until the phase completes or
// kSuspendNs nanoseconds pass, so a waiting warp does not spin on the issue
// slots the other warps need.
constexpr uint32_t kSuspendNs = 1000000;
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}

// One poll that never suspends the thread.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of `bar` for at most `limit` SM cycles.
__device__ __forceinline__ bool mbar_wait_for(uint64_t* bar, uint32_t parity, long long limit) {
    if (limit < kWaitCycles) {
        // short (diagnostic) limit: poll without suspending
        const long long t0 = clock64();
        while (!mbar_test_wait(bar, parity))
            if (clock64() - t0 > limit) return false;
        return true;
    }
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Bounded wait for phase `parity` of `bar`; false if it did not complete
// within the current limit (c_wait_limit, normally kWaitCycles).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    return mbar_wait_for(bar, parity, c_wait_limit);
}

// After a wait gave up: wait for the copies still in flight (kWaitCycles).
__device__ __forceinline__ bool mbar_drain(uint64_t* bar, uint32_t parity) {
    return mbar_wait_for(bar, parity, kWaitCycles);
}

// 2-D / 3-D tiled loads into this CTA's shared memory; x is the innermost
// coordinate (elements) and must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
        "[%5];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
        : "memory");
}

// Host: tiled tensor map of `planes` planes of rows x cols elements
// (element pitch `pitch`, plane stride `plane` elements) with a box of
// box_x x box_y x planes.  Returns false if the driver rejects it.
bool make_tensor_map(CUtensorMap* map, const void* base, int storage, int rows, int cols, int pitch, long plane,
                     int planes, int box_x, int box_y);

}  // namespace tvs
