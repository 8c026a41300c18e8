// cn_tma.cuh -- bulk asynchronous copies global -> shared (TMA, cp.async.bulk)
// completed on a shared-memory mbarrier, with a bounded wait.
//
// One thread initialises the barrier, announces the byte count the phase will
// receive (arrive.expect_tx) and issues the copies; every thread then waits on
// phase 0.  A copy must start and end on 16-byte boundaries (both addresses and
// the size), which the callers' layouts guarantee.
#pragma once
#include <cstdint>

namespace cnb {

constexpr int kStatusTimeout = 5;        // cn_status CN_ERR_TIMEOUT
constexpr int kWaitSpinLimit = 1 << 24;  // polls of a barrier (with a 64 ns back-off: about a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the async proxy that completes it
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// bytes: multiple of 16; dst and src 16-byte aligned
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// Bulk prefetch of [src, src + bytes) into L2 (no destination, no completion to
// wait for); bytes a multiple of 16, src 16-byte aligned.
__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Wait for phase `parity` of the barrier, giving up after `limit` polls.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, int limit = kWaitSpinLimit) {
    for (int i = 0; i < limit; ++i) {
        if (mbar_test_wait(bar, parity)) return true;
        if (i >= 32) __nanosleep(64);
    }
    return false;
}

// Diagnostics: one CTA waits, as the TMA-staged kernels do, on a barrier that
// nothing completes (it expects one arrival that never comes), with a limit of
// `limit` polls, and reports the timeout in the status word like they do.
static __global__ void k_diag_wait_timeout(int* status, int limit) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    const bool landed = mbar_wait_bounded(&bar, 0, limit);
    if (!landed && threadIdx.x == 0) atomicCAS(status, 0, kStatusTimeout);
}

}  // namespace cnb
