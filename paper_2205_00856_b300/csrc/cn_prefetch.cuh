// cn_prefetch.cuh -- bulk L2 prefetch (cp.async.bulk.prefetch.L2): one
// instruction asks the memory system to bring a contiguous range into L2, with
// no destination registers or shared memory and nothing to wait for.  The
// range must start and end on 16-byte boundaries (both the address and the
// size), which the callers' layouts guarantee.
#pragma once
#include <cstdint>

#include "cn_debug.cuh"

namespace cnb {

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
#if defined(CN_DEBUG)
    if (!dbg_ok(src, bytes)) return;  // a range outside the registered buffers is a layout error
#endif
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

}  // namespace cnb
