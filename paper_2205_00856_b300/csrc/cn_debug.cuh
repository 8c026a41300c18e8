// cn_debug.cuh -- bounds checks of the CN_DEBUG build (compiled in only with
// -DCN_DEBUG; the default build has none of this).
//
// compute-sanitizer is not available where this library is tested, so the
// debug build checks every global-memory access of the kernels itself: before
// each call enqueues work, the host registers the extents of every buffer the
// call may touch (the plan's workspace and the caller's arrays at the sizes the
// call implies) in a table in constant memory; each checked load or store
// verifies that its bytes lie inside one registered extent.  A violation is
// recorded (first address and size; cn_debug_report reads and clears it) and
// the access is skipped -- a load returns zero -- so the check itself never
// touches memory outside the registered buffers.  Shared and local memory are
// not checked.  Each translation unit has its own table.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cnb {

#if defined(CN_DEBUG)
constexpr int kDbgMaxRanges = 128;
struct DbgRange {
    unsigned long long lo, hi;  // [lo, hi)
};
static __constant__ DbgRange g_dbg_ranges[kDbgMaxRanges];
static __constant__ int g_dbg_nranges;
static __device__ int g_dbg_flag;
static __device__ unsigned long long g_dbg_addr;
static __device__ unsigned long long g_dbg_bytes;

__device__ __forceinline__ bool dbg_ok(const void* p, size_t bytes) {
    if (__isShared(p) || __isLocal(p)) return true;
    const unsigned long long a = (unsigned long long)(uintptr_t)p;
    for (int i = 0; i < g_dbg_nranges; ++i)
        if (a >= g_dbg_ranges[i].lo && a + bytes <= g_dbg_ranges[i].hi) return true;
    if (atomicCAS(&g_dbg_flag, 0, 1) == 0) {
        g_dbg_addr = a;
        g_dbg_bytes = bytes;
    }
    return false;
}
#endif

// Checked load and store of one object (plain access in the default build and on the host).
template <class T> __host__ __device__ __forceinline__ T dbg_ld(const T* p) {
#if defined(CN_DEBUG) && defined(__CUDA_ARCH__)
    if (!dbg_ok(p, sizeof(T))) return T{};
#endif
    return *p;
}
template <class T> __host__ __device__ __forceinline__ void dbg_st(T* p, const T& v) {
#if defined(CN_DEBUG) && defined(__CUDA_ARCH__)
    if (!dbg_ok(p, sizeof(T))) return;
#endif
    *p = v;
}

}  // namespace cnb
