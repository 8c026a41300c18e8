// cn_noalloc.cu -- cn_solve_tridiag_noalloc: the general tridiagonal solve of
// cn_solve_tridiag without a plan and without allocating device memory.
//
// Some callers cannot allocate device memory on their solve path: code that
// runs inside a framework whose memory pool owns all device memory, or a
// latency-critical loop where cudaMalloc / cudaFree would synchronise the
// device.  For them the reduced systems of every nesting level live in one
// file-scope device array of fixed size, g_noalloc_scratch, that every GPU
// which loads this library holds until the process exits.  The caller passes
// only the system and the output, as for cn_solve_tridiag.
#include <cuda_runtime.h>

#include <cstdint>

#include "../../include/cn.h"
#include "cn_kernels.cuh"

using namespace cnb;

namespace {

constexpr int kNaBlock = 8;            // rows per block on every level
constexpr size_t kNaScratchBytes = 16u << 20;  // 16 MiB, enough for CN_NOALLOC_MAX_N rows
constexpr int kNaMaxLevels = CN_MAX_LEVELS;

}  // namespace

// The shared scratch.  In host code this name is only a host-side stand-in for
// the device array: its address must be looked up with cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNaScratchBytes];

namespace {

// Device address of g_noalloc_scratch on the current device.  Looked up on every
// call rather than cached: after a device reset (or any re-creation of the
// primary context) a cached address would be stale, and the lookup is cheap
// next to the solve's launches.
cudaError_t scratch_address(void** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

struct NaLevel {
    int64_t n, P;
    size_t rows, slot, x;  // byte offsets into the scratch
};

int64_t na_ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
size_t na_align(size_t v) { return (v + 255) & ~(size_t)255; }

// Level sizes and scratch offsets (host arithmetic only); returns the number of
// levels below level 0, or -1 if they do not fit.
int plan_levels(int64_t n, NaLevel* lv, size_t* used) {
    int L = 0;
    lv[0].n = n;
    lv[0].P = na_ceil_div(n - 1, kNaBlock);
    size_t off = 0;
    for (;;) {
        const int64_t nn = lv[L].P + 1;
        if (L + 1 >= kNaMaxLevels) return -1;
        NaLevel& nx = lv[L + 1];
        nx.n = nn;
        nx.P = nn <= kBaseMax ? 0 : na_ceil_div(nn - 1, kNaBlock);
        nx.rows = off;
        off = na_align(off + (size_t)nn * 4 * 16);
        nx.slot = off;
        off = na_align(off + (size_t)(na_ceil_div(lv[L].P, kThreads) + 1) * 3 * 16);
        nx.x = off;
        off = na_align(off + (size_t)nn * 16);
        ++L;
        if (nn <= kBaseMax) break;
    }
    *used = off;
    return L;
}

// The single system's entry at level l (offsets 0; every level in row order).
OneSys na_sys(const NaLevel* lv, int l) {
    OneSys s;
    s.e = LvlSys{};
    s.e.n = lv[l].n;
    s.e.P = lv[l].P;
    return s;
}

template <class R>
cudaError_t na_solve(unsigned char* base, const NaLevel* lv, int L, const ArraySource& src, double2* x,
                     cudaStream_t st) {
    typedef typename Store<R>::T ST;
    auto planes = [&](int l) { return LevelPlanes<R>{reinterpret_cast<ST*>(base + lv[l].rows), lv[l].n}; };
    auto slot = [&](int l) { return reinterpret_cast<LevelSlot<R>*>(base + lv[l].slot); };
    auto xs = [&](int l) { return reinterpret_cast<ST*>(base + lv[l].x); };
    auto lsrc = [&](int l) {
        const LevelPlanes<R> pl = planes(l);
        LevelSource<R> s;
        s.b = pl.p;
        s.L = pl.L;
        s.slot = slot(l);
        s.n = lv[l].n;
        s.prod = 0;
        s.stride = 0;
        s.slot_shift = 7;  // k_reduce: one slot per kThreads blocks
        return s;
    };
    auto grid = [&](int l) { return (unsigned)na_ceil_div(lv[l].P, kThreads); };
    const size_t smem = 2 * (size_t)kNaBlock * kThreads * 16;  // 32 KiB: below the default limit
    k_reduce<R, ArraySource, OneSys><<<grid(0), kThreads, 0, st>>>(src, na_sys(lv, 0), na_sys(lv, 1), kNaBlock,
                                                                   kNaBlock, planes(1), slot(1), nullptr);
    for (int l = 1; l < L; ++l)
        k_reduce<R, LevelSource<R>, OneSys><<<grid(l), kThreads, 0, st>>>(lsrc(l), na_sys(lv, l), na_sys(lv, l + 1),
                                                                          kNaBlock, kNaBlock, planes(l + 1), slot(l + 1),
                                                                          nullptr);
    k_base<R><<<1, 32, 0, st>>>(lsrc(L), xs(L), nullptr);
    // levels >= 1 substitute from the RD results their reductions kept in place
    for (int l = L - 1; l >= 1; --l)
        k_substitute_rd<R, OneSys><<<grid(l), kThreads, 0, st>>>(lsrc(l), na_sys(lv, l), na_sys(lv, l + 1),
                                                                  kNaBlock, xs(l + 1), xs(l));
    k_substitute<R, ArraySource, OneSys, double2><<<grid(0), kThreads, smem, st>>>(
        src, na_sys(lv, 0), na_sys(lv, 1), kNaBlock, xs(1), x, nullptr);
    return cudaGetLastError();
}

}  // namespace

// Debug build: the violation record of this translation unit's bounds checks
// (cn_debug.cuh), read and cleared by cn_debug_report.
namespace cnb_noalloc_debug {
int read_and_clear(unsigned long long* addr, unsigned long long* bytes) {
#if defined(CN_DEBUG)
    int flag = 0;
    if (cudaMemcpyFromSymbol(&flag, g_dbg_flag, sizeof(int)) != cudaSuccess || !flag) return 0;
    cudaMemcpyFromSymbol(addr, g_dbg_addr, sizeof(*addr));
    cudaMemcpyFromSymbol(bytes, g_dbg_bytes, sizeof(*bytes));
    const int z = 0;
    cudaMemcpyToSymbol(g_dbg_flag, &z, sizeof(int));
    return 1;
#else
    (void)addr;
    (void)bytes;
    return 0;
#endif
}
}  // namespace cnb_noalloc_debug

extern "C" cn_status cn_solve_tridiag_noalloc(const void* b, const void* a, const void* c, const void* d, void* x,
                                              int64_t n, int32_t arith, void* stream) {
    if (!b || !a || !c || !d || !x || n < 3) return CN_ERR_INVALID_ARG;
    if (arith != CN_ARITH_F64 && arith != CN_ARITH_DF64) return CN_ERR_INVALID_ARG;
    const uintptr_t mis = reinterpret_cast<uintptr_t>(b) | reinterpret_cast<uintptr_t>(a) |
                          reinterpret_cast<uintptr_t>(c) | reinterpret_cast<uintptr_t>(d) |
                          reinterpret_cast<uintptr_t>(x);
    if (mis & 15u) return CN_ERR_INVALID_ARG;
    if (x == b || x == a || x == c) return CN_ERR_INVALID_ARG;
    if (n > CN_NOALLOC_MAX_N) return CN_ERR_UNSUPPORTED;
    NaLevel lv[kNaMaxLevels];
    size_t used = 0;
    const int L = plan_levels(n, lv, &used);
    if (L < 1 || used > kNaScratchBytes) return CN_ERR_UNSUPPORTED;
    void* base = nullptr;
    if (scratch_address(&base) != cudaSuccess) return CN_ERR_CUDA;
    ArraySource s;
    s.b = static_cast<const double2*>(b);
    s.a = static_cast<const double2*>(a);
    s.c = static_cast<const double2*>(c);
    s.d = static_cast<const double2*>(d);
    s.n = n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* p = static_cast<unsigned char*>(base);
#if defined(CN_DEBUG)
    {
        const size_t vb = sizeof(double2) * (size_t)n;
        const void* ptrs[6] = {b, a, c, d, x, base};
        const size_t sizes[6] = {vb, vb, vb, vb, vb, kNaScratchBytes};
        DbgRange r[6];
        for (int i = 0; i < 6; ++i) {
            r[i].lo = (unsigned long long)reinterpret_cast<uintptr_t>(ptrs[i]);
            r[i].hi = r[i].lo + sizes[i];
        }
        const int nr = 6;
        if (cudaMemcpyToSymbolAsync(g_dbg_ranges, r, sizeof(r), 0, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyToSymbolAsync(g_dbg_nranges, &nr, sizeof(int), 0, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return CN_ERR_CUDA;
    }
#endif
    cudaError_t e = (arith == CN_ARITH_DF64) ? na_solve<df>(p, lv, L, s, static_cast<double2*>(x), st)
                                             : na_solve<double>(p, lv, L, s, static_cast<double2*>(x), st);
    return e == cudaSuccess ? CN_OK : CN_ERR_CUDA;
}
