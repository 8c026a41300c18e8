// cn_api.cu -- C ABI (include/cn.h): plans and batches, argument validation, and
// the launch sequence of the nested N-shaped solve (Eq. iteration of the paper).
//
// A plan is a batch of one system.  Both hold an Engine: the level hierarchy of
// every system (rows, blocks and offsets per level), the reduced-system storage
// of all levels, and the CN parameters.  One launch per stage and level serves
// all systems of a batch; a plan passes its single system's entries by value.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <initializer_list>
#include <map>
#include <mutex>
#include <type_traits>
#include <utility>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cn.h"
#include "cn_kernels.cuh"
#include "cn_scan.cuh"

using namespace cnb;

namespace {

constexpr int kDefaultLevelBlock = 8;  // rows per block on the reduced levels (>= 1)
constexpr int kDefaultBlock = 8;       // rows per level-0 block unless the descriptor says otherwise
constexpr int kMaxBlockRows = 32;      // shared memory of the substitution: 2 x 32 x 128 x 16 B
constexpr size_t kCplx = 16;           // bytes per complex in either compute type
constexpr int64_t kMaxBatch = 1 << 24;

struct LevelData {
    int m = 0;                // rows per block at this level
    int64_t total = 0;        // blocks of all systems (sum of P)
    int64_t rows_total = 0;   // rows of all systems present at this level
    std::vector<LvlSys> sys;  // one entry per system
    LvlSys* d_sys = nullptr;  // device copy (batches)
    int64_t L = 0;            // entries per plane (levels >= 1): sum of the systems' slots
    void* rows = nullptr;     // planes b, a, c, d of L entries each (levels >= 1)
    void* slot = nullptr;     // LevelSlot<R>[exchange units of the level below + 1]
    int slot_shift = 7;       // log2 blocks per exchange unit of the producer: 7 (a CTA), 5 (a warp)
    void* x = nullptr;        // Store<R>::T[rows_total]: solution (levels >= 1)
};

}  // namespace

struct Engine {
    cn_desc desc;                 // desc.n: rows of all systems
    int device = 0;
    int sms = 0;                  // multiprocessors of the device
    bool pdl = true;              // launch with programmatic stream serialization
    bool batched = false;
    bool scan0 = false;           // level 0 by one CTA per block (cn_scan.cuh): few long blocks
    int nsys = 0;
    std::vector<LevelData> lv;    // lv[0]: the systems themselves
    std::vector<int> base_level;  // per system: the level the RS stage solves
    std::vector<int> lvl_m;       // explicit block size per reduced level (cn_plan_create_levels), else empty
    void* zc = nullptr;           // substitution scratch for blocks longer than kSmemRowsMax
    void* base_cs = nullptr;      // serial RS scratch for a last level longer than kBaseMax
    void* d_base = nullptr;       // BaseSys<R>[nsys] (batches)
    std::vector<SysGrid> grid;    // per system
    SysGrid* d_grid = nullptr;    // device copy (batches)
    double2* state = nullptr;     // ping-pong state (recompute mode)
    void* keep = nullptr;         // 2 m entries per level-0 block: d^ and pivot (store mode)
    void* tab = nullptr;          // coefficient table (CoefTab<R>::T per row) or NULL
    int* status = nullptr;        // device status word
    CNParams cnp;
    std::vector<double> cos_a;    // n_cos coefficients per system
    // cn_step_host staging (allocated on first use)
    double2* h_in = nullptr;
    double2* h_out = nullptr;
    double* h_E = nullptr;
    int64_t h_E_cap = 0;
    // adjoint (allocated on first use)
    double2* mu = nullptr;
    void* part = nullptr;
    unsigned int* ticket = nullptr;  // inside the part allocation
    int part_n = 0;
    // kernel timing (cn_plan_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;  // events owned by the engine
    size_t ev_used = 0;                // events handed out since the last read
    std::vector<int> rec_class;        // class of record r (events 2r, 2r+1)
    int64_t workspace_bytes = 0;
    // slab of a sharded grid (cn_slab_create): the hierarchy is nested down to the
    // slab's two edge rows; rows slab_lo .. slab_hi of the global grid
    bool slab = false;
    bool own_last = true;           // the slab holds the global grid's last row
    int nslabs = 1, slab_rank = 0;
    int64_t slab_lo = 0, slab_hi = 0;
    double2* joint_work = nullptr;  // 2 (nslabs + 1): forward-sweep scratch, then the joint values
    // levels >= 1 in one persistent cooperative launch (k_levels)
    bool persistent = false;
    unsigned int* pbar = nullptr;   // grid barrier words {arrivals, generation}
    int p_grid = 0;                 // CTAs of the launch (all resident)
    size_t p_smem = 0;              // dynamic shared memory of the launch
    long long wait_ns = 2000000000ll;  // a grid barrier gives up after this long
    unsigned int wait_missing = 0;  // test hook: CTAs a barrier waits for beyond the grid
};

struct cn_plan_s : Engine {};
struct cn_batch_s : Engine {};

namespace {

// The last CUDA runtime error a call of this thread turned into CN_ERR_CUDA or
// CN_ERR_OOM (cn_cuda_error_string).
thread_local cudaError_t t_last_cuda_error = cudaSuccess;

cn_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return CN_OK;
    t_last_cuda_error = e;
    return CN_ERR_CUDA;
}
cn_status alloc_status(cudaError_t e) {
    cudaGetLastError();
    t_last_cuda_error = e;
    return e == cudaErrorMemoryAllocation ? CN_ERR_OOM : CN_ERR_CUDA;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }
bool aligned8(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 7u) == 0; }

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }
unsigned grid_for(int64_t P) { return (unsigned)ceil_div(P, kThreads); }

// need_n: a plan (one system of desc->n rows); a batch gives its sizes apart.
cn_status validate_desc(const cn_desc* d, bool need_n) {
    if (!d) return CN_ERR_INVALID_ARG;
    if (need_n && d->n < 3) return CN_ERR_INVALID_ARG;
    if (!(d->dx > 0.0) || !std::isfinite(d->dx)) return CN_ERR_INVALID_ARG;
    if (!std::isfinite(d->dt) || d->dt == 0.0 || !std::isfinite(d->x_min)) return CN_ERR_INVALID_ARG;
    if (d->pot < CN_POT_NONE || d->pot > CN_POT_COSSERIES) return CN_ERR_INVALID_ARG;
    if (d->pot == CN_POT_ARRAY && (!d->V0 || !aligned8(d->V0))) return CN_ERR_INVALID_ARG;
    if (d->pot == CN_POT_SOFTCOULOMB && !(d->soft_s > 0.0)) return CN_ERR_INVALID_ARG;
    if (d->pot == CN_POT_COSSERIES) {
        if (d->n_cos < 0 || d->n_cos > kMaxCos) return CN_ERR_INVALID_ARG;
        if (need_n && ((d->n_cos > 0 && !d->cos_a) || !(d->L > 0.0))) return CN_ERR_INVALID_ARG;
        if (!std::isfinite(d->L)) return CN_ERR_INVALID_ARG;
    }
    if (d->block != 0 && (d->block < 3 || d->block > kMaxBlockRows)) return CN_ERR_INVALID_ARG;
    if (d->level_block != 0 && (d->level_block < 3 || d->level_block > kMaxBlockRows)) return CN_ERR_INVALID_ARG;
    if (d->level1_block != 0 && (d->level1_block < 3 || d->level1_block > kMaxBlockRows)) return CN_ERR_INVALID_ARG;
    if (d->arith != CN_ARITH_F64 && d->arith != CN_ARITH_DF64) return CN_ERR_INVALID_ARG;
    if ((d->flags & ~(CN_FLAG_COEFF_TABLE | CN_FLAG_RECOMPUTE | CN_FLAG_LEVEL_LAUNCHES | CN_FLAG_PERSISTENT_LEVELS |
                      CN_FLAG_SERIAL_BLOCKS)) != 0)
        return CN_ERR_INVALID_ARG;
    if ((d->flags & CN_FLAG_LEVEL_LAUNCHES) && (d->flags & CN_FLAG_PERSISTENT_LEVELS)) return CN_ERR_INVALID_ARG;
    return CN_OK;
}

void free_engine(Engine* p) {
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    p->ev_pool.clear();
    for (LevelData& L : p->lv) {
        cudaFree(L.rows);
        cudaFree(L.slot);
        cudaFree(L.x);
        cudaFree(L.d_sys);
    }
    cudaFree(p->d_base);
    cudaFree(p->zc);
    cudaFree(p->base_cs);
    cudaFree(p->d_grid);
    cudaFree(p->state);
    cudaFree(p->keep);
    cudaFree(p->tab);
    cudaFree(p->status);
    cudaFree(p->h_in);
    cudaFree(p->h_out);
    cudaFree(p->h_E);
    cudaFree(p->mu);
    cudaFree(p->part);
    cudaFree(p->joint_work);
    cudaFree(p->pbar);
}

// Slots of level l (l >= 1): one per exchange unit of the level below, at the
// finest unit (a warp of 32 blocks; one block for a level produced by the scan
// kernels), plus one.
size_t slot_entries(const Engine* p, size_t l) {
    const int64_t units = p->lv[l].slot_shift == 0 ? p->lv[l - 1].total : ceil_div(p->lv[l - 1].total, 32);
    return (size_t)units + 1;
}

// Substitution scratch (two entries per row) for level-0 blocks longer than the
// shared-memory staging allows; the levels below substitute from their kept RD
// results and need none.
size_t zc_entries_of(const Engine* p) {
    return p->lv[0].m > kSmemRowsMax ? 2 * (size_t)p->lv[0].rows_total : 0;
}

// --------------------------------------------------------------- debug build: bounds registry
// Extents of the buffers a call may touch, installed in the kernels' range table
// (cn_debug.cuh) on the call's stream before its first launch.  No-ops in the
// default build.
// kept (d^, w) of level 0 (store mode), in entries: 2 m per block in chunks of 128
// blocks (one per CTA of the one-thread kernels' grid), or the scan kernels' 2 (m + nt)
// per block
size_t keep_entries(const Engine* p) {
    const LevelData& L0 = p->lv[0];
    if (p->scan0) return scan_keep_entries(L0.m, L0.total);
    return 2 * (size_t)L0.m * (size_t)grid_for(L0.total) * kThreads;
}
#if defined(CN_DEBUG)
struct DbgList {
    std::vector<std::pair<const void*, size_t>> v;
    void add(const void* p, size_t bytes) {
        if (p && bytes) v.push_back({p, bytes});
    }
};

size_t keep_bytes(const Engine* p) {
    return p->keep ? kCplx * keep_entries(p) : 0;
}

void dbg_engine(const Engine* p, DbgList& L) {
    const int64_t rows0 = p->lv[0].rows_total;
    L.add(p->keep, keep_bytes(p));
    L.add(p->state, kCplx * (size_t)rows0);
    L.add(p->tab, (p->desc.arith == CN_ARITH_DF64 ? sizeof(df) : sizeof(double2)) * (size_t)rows0);
    L.add(p->status, sizeof(int));
    for (size_t l = 1; l < p->lv.size(); ++l) {
        const LevelData& Lv = p->lv[l];
        L.add(Lv.rows, 4 * kCplx * (size_t)std::max<int64_t>(Lv.L, 1));
        L.add(Lv.slot, 3 * kCplx * slot_entries(p, l));
        L.add(Lv.x, kCplx * (size_t)Lv.rows_total);
    }
    for (const LevelData& Lv : p->lv) L.add(Lv.d_sys, sizeof(LvlSys) * (size_t)p->nsys);
    const size_t zc_entries = zc_entries_of(p);
    L.add(p->zc, kCplx * zc_entries);
    if (p->base_cs) L.add(p->base_cs, kCplx * (size_t)p->lv[(size_t)p->base_level[0]].sys[0].n);
    L.add(p->d_base, std::max(sizeof(BaseSys<double>), sizeof(BaseSys<df>)) * (size_t)p->nsys);
    L.add(p->d_grid, sizeof(SysGrid) * (size_t)p->nsys);
    L.add(p->mu, sizeof(double2) * (size_t)p->desc.n);
    L.add(p->part, 16 * (size_t)p->part_n + 16);
    L.add(p->h_in, sizeof(double2) * (size_t)p->desc.n);
    L.add(p->h_out, sizeof(double2) * (size_t)p->desc.n);
    L.add(p->h_E, sizeof(double) * (size_t)p->h_E_cap);
    L.add(p->joint_work, 2 * sizeof(double2) * ((size_t)p->nslabs + 1));
    L.add(p->pbar, 2 * sizeof(unsigned int));
    if (p->desc.pot == CN_POT_ARRAY) L.add(p->desc.V0, sizeof(double) * (size_t)rows0);
}

cudaError_t dbg_install(const DbgList& L, cudaStream_t st) {
    DbgRange r[kDbgMaxRanges];
    int n = 0;
    for (const auto& e : L.v) {
        if (n == kDbgMaxRanges) break;
        r[n].lo = (unsigned long long)reinterpret_cast<uintptr_t>(e.first);
        r[n].hi = r[n].lo + (unsigned long long)e.second;
        ++n;
    }
    cudaError_t e = n ? cudaMemcpyToSymbolAsync(g_dbg_ranges, r, sizeof(DbgRange) * (size_t)n, 0,
                                                cudaMemcpyHostToDevice, st)
                      : cudaSuccess;
    if (e == cudaSuccess) e = cudaMemcpyToSymbolAsync(g_dbg_nranges, &n, sizeof(int), 0, cudaMemcpyHostToDevice, st);
    return e;
}
#endif

cudaError_t dbg_register(const Engine* p, cudaStream_t st, std::initializer_list<std::pair<const void*, size_t>> extra) {
#if defined(CN_DEBUG)
    DbgList L;
    if (p) dbg_engine(p, L);
    for (const auto& e : extra) L.add(e.first, e.second);
    return dbg_install(L, st);
#else
    (void)p;
    (void)st;
    (void)extra;
    return cudaSuccess;
#endif
}

// --------------------------------------------------------------- kernel timing
enum { kProfReduce0 = 0, kProfSubst0 = 1, kProfReduceL = 2, kProfSubstL = 3, kProfBase = 4, kProfFused0 = 5,
       kProfLevels = 6 };

// Two events per record; the pool grows on demand and is reused after a read.
bool reserve_events(Engine* p, size_t k) {
    while (p->ev_pool.size() < p->ev_used + k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        p->ev_pool.push_back(e);
    }
    return true;
}

struct ProfScope {
    Engine* p;
    cudaStream_t st;
    cudaEvent_t stop = nullptr;
    ProfScope(Engine* p_, int cls, cudaStream_t st_) : p(p_), st(st_) {
        if (!p->profiling || !reserve_events(p, 2)) return;
        cudaEvent_t start = p->ev_pool[p->ev_used++];
        stop = p->ev_pool[p->ev_used++];
        p->rec_class.push_back(cls);
        cudaEventRecord(start, st);
    }
    ~ProfScope() {
        if (stop) cudaEventRecord(stop, st);
    }
};

// --------------------------------------------------------------- hierarchy
// Level l of system s has n rows cut into P = ceil((n-1)/m) blocks; its P + 1
// joint lines are the rows of level l + 1, until a level has <= kCrMax rows,
// which the RS stage solves in one CTA by cyclic reduction (explicit-depth plans: exactly
// the requested levels, then the serial RS).  Systems that reached their RS
// level have no rows below it.
cudaError_t build_hierarchy(Engine* p, const std::vector<int64_t>& sizes) {
    const int ns = (int)sizes.size();
    p->nsys = ns;
    p->base_level.assign(ns, -1);
    {
        LevelData L0;
        L0.m = p->lvl_m.empty() ? p->desc.block : p->lvl_m[0];
        L0.sys.resize(ns);
        int64_t roff = 0, boff = 0;
        for (int s = 0; s < ns; ++s) {
            LvlSys& e = L0.sys[s];
            e = LvlSys{};
            e.n = sizes[s];
            e.P = ceil_div(e.n - 1, L0.m);
            e.row_off = roff;
            e.blk_off = boff;
            roff += e.n;
            boff += e.P;
        }
        L0.rows_total = roff;
        L0.total = boff;
        p->lv.push_back(std::move(L0));
    }
    const int nlev = (int)p->lvl_m.size();
    for (;;) {
        const int l = (int)p->lv.size();
        if (l >= CN_MAX_LEVELS) return cudaErrorInvalidValue;
        LevelData L;
        L.m = nlev ? (l < nlev ? p->lvl_m[(size_t)l] : 0)
                   : ((l == 1 && p->desc.level1_block) ? p->desc.level1_block : p->desc.level_block);
        L.sys.resize(ns);
        int64_t roff = 0, boff = 0, soff = 0;
        for (int s = 0; s < ns; ++s) {
            LvlSys& e = L.sys[s];
            const LvlSys& q = p->lv[(size_t)l - 1].sys[s];
            e = LvlSys{};
            e.n = q.P > 0 ? q.P + 1 : 0;
            e.P = 0;
            if (e.n > 0) {
                // explicit depth: reduce exactly nlev levels; a slab: down to its two edge
                // rows; else until the CR stage can take it
                const bool base = p->slab ? (e.n == 2) : nlev ? (l == nlev) : (e.n <= kCrMax);
                if (base) p->base_level[s] = l;
                else if (e.n < 3) return cudaErrorInvalidValue;  // too short to cut into blocks
                else e.P = ceil_div(e.n - 1, L.m);
            }
            e.row_off = roff;
            e.blk_off = boff;
            e.prod_blk_off = q.blk_off;
            // plane layout for the kernels that read this level (see LvlSys)
            e.slot_off = soff;
            if (e.P > 0) {
                e.stride = e.P + 1;
                const int64_t excess = e.n - 1 - 2 * e.P;
                e.tc = excess > 0 ? ceil_div(excess, L.m - 2) : 0;
                e.Jtc = joint_line(e.tc, e.P, L.m, e.n);
                soff += (int64_t)L.m * (e.P + 1);
            } else {
                soff += e.n;
            }
            roff += e.n;
            boff += e.P;
        }
        L.rows_total = roff;
        L.total = boff;
        L.L = soff;
        p->lv.push_back(std::move(L));
        if (boff == 0) break;
    }
    // few long level-0 blocks of one system (store mode): one CTA per block, the
    // recurrences as prefix scans (cn_scan.cuh); level 1 then takes one slot per block
    p->scan0 = !p->batched && !p->slab && !(p->desc.flags & (CN_FLAG_RECOMPUTE | CN_FLAG_SERIAL_BLOCKS)) &&
               p->lv.size() >= 2 &&
               p->lv[0].m >= kScanMinRows && p->lv[0].m <= kScanMaxRows && p->lv[0].total <= kScanMaxBlocks;
    if (p->scan0) p->lv[1].slot_shift = 0;
    cudaError_t e = cudaSuccess;
    for (size_t l = 1; l < p->lv.size() && e == cudaSuccess; ++l) {
        LevelData& L = p->lv[l];
        const size_t nslot = slot_entries(p, l);
        p->workspace_bytes += (int64_t)(4 * kCplx * L.L + kCplx * L.rows_total + 3 * kCplx * nslot);
        e = cudaMalloc(&L.rows, 4 * kCplx * (size_t)std::max<int64_t>(L.L, 1));
        if (e == cudaSuccess) e = cudaMalloc(&L.slot, 3 * kCplx * nslot);
        if (e == cudaSuccess) e = cudaMalloc(&L.x, kCplx * (size_t)L.rows_total);
        if (e == cudaSuccess) e = cudaMemset(L.slot, 0, 3 * kCplx * nslot);
    }
    // long blocks (substitution scratch, two entries per row) and a long last level (serial RS)
    const size_t zc_entries = zc_entries_of(p);
    if (e == cudaSuccess && zc_entries) {
        p->workspace_bytes += (int64_t)(kCplx * zc_entries);
        e = cudaMalloc(&p->zc, kCplx * zc_entries);
    }
    if (e == cudaSuccess && !p->batched && !p->lvl_m.empty()) {
        const int64_t nb = p->lv[(size_t)p->base_level[0]].sys[0].n;
        if (nb > kBaseMax) {
            p->workspace_bytes += (int64_t)(kCplx * (size_t)nb);
            e = cudaMalloc(&p->base_cs, kCplx * (size_t)nb);
        }
    }
    if (e == cudaSuccess && p->batched) {
        for (LevelData& L : p->lv) {
            p->workspace_bytes += (int64_t)(sizeof(LvlSys) * (size_t)ns);
            e = cudaMalloc(&L.d_sys, sizeof(LvlSys) * (size_t)ns);
            if (e == cudaSuccess)
                e = cudaMemcpy(L.d_sys, L.sys.data(), sizeof(LvlSys) * (size_t)ns, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) break;
        }
    }
    return e;
}

template <class R> LevelPlanes<R> planes_of(const LevelData& L) {
    return LevelPlanes<R>{static_cast<typename Store<R>::T*>(L.rows), L.L};
}
template <class R> LevelSlot<R>* slot_of(const LevelData& L) { return static_cast<LevelSlot<R>*>(L.slot); }
template <class R> typename Store<R>::T* x_of(const LevelData& L) { return static_cast<typename Store<R>::T*>(L.x); }

template <class R> LevelSource<R> level_source(const LevelData& L) {
    const LevelPlanes<R> pl = planes_of<R>(L);
    LevelSource<R> s;
    s.b = pl.p;
    s.L = pl.L;
    s.slot = slot_of<R>(L);
    s.n = 0;
    s.prod = 0;
    s.stride = 0;
    s.slot_shift = L.slot_shift;
    return s;
}

// Per-system RS inputs of a batch, on the device.
template <class R>
cudaError_t build_base_table(Engine* p) {
    std::vector<BaseSys<R>> tb((size_t)p->nsys);
    for (int s = 0; s < p->nsys; ++s) {
        const LevelData& L = p->lv[(size_t)p->base_level[s]];
        tb[s].src = level_source<R>(L).bind(L.sys[s]);
        tb[s].x = x_of<R>(L) + L.sys[s].row_off;
    }
    p->workspace_bytes += (int64_t)(sizeof(BaseSys<R>) * tb.size());
    cudaError_t e = cudaMalloc(&p->d_base, sizeof(BaseSys<R>) * tb.size());
    if (e == cudaSuccess) e = cudaMemcpy(p->d_base, tb.data(), sizeof(BaseSys<R>) * tb.size(), cudaMemcpyHostToDevice);
    return e;
}

// Calls f(map of level l, map of level l + 1).
template <class F>
void with_maps(const Engine* p, size_t l, F f) {
    const LevelData& L = p->lv[l];
    const LevelData& N = p->lv[std::min(l + 1, p->lv.size() - 1)];
    if (p->batched) f(ManySys{L.d_sys, p->nsys, L.total}, ManySys{N.d_sys, p->nsys, N.total});
    else f(OneSys{L.sys[0]}, OneSys{N.sys[0]});
}

// Calls f(map of level 0, map of level 1, per-system grids).
template <class F>
void with_maps_grid(const Engine* p, F f) {
    const LevelData& L = p->lv[0];
    const LevelData& N = p->lv[1];
    if (p->batched) f(ManySys{L.d_sys, p->nsys, L.total}, ManySys{N.d_sys, p->nsys, N.total}, ManyGrid{p->d_grid});
    else f(OneSys{L.sys[0]}, OneSys{N.sys[0]}, OneGrid{p->grid[0]});
}

// --------------------------------------------------------------- launches
// Launches a kernel of the solve and step paths.  pdl (a single system's plan
// outside the adjoint step, Engine::pdl): programmatic stream serialization, so the
// kernel may be scheduled while the previous kernel in the stream still runs; it
// waits on the device (grid_dep_enter) for that kernel's results before touching
// memory.  Otherwise an ordinary stream-ordered launch.
template <class... KArgs, class... Args>
cudaError_t launch(bool pdl, void (*kernel)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                   Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = pdl ? 1 : 0;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Shared memory of the substitutions: two complex values per block row and thread.
size_t subst_smem(int m) { return 2 * (size_t)m * kThreads * kCplx; }
size_t kept_smem(int m) { return (size_t)m * kTileStride * kCplx; }
size_t fused_smem(int m) { return (size_t)(m + 2) * kTileStride * kCplx; }  // rows 0..g+1 per column
size_t cr_smem() { return 6 * (size_t)kCrMax * kCplx; }
size_t ws_reduce_smem(int m) { return ws_reduce_entries(m) * kCplx; }

// In per-level launches the two-group reduction takes the levels below level 1
// that need at most one CTA of kThreads blocks per multiprocessor, with blocks of
// at most kWsRowsMax rows.  (Level 1 stays on the one-thread-per-block kernel:
// where it qualifies, at n = 2^20, the two-group kernels there made the step 5 %
// slower on B300, while levels 2 and 3 at n = 2^24 gained 1.3 % of the step.)
bool two_group_level(const Engine* p, size_t l) {
    const LevelData& L = p->lv[l];
    return l >= 2 && L.m <= kWsRowsMax && L.total > 0 && (int64_t)grid_for(L.total) <= (int64_t)p->sms;
}

template <class R, class Src, class Map>
cudaError_t launch_reduce(bool pdl, const Src& src, Map sys, Map next, int m, const LevelData& nextL, int* status,
                          int64_t total, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    return launch(pdl, k_reduce<R, Src, Map>, grid_for(total), kThreads, 0, st, src, sys, next, m, nextL.m,
                  planes_of<R>(nextL), slot_of<R>(nextL), status);
}

template <class R, class Src, class Map, class XT>
cudaError_t launch_substitute(bool pdl, const Src& src, Map sys, Map next, int m, const LevelData& nextL, XT* x,
                              int* status, int64_t total, void* zc, cudaStream_t st) {
    if (total == 0) return cudaSuccess;
    if constexpr (Src::kKeepsRD)  // a reduced level: the RD results are in its planes
        return launch(pdl, k_substitute_rd<R, Map>, grid_for(total), kThreads, 0, st, src, sys, next, m,
                      x_of<R>(nextL), x);
    if (m > kSmemRowsMax)
        return launch(pdl, k_substitute_gmem<R, Src, Map, XT>, grid_for(total), kThreads, 0, st, src, sys, next, m,
                      x_of<R>(nextL), x, static_cast<typename Store<R>::T*>(zc), status);
    return launch(pdl, k_substitute<R, Src, Map, XT>, grid_for(total), kThreads, subst_smem(m), st, src, sys, next, m,
                  x_of<R>(nextL), x, status);
}

// Opt the substitution kernels into the dynamic shared memory their largest block needs.
// A kernel's dynamic shared memory limit is a property of the function for the
// whole process (per device), shared by every plan: a plan may only raise it,
// never lower it below what another live plan launches with.  The largest value
// requested so far is kept per (device, kernel) and set again on every request
// (so a device reset, which clears the attribute, is repaired by the next plan).
std::mutex g_smem_mutex;
std::map<std::pair<int, const void*>, int> g_smem_max;

template <class... KArgs>
cudaError_t raise_smem_limit(void (*kernel)(KArgs...), size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    int& cur = g_smem_max[{dev, reinterpret_cast<const void*>(kernel)}];
    cur = std::max(cur, (int)bytes);
    return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cur);
}

template <class R, class Map, class Grid>
cudaError_t set_smem_limits_map(int m0) {
    cudaError_t e = raise_smem_limit(k_substitute<R, ArraySource, Map, double2>, subst_smem(m0));
    if (e == cudaSuccess) e = raise_smem_limit(k_cn_substitute<R, -1, Map, Grid>, subst_smem(m0));
    if (e == cudaSuccess) e = raise_smem_limit(k_cn_substitute<R, 0, Map, Grid>, subst_smem(m0));
    if (e == cudaSuccess) e = raise_smem_limit(k_cn_substitute_kept<R, Map>, kept_smem(m0));
    if (e == cudaSuccess) e = raise_smem_limit(k_cn_fused<R, -1, Map, Grid, false>, fused_smem(m0));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cn_fused<R, -1, Map, Grid, false>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 (int)cudaSharedmemCarveoutMaxShared);
    if (e == cudaSuccess) e = raise_smem_limit(k_cn_fused<R, -1, Map, Grid, true>, fused_smem(m0));
    if (e == cudaSuccess) e = raise_smem_limit(k_base_cr<R>, cr_smem());
    if (e == cudaSuccess) e = raise_smem_limit(k_base_cr_many<R>, cr_smem());
    if (e == cudaSuccess) e = raise_smem_limit(k_reduce_ws<R, Map>, ws_reduce_smem(kWsRowsMax));
    return e;
}

template <class R>
cudaError_t set_scan_smem_limits(int m0) {
    cudaError_t e = raise_smem_limit(k_cn_reduce_scan<R, -1>, scan_reduce_entries(m0) * kCplx);
    if (e == cudaSuccess && std::is_same<R, double>::value)
        e = raise_smem_limit(k_base_scan<R>, scan_rs_entries(kScanRsMax) * kCplx);
    if (e == cudaSuccess) e = raise_smem_limit(k_cn_reduce_scan<R, 0>, scan_reduce_entries(m0) * kCplx);
    if (e == cudaSuccess) e = raise_smem_limit(k_cn_substitute_scan<R>, scan_subst_entries(m0) * kCplx);
    return e;
}

template <class R>
cudaError_t set_smem_limits(const Engine* p) {
    // the largest staged level-0 block (longer blocks take the scratch variants;
    // the levels below substitute from their kept RD results, unstaged)
    const int m0 = std::min(p->lv[0].m, kSmemRowsMax);
    if (p->scan0) {
        cudaError_t e = set_scan_smem_limits<R>(p->lv[0].m);
        if (e != cudaSuccess) return e;
    }
    if (p->batched) return set_smem_limits_map<R, ManySys, ManyGrid>(m0);
    return set_smem_limits_map<R, OneSys, OneGrid>(m0);
}

// The persistent launch of the levels below level 0 (k_levels) serves a single
// system of the default hierarchy (reduced to <= 1024 rows, cyclic-reduction RS
// stage) unless CN_FLAG_LEVEL_LAUNCHES asks for one launch per stage and level:
// its shared memory holds the RS stage's arrays, one CTA per multiprocessor (512
// threads, <= 128 registers).
template <class R>
cudaError_t setup_persistent(Engine* p) {
    p->persistent = false;
    for (size_t l = 2; l < p->lv.size(); ++l) p->lv[l].slot_shift = 7;  // the per-level kernels' exchange unit
    // the default per arithmetic, from N = 2^24 measurements on B300: binary64
    // 1.402 (persistent) vs 1.422 ms per step (blocks 32 / 16 / 8), double-float
    // 0.459 vs 0.442 ms (blocks 13 / 10 / 8: the two-group kernels of levels 2
    // and 3 and the programmatic launch overlap outweigh the saved launches)
    const int fl = p->desc.flags;
    const bool want = (fl & CN_FLAG_PERSISTENT_LEVELS) ||
                      (!(fl & CN_FLAG_LEVEL_LAUNCHES) && p->desc.arith == CN_ARITH_F64);
    if (!want || p->batched || p->slab || !p->lvl_m.empty() || p->lv.size() < 3) return cudaSuccess;
    const size_t smem = cr_smem();
    cudaError_t e = raise_smem_limit(k_levels<R>, smem);
    int per_sm = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_levels<R>, kPThreads, smem);
    if (e != cudaSuccess || per_sm < 1) {
        cudaGetLastError();
        return cudaSuccess;  // not resident: keep the per-level launches
    }
    if (!p->pbar) {
        e = cudaMalloc(&p->pbar, 2 * sizeof(unsigned int));
        if (e == cudaSuccess) e = cudaMemset(p->pbar, 0, 2 * sizeof(unsigned int));
        if (e != cudaSuccess) return e;
        p->workspace_bytes += 2 * sizeof(unsigned int);
    }
    p->p_smem = smem;
    p->p_grid = per_sm * p->sms;
    p->persistent = true;
    // levels 2 .. L-1 are produced by k_levels' warp-unit reductions
    for (size_t l = 2; l < p->lv.size(); ++l) p->lv[l].slot_shift = 5;
    return cudaSuccess;
}

// Levels >= 1 of the nested solve: reductions down (reduce_levels), the RS
// stage (rs_stage), substitutions up (substitute_levels).
template <class R>
cudaError_t reduce_levels(Engine* p, cudaStream_t st) {
    const size_t L = p->lv.size();
    cudaError_t e = cudaSuccess;
    for (size_t l = 1; l + 1 < L && e == cudaSuccess; ++l) {
        ProfScope ps(p, kProfReduceL, st);
        with_maps(p, l, [&](auto a, auto b) {
            const LevelData& L = p->lv[l];
            const LevelData& N = p->lv[l + 1];
            if (two_group_level(p, l)) {
                e = launch(p->pdl, k_reduce_ws<R, decltype(a)>, kWsCluster * grid_for(L.total), 2 * kWsLanes,
                           ws_reduce_smem(L.m), st, level_source<R>(L), a, b, L.m, N.m, planes_of<R>(N),
                           slot_of<R>(N), p->status);
            } else {
                e = launch_reduce<R>(p->pdl, level_source<R>(L), a, b, L.m, N, p->status, L.total, st);
            }
        });
    }
    return e;
}

template <class R>
cudaError_t rs_stage(Engine* p, cudaStream_t st) {
    ProfScope ps(p, kProfBase, st);
    if (p->batched)
        return launch(p->pdl, k_base_cr_many<R>, (unsigned)p->nsys, kCrThreads, cr_smem(), st,
                      static_cast<const BaseSys<R>*>(p->d_base), p->status);
    const LevelData& B = p->lv[(size_t)p->base_level[0]];
    const LevelSource<R> src = level_source<R>(B).bind(B.sys[0]);
    if (p->lvl_m.empty())
        return launch(p->pdl, k_base_cr<R>, 1, kCrThreads, cr_smem(), st, src, x_of<R>(B), p->status);
    // a reduced system of at most 32 rows: parallel cyclic reduction on one warp (unless
    // the blocks are to be walked serially, the partition study's model)
    if (src.n <= kPcrMax && !(p->desc.flags & CN_FLAG_SERIAL_BLOCKS))
        return launch(p->pdl, k_base_pcr<R>, 1, 32, 0, st, src, x_of<R>(B), p->status);
    // level 0 by scans, binary64, 33 .. 512 rows (65 for 64-row blocks of n = 4096): the RS
    // stage by scans on one warp too (the paper's P = 16, 17 rows, before the above: 30 ->
    // 21 us on B300; in double-float the one-thread walk is the faster, 16 us)
    if (std::is_same<R, double>::value && p->scan0 && src.n <= kScanRsMax)
        return launch(p->pdl, k_base_scan<R>, 1, 32, scan_rs_entries((int)src.n) * kCplx, st, src, x_of<R>(B),
                      p->status);
    if (p->base_cs)
        return launch(p->pdl, k_base_serial<R>, 1, 32, 0, st, src, x_of<R>(B),
                      static_cast<typename Store<R>::T*>(p->base_cs), p->status);
    return launch(p->pdl, k_base<R>, 1, 32, 0, st, src, x_of<R>(B), p->status);
}

template <class R>
cudaError_t substitute_levels(Engine* p, cudaStream_t st) {
    const size_t L = p->lv.size();
    cudaError_t e = cudaSuccess;
    for (size_t l = L - 2; l >= 1 && e == cudaSuccess; --l) {
        ProfScope ps(p, kProfSubstL, st);
        with_maps(p, l, [&](auto a, auto b) {
            const LevelData& L = p->lv[l];
            const LevelData& N = p->lv[l + 1];
            e = launch_substitute<R>(p->pdl, level_source<R>(L), a, b, L.m, N, x_of<R>(L), p->status, L.total,
                                     p->zc, st);
        });
    }
    return e;
}

// All stages below level 0 in one cooperative launch of k_levels.
template <class R>
cudaError_t persistent_levels(Engine* p, cudaStream_t st) {
    ProfScope ps(p, kProfLevels, st);
    PLevels<R> a;
    std::memset(&a, 0, sizeof(a));
    const size_t L = p->lv.size();  // levels 0 .. L-1; L-1 is the RS level
    a.nl = (int)L - 2;
    for (int l = 1; l <= a.nl; ++l) {
        const LevelData& Lv = p->lv[(size_t)l];
        const LevelData& N = p->lv[(size_t)l + 1];
        PLevel<R>& q = a.lv[l - 1];
        q.src = level_source<R>(Lv);
        q.sys = OneSys{Lv.sys[0]};
        q.next = OneSys{N.sys[0]};
        q.m = Lv.m;
        q.m_next = N.m;
        q.out = planes_of<R>(N);
        q.out_slot = slot_of<R>(N);
        q.x = x_of<R>(Lv);
        q.x_next = x_of<R>(N);
        q.units = ceil_div(Lv.total, 32);
        // a level of at most one unit per CTA reduces on four warps a unit
        q.split4 = (Lv.m >= 2 && Lv.m <= kSplitRowsMax && q.units <= p->p_grid &&
                    split4_entries(Lv.m) * kCplx <= p->p_smem) ? 1 : 0;
    }
    const LevelData& B = p->lv[L - 1];
    a.base = level_source<R>(B).bind(B.sys[0]);
    a.base_x = x_of<R>(B);
    a.status = p->status;
    a.bar = p->pbar;
    a.expect = (unsigned)p->p_grid + p->wait_missing;
    a.timeout_ns = p->wait_ns;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)p->p_grid);
    cfg.blockDim = dim3(kPThreads);
    cfg.dynamicSmemBytes = p->p_smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_levels<R>, a);
}

template <class R>
cudaError_t solve_levels(Engine* p, cudaStream_t st) {
    if (p->persistent) return persistent_levels<R>(p, st);
    cudaError_t e = reduce_levels<R>(p, st);
    if (e == cudaSuccess) e = rs_stage<R>(p, st);
    if (e == cudaSuccess) e = substitute_levels<R>(p, st);
    return e;
}

// General tridiagonal solve (arrays at level 0, one system).
template <class R>
cudaError_t solve_arrays(Engine* p, const ArraySource& src, double2* x, cudaStream_t st) {
    // level 0 of arrays runs the one-thread kernels, which leave one JD slot per CTA
    // of kThreads blocks, also in a plan whose CN steps reduce level 0 by scans (one
    // slot per block): level 1 is read accordingly for this call
    struct SlotShift {
        int& v;
        const int old;
        SlotShift(int& r, int s) : v(r), old(r) { v = s; }
        ~SlotShift() { v = old; }
    } level1_slots(p->lv[1].slot_shift, 7);
    cudaError_t e = cudaSuccess;
    {
        ProfScope ps(p, kProfReduce0, st);
        with_maps(p, 0, [&](auto a, auto b) {
            e = launch_reduce<R>(p->pdl, src, a, b, p->lv[0].m, p->lv[1], p->status, p->lv[0].total, st);
        });
    }
    if (e != cudaSuccess) return e;
    if ((e = solve_levels<R>(p, st)) != cudaSuccess) return e;
    ProfScope ps(p, kProfSubst0, st);
    with_maps(p, 0, [&](auto a, auto b) {
        e = launch_substitute<R>(p->pdl, src, a, b, p->lv[0].m, p->lv[1], x, p->status, p->lv[0].total, p->zc, st);
    });
    return e;
}

// e s of a step as the kernels' template argument: -1 for the CN step (its
// right-hand side T^dagger psi), 0 for the adjoint's identity right-hand side.
template <class F>
cudaError_t with_es(const CNStep& s, F f) {
    switch (s.e * s.s) {
    case -1: return f(std::integral_constant<int, -1>());
    case 0: return f(std::integral_constant<int, 0>());
    default: return cudaErrorInvalidValue;
    }
}

template <class R>
cudaError_t cn_reduce0(Engine* p, const CNStep& s, cudaStream_t st) {
    typedef typename Store<R>::T ST;
    const LevelData& L0 = p->lv[0];
    const LevelData& L1 = p->lv[1];
    ProfScope ps(p, kProfReduce0, st);
    if (p->scan0)
        return with_es(s, [&](auto es) {
            return launch(p->pdl, k_cn_reduce_scan<R, decltype(es)::value>, (unsigned)L0.total,
                          (unsigned)scan_threads(L0.m),
                          scan_reduce_entries(L0.m) * kCplx, st, s, OneSys{L0.sys[0]}, OneSys{L1.sys[0]},
                          OneGrid{p->grid[0]}, L0.m, L1.m, planes_of<R>(L1), slot_of<R>(L1),
                          static_cast<ST*>(p->keep), p->status);
        });
    return with_es(s, [&](auto es) {
        cudaError_t e = cudaSuccess;
        with_maps_grid(p, [&](auto a, auto b, auto gr) {
            e = launch(p->pdl, k_cn_reduce<R, decltype(es)::value, decltype(a), decltype(gr)>, grid_for(L0.total),
                       kThreads, 0, st, s, a, b, gr, L0.m, L1.m, planes_of<R>(L1), slot_of<R>(L1),
                       static_cast<ST*>(p->keep), p->status);
        });
        return e;
    });
}

template <class R>
cudaError_t cn_subst0(Engine* p, const CNStep& s, double2* x, cudaStream_t st) {
    typedef typename Store<R>::T ST;
    const LevelData& L0 = p->lv[0];
    const LevelData& L1 = p->lv[1];
    const unsigned grid = grid_for(L0.total);
    ST* keep = static_cast<ST*>(p->keep);
    ProfScope ps(p, kProfSubst0, st);
    if (p->scan0)
        return launch(p->pdl, k_cn_substitute_scan<R>, (unsigned)L0.total, (unsigned)scan_threads(L0.m),
                      scan_subst_entries(L0.m) * kCplx, st,
                      OneSys{L0.sys[0]}, OneSys{L1.sys[0]}, L0.m, static_cast<const ST*>(keep),
                      static_cast<const ST*>(x_of<R>(L1)), x);
    return with_es(s, [&](auto es) {
        cudaError_t e = cudaSuccess;
        with_maps_grid(p, [&](auto a, auto b, auto gr) {
            typedef decltype(a) M;
            if (keep && L0.m > kSmemRowsMax)
                e = launch(p->pdl, k_cn_substitute_kept_gmem<R, M>, grid, kThreads, 0, st, a, b, L0.m,
                           static_cast<const ST*>(keep), static_cast<const ST*>(x_of<R>(L1)), x,
                           static_cast<ST*>(p->zc));
            else if (keep)
                e = launch(p->pdl, k_cn_substitute_kept<R, M>, grid, kThreads, kept_smem(L0.m), st, a, b, L0.m,
                           static_cast<const ST*>(keep), static_cast<const ST*>(x_of<R>(L1)), x, p->status);
            else
                e = launch(p->pdl, k_cn_substitute<R, decltype(es)::value, M, decltype(gr)>, grid, kThreads,
                           subst_smem(L0.m), st, s, a, b, gr, L0.m, static_cast<const ST*>(x_of<R>(L1)), x,
                           p->status);
        });
        return e;
    });
}

// SS of the previous step fused with the level-0 reduction of step s (store mode,
// CN steps: e s = -1); x_out != NULL also receives the previous step's result.
template <class R>
cudaError_t cn_fused0(Engine* p, const CNStep& s, double2* x_out, cudaStream_t st) {
    typedef typename Store<R>::T ST;
    const LevelData& L0 = p->lv[0];
    const LevelData& L1 = p->lv[1];
    if (s.e * s.s != -1) return cudaErrorInvalidValue;
    ProfScope ps(p, kProfFused0, st);
    cudaError_t e = cudaSuccess;
    with_maps_grid(p, [&](auto a, auto b, auto gr) {
        typedef decltype(a) M;
        typedef decltype(gr) G;
        auto kern = x_out ? k_cn_fused<R, -1, M, G, true> : k_cn_fused<R, -1, M, G, false>;
        e = launch(p->pdl, kern, grid_for(L0.total), kThreads, fused_smem(L0.m), st, s, a, b, gr, L0.m, L1.m,
                   static_cast<const ST*>(x_of<R>(L1)), planes_of<R>(L1), slot_of<R>(L1), static_cast<ST*>(p->keep),
                   x_out, p->status);
    });
    return e;
}

// One CN-type step of every system (level 0 generated on the fly), result in x.
template <class R>
cudaError_t cn_solve(Engine* p, const CNStep& s, double2* x, cudaStream_t st) {
    cudaError_t e = cn_reduce0<R>(p, s, st);
    if (e == cudaSuccess) e = solve_levels<R>(p, st);
    if (e == cudaSuccess) e = cn_subst0<R>(p, s, x, st);
    return e;
}

// Whether consecutive steps pass psi on chip (store mode with the block staged
// in shared memory): step k's substitution and step k + 1's level-0 reduction
// then run as one kernel, and only the last step writes psi.  In binary64 too:
// at N = 2^24 with blocks of 24 the fused kernel took 1.23 ms per step where the
// two level-0 kernels took 1.01 + 0.37 ms (the substitution's latency hides
// behind the reduction's FP64 work of the other warps).
bool fuses_steps(const Engine* p) { return p->keep != nullptr && p->lv[0].m <= kSmemRowsMax; }

// nsteps CN steps from in; the result goes to out, or with states != NULL every
// step's result to states + k rows (k = 0 .. nsteps-1; in must not lie in states).
template <class R>
cudaError_t cn_steps(Engine* p, const double2* in, double2* out, const double* E_mid, int64_t nsteps,
                     cudaStream_t st, double2* states = nullptr) {
    const int64_t rows = p->lv[0].rows_total;
    const size_t bytes = sizeof(double2) * (size_t)rows;
    if (nsteps == 0) {
        if (in == out || states) return cudaSuccess;
        return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
    }
    const bool kept = p->keep != nullptr;
    auto state_k = [&](int64_t k) { return states + k * rows; };
    if (states) out = state_k(nsteps - 1);
    auto step_k = [&](int64_t k, const double2* psi) {
        CNStep s;
        s.p = p->cnp;
        s.psi = psi;
        s.s = 1;
        s.e = -1;
        s.E = E_mid ? E_mid + k : nullptr;
        s.tab = p->tab;
        s.own_last = p->own_last ? 1 : 0;
        return s;
    };
    if (fuses_steps(p)) {
        // reduce(0), levels, [fused(k), levels] for k = 1..nsteps-1, SS(last) -> out;
        // in is read by the first reduction only, so in == out is fine
        cudaError_t e = cn_reduce0<R>(p, step_k(0, in), st);
        if (e == cudaSuccess) e = solve_levels<R>(p, st);
        for (int64_t k = 1; k < nsteps && e == cudaSuccess; ++k) {
            e = cn_fused0<R>(p, step_k(k, nullptr), states ? state_k(k - 1) : nullptr, st);
            if (e == cudaSuccess) e = solve_levels<R>(p, st);
        }
        if (e == cudaSuccess) e = cn_subst0<R>(p, step_k(nsteps - 1, nullptr), out, st);
        return e;
    }
    if (states) {  // every step writes its own state; recompute mode reads the previous one
        const double2* src = in;
        for (int64_t k = 0; k < nsteps; ++k) {
            cudaError_t e = cn_solve<R>(p, step_k(k, src), state_k(k), st);
            if (e != cudaSuccess) return e;
            src = state_k(k);
        }
        return cudaSuccess;
    }
    // Store mode: the substitution does not read psi, so every step after the
    // first updates out in place.  Recompute mode: step k writes dest(k), the
    // last step writes out, destinations alternate between out and the
    // scratch, and in is never written unless it is out.
    const double2* src = in;
    if (!kept && in == out && ((nsteps - 1) % 2) == 0) {
        cudaError_t e = cudaMemcpyAsync(p->state, in, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        src = p->state;
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        double2* dst = kept ? out : ((((nsteps - 1 - k) % 2) == 0) ? out : p->state);
        cudaError_t e = cn_solve<R>(p, step_k(k, src), dst, st);
        if (e != cudaSuccess) return e;
        src = dst;
    }
    return cudaSuccess;
}

// bytes per row of the coefficient table (CoefTab: bt0 in double-float, {bt0, x} in binary64)
size_t table_entry_size(int arith) { return arith == CN_ARITH_DF64 ? sizeof(df) : sizeof(double2); }

DFc split(double v) {
    df d = df_from_double(v);
    DFc r;
    r.hi = d.hi;
    r.lo = d.lo;
    return r;
}

SysGrid make_grid(double x_min, double dx, int64_t n) {
    SysGrid g;
    double jo = std::nearbyint(-x_min / dx);
    if (jo < 0) jo = 0;
    if (jo > (double)(n - 1)) jo = (double)(n - 1);
    g.j_o = (int64_t)jo;
    g.x_o = x_min + (double)g.j_o * dx;
    g.xo_f = split(g.x_o);
    return g;
}

// Common part of plan and batch creation: sizes and x_min per system, cos_a
// (n_cos per system, row-major) for CN_POT_COSSERIES with period desc->L if
// > 0, else the system's own length n_s dx.
cn_status create_engine(Engine* p, const cn_desc* desc, const std::vector<int64_t>& sizes,
                        const std::vector<double>& x_min, const double* cos_a, const SysGrid* grid0 = nullptr) {
    p->desc = *desc;
    if (p->desc.block == 0) p->desc.block = kDefaultBlock;
    if (p->desc.level_block == 0) p->desc.level_block = kDefaultLevelBlock;
    if (cudaGetDevice(&p->device) != cudaSuccess) return CN_ERR_CUDA;
    // A batch launches in plain stream order: its kernels are many CTAs deep, and
    // with programmatic launches the 4096-system workload measured 1 % slower on
    // B300 (4.025e10 vs 4.065e10 unknown-steps/s), the single systems 3 % faster.
    p->pdl = !p->batched;
    if (cudaDeviceGetAttribute(&p->sms, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) return CN_ERR_CUDA;
    const int ns = (int)sizes.size();
    const int ncos = desc->pot == CN_POT_COSSERIES ? desc->n_cos : 0;
    if (ncos > 0) p->cos_a.assign(cos_a, cos_a + (size_t)ncos * (size_t)ns);
    p->desc.cos_a = nullptr;
    const bool df_mode = desc->arith == CN_ARITH_DF64;
    // A batch always tabulates bt0 (one launch per system here, none per step).
    const bool use_table = (desc->flags & CN_FLAG_COEFF_TABLE) || p->batched ||
                           (df_mode && (desc->pot == CN_POT_ARRAY || desc->pot == CN_POT_COSSERIES));
    const bool recompute = (desc->flags & CN_FLAG_RECOMPUTE) != 0;
    if (recompute && !p->lvl_m.empty() && p->lvl_m[0] > kSmemRowsMax) return CN_ERR_UNSUPPORTED;

    cudaError_t e = build_hierarchy(p, sizes);
    if (e == cudaErrorInvalidValue) return p->lvl_m.empty() ? CN_ERR_UNSUPPORTED : CN_ERR_INVALID_ARG;
    if (e != cudaSuccess) return alloc_status(e);
    const int64_t rows0 = p->lv[0].rows_total;
    const size_t kept = keep_entries(p);
    p->workspace_bytes += (int64_t)(recompute ? kCplx * rows0 : kCplx * kept) + (int64_t)sizeof(int);
    if (recompute) e = cudaMalloc(&p->state, kCplx * (size_t)rows0);
    else e = cudaMalloc(&p->keep, kCplx * kept);
    if (e == cudaSuccess) e = cudaMalloc(&p->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(int));
    if (e == cudaSuccess && use_table) {
        p->workspace_bytes += (int64_t)(table_entry_size(desc->arith) * (size_t)rows0);
        e = cudaMalloc(&p->tab, table_entry_size(desc->arith) * (size_t)rows0);
    }
    p->grid.resize(ns);
    for (int s = 0; s < ns; ++s) p->grid[s] = make_grid(x_min[s], desc->dx, sizes[s]);
    if (grid0) p->grid[0] = *grid0;  // a slab: the global grid's coordinates, shifted
    if (e == cudaSuccess && p->batched) {
        p->workspace_bytes += (int64_t)(sizeof(SysGrid) * (size_t)ns);
        e = cudaMalloc(&p->d_grid, sizeof(SysGrid) * (size_t)ns);
        if (e == cudaSuccess)
            e = cudaMemcpy(p->d_grid, p->grid.data(), sizeof(SysGrid) * (size_t)ns, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = df_mode ? build_base_table<df>(p) : build_base_table<double>(p);
    }
    if (e != cudaSuccess) return alloc_status(e);

    CNParams& c = p->cnp;
    std::memset(&c, 0, sizeof(c));
    c.dx = desc->dx;
    c.c1 = 2.0 * desc->dx * desc->dx;
    c.gt = 4.0 * desc->dx * desc->dx / desc->dt;
    c.pot = desc->pot;
    c.V0 = desc->V0;
    c.soft_s = desc->soft_s;
    c.n_cos = ncos;
    c.dx_f = split(c.dx);
    c.c1_f = split(c.c1);
    c.gt_f = split(c.gt);
    c.soft_f = split(c.soft_s);
    // the explicit row on the integer pipe where level 0 fills the GPU (two or more CTAs
    // of kThreads blocks per SM): the FP64 pipe bounds such steps (N = 2^24: 1.299 ->
    // 1.260 ms with its additions there, 1.226 with its inner FMAs too), while a
    // latency-bound small grid only gets longer threads (n = 4096: 43 -> 46 us).  A batch
    // keeps its inner FMAs on the FP64 pipe: its level-0 kernels run four CTAs per SM,
    // and the integer FMAs cost it 10 % (1.39e10 -> 1.26e10 unknown-steps/s)
    const bool fills = p->lv[0].total >= 2 * (int64_t)p->sms * kThreads;
    c.sigma_int = !fills ? 0 : (p->batched ? 1 : 2);
    const double two_pi = 2.0 * 3.14159265358979323846;
    if (use_table && e == cudaSuccess) e = dbg_register(p, nullptr, {});
    if (use_table) {
        // static part of the diagonal, one system at a time (once per plan or batch)
        for (int s = 0; s < ns && e == cudaSuccess; ++s) {
            CNParams cs = c;
            const int64_t ro = p->lv[0].sys[s].row_off;
            if (desc->pot == CN_POT_ARRAY) cs.V0 = desc->V0 + ro;
            if (ncos > 0) {
                const double L = desc->L > 0.0 ? desc->L : (double)sizes[s] * desc->dx;
                cs.two_pi_over_L = two_pi / L;
                for (int k = 0; k < ncos; ++k) cs.cos_a[k] = p->cos_a[(size_t)s * ncos + k];
            }
            const unsigned g = (unsigned)ceil_div(sizes[s], 256);
            if (df_mode) k_beta0_table<df><<<g, 256>>>(cs, p->grid[s], sizes[s], static_cast<df*>(p->tab) + ro);
            else k_beta0_table<double><<<g, 256>>>(cs, p->grid[s], sizes[s], static_cast<double2*>(p->tab) + ro);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    } else if (ncos > 0) {
        c.two_pi_over_L = two_pi / desc->L;
        for (int k = 0; k < ncos; ++k) c.cos_a[k] = p->cos_a[(size_t)k];
    }
    if (e == cudaSuccess) e = df_mode ? set_smem_limits<df>(p) : set_smem_limits<double>(p);
    if (e == cudaSuccess) e = df_mode ? setup_persistent<df>(p) : setup_persistent<double>(p);
    if (e != cudaSuccess) return alloc_status(e);
    return CN_OK;
}

cn_status run_steps(Engine* p, const void* psi_in, void* psi_out, const double* E_mid, int64_t nsteps, void* stream,
                    void* states = nullptr) {
    if (p->slab) return CN_ERR_UNSUPPORTED;  // a slab steps through cn_slab_reduce / cn_slab_finish
    if (!psi_in || (!psi_out && !states) || nsteps < 0) return CN_ERR_INVALID_ARG;
    if (!aligned16(psi_in) || (psi_out && !aligned16(psi_out)) || (states && !aligned16(states)))
        return CN_ERR_INVALID_ARG;
    if (E_mid && !aligned8(E_mid)) return CN_ERR_INVALID_ARG;
    if (states) {  // psi_in must not lie inside the states
        const uintptr_t a = reinterpret_cast<uintptr_t>(psi_in), s0 = reinterpret_cast<uintptr_t>(states);
        const uintptr_t len = sizeof(double2) * (uintptr_t)p->lv[0].rows_total;
        if (a + len > s0 && a < s0 + len * (uintptr_t)nsteps) return CN_ERR_INVALID_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double2* in = static_cast<const double2*>(psi_in);
    double2* out = static_cast<double2*>(psi_out);
    double2* sts = static_cast<double2*>(states);
    const size_t sb = sizeof(double2) * (size_t)p->lv[0].rows_total;
    cudaError_t e = dbg_register(p, st, {{psi_in, sb}, {psi_out, sb}, {states, sb * (size_t)nsteps},
                                         {E_mid, sizeof(double) * (size_t)nsteps}});
    if (e == cudaSuccess)
        e = (p->desc.arith == CN_ARITH_DF64) ? cn_steps<df>(p, in, out, E_mid, nsteps, st, sts)
                                             : cn_steps<double>(p, in, out, E_mid, nsteps, st, sts);
    return cuda_status(e);
}

// Fill every scratch buffer of the engine with `byte` (synchronously): the kept
// right-hand sides and pivots (or the recompute-mode state buffer), the reduced
// systems, CTA slots and solutions of every level, the long-block and serial-RS
// scratch, the adjoint's mu buffer, the host-call staging buffers and a slab's
// joint-solve scratch.  Not touched: the coefficient table and the per-system
// tables (built once at creation, read-only afterwards), the status word, the
// adjoint's ticket counter and the persistent launch's barrier words (which
// must hold their between-calls values).
cn_status fill_workspace(Engine* p, int byte) {
    if (byte < 0 || byte > 255) return CN_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess) return CN_ERR_CUDA;
    cudaError_t e = cudaSuccess;
    auto fill = [&](void* ptr, size_t bytes) {
        if (e == cudaSuccess && ptr && bytes) e = cudaMemset(ptr, byte, bytes);
    };
    const int64_t rows0 = p->lv[0].rows_total;
    if (p->keep)
        fill(p->keep, kCplx * keep_entries(p));
    fill(p->state, kCplx * (size_t)rows0);
    for (size_t l = 1; l < p->lv.size(); ++l) {
        const LevelData& L = p->lv[l];
        fill(L.rows, 4 * kCplx * (size_t)std::max<int64_t>(L.L, 1));
        fill(L.slot, 3 * kCplx * slot_entries(p, l));
        fill(L.x, kCplx * (size_t)L.rows_total);
    }
    const size_t zc_entries = zc_entries_of(p);
    fill(p->zc, kCplx * zc_entries);
    if (p->base_cs) fill(p->base_cs, kCplx * (size_t)p->lv[(size_t)p->base_level[0]].sys[0].n);
    fill(p->mu, sizeof(double2) * (size_t)p->desc.n);
    fill(p->h_in, sizeof(double2) * (size_t)p->desc.n);
    fill(p->h_out, sizeof(double2) * (size_t)p->desc.n);
    if (p->h_E) fill(p->h_E, sizeof(double) * (size_t)p->h_E_cap);
    fill(p->joint_work, 2 * sizeof(double2) * ((size_t)p->nslabs + 1));
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return cuda_status(e);
}

cn_status read_status(Engine* p) {
    if (cudaDeviceSynchronize() != cudaSuccess) return CN_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CN_ERR_CUDA;
    if (h != 0 && cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return CN_ERR_CUDA;
    // a grid barrier that gave up leaves its words mid-count: start them afresh
    if (h == CN_ERR_TIMEOUT && p->pbar && cudaMemset(p->pbar, 0, 2 * sizeof(unsigned int)) != cudaSuccess)
        return CN_ERR_CUDA;
    return static_cast<cn_status>(h);
}

void destroy_engine(Engine* p) {
    cudaDeviceSynchronize();
    free_engine(p);
}

}  // namespace

extern "C" {

const char* cn_status_string(cn_status s) {
    switch (s) {
    case CN_OK: return "ok";
    case CN_ERR_INVALID_ARG: return "invalid argument";
    case CN_ERR_UNSUPPORTED: return "unsupported";
    case CN_ERR_OOM: return "device out of memory";
    case CN_ERR_CUDA: return "CUDA runtime error";
    case CN_ERR_TIMEOUT: return "device-side wait timed out";
    case CN_ERR_NONFINITE: return "zero or non-finite pivot / result";
    case CN_ERR_BOUNDS: return "debug build: out-of-bounds access caught and skipped";
    default: return "unknown status";
    }
}

const char* cn_version(void) {
#if defined(CN_DEBUG)
    return "cn_b300 0.6 sm_103a debug";
#else
    return "cn_b300 0.6 sm_103a";
#endif
}

const char* cn_cuda_error_string(void) { return cudaGetErrorName(t_last_cuda_error); }

}  // extern "C"

namespace cnb_noalloc_debug {
int read_and_clear(unsigned long long* addr, unsigned long long* bytes);  // cn_noalloc.cu
}

#if defined(CN_DEBUG)
namespace {
__global__ void k_dbg_selftest(const double2* p, double2* out) {
    // p[0] is registered, p[1] lies in the same allocation but outside every
    // registered extent: the check must catch it and skip the load
    out[0] = dbg_ld(p + 1);
}
}  // namespace
#endif

extern "C" {

cn_status cn_debug_report(uint64_t* addr, uint64_t* bytes) {
#if defined(CN_DEBUG)
    if (cudaDeviceSynchronize() != cudaSuccess) return CN_ERR_CUDA;
    int flag = 0;
    unsigned long long a = 0, b = 0, zero = 0;
    if (cudaMemcpyFromSymbol(&flag, g_dbg_flag, sizeof(int)) != cudaSuccess) return CN_ERR_CUDA;
    if (flag) {
        cudaMemcpyFromSymbol(&a, g_dbg_addr, sizeof(a));
        cudaMemcpyFromSymbol(&b, g_dbg_bytes, sizeof(b));
        const int z = 0;
        cudaMemcpyToSymbol(g_dbg_flag, &z, sizeof(int));
        cudaMemcpyToSymbol(g_dbg_addr, &zero, sizeof(zero));
    } else {
        flag = cnb_noalloc_debug::read_and_clear(&a, &b);
    }
    if (addr) *addr = a;
    if (bytes) *bytes = b;
    return flag ? CN_ERR_BOUNDS : CN_OK;
#else
    if (addr) *addr = 0;
    if (bytes) *bytes = 0;
    return CN_ERR_UNSUPPORTED;
#endif
}

cn_status cn_debug_selftest(void) {
#if defined(CN_DEBUG)
    double2* buf = nullptr;
    if (cudaMalloc(&buf, 4 * sizeof(double2)) != cudaSuccess) return alloc_status(cudaErrorMemoryAllocation);
    cn_status r = CN_OK;
    uint64_t a = 0, b = 0;
    cn_debug_report(nullptr, nullptr);  // start from a clear record
    cudaError_t e = dbg_register(nullptr, nullptr, {{buf, sizeof(double2)}, {buf + 2, 2 * sizeof(double2)}});
    if (e == cudaSuccess) {
        k_dbg_selftest<<<1, 1>>>(buf, buf + 2);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) r = cuda_status(e);
    else if (cn_debug_report(&a, &b) != CN_ERR_BOUNDS || a != reinterpret_cast<uintptr_t>(buf + 1) ||
             b != sizeof(double2))
        r = CN_ERR_CUDA;  // the check missed the planted access
    dbg_register(nullptr, nullptr, {});
    cudaFree(buf);
    return r;
#else
    return CN_ERR_UNSUPPORTED;
#endif
}

cn_status cn_plan_create(const cn_desc* desc, cn_plan* out) {
    if (!out) return CN_ERR_INVALID_ARG;
    *out = nullptr;
    cn_status v = validate_desc(desc, true);
    if (v != CN_OK) return v;
    cn_plan p = new (std::nothrow) cn_plan_s();
    if (!p) return CN_ERR_OOM;
    v = create_engine(p, desc, std::vector<int64_t>{desc->n}, std::vector<double>{desc->x_min}, desc->cos_a);
    if (v != CN_OK) {
        destroy_engine(p);
        delete p;
        return v;
    }
    *out = p;
    return CN_OK;
}

cn_status cn_plan_create_levels(const cn_desc* desc, int32_t nlevels, const int32_t* blocks, cn_plan* out) {
    if (!out) return CN_ERR_INVALID_ARG;
    *out = nullptr;
    if (!desc || !blocks || nlevels < 1 || nlevels >= CN_MAX_LEVELS) return CN_ERR_INVALID_ARG;
    for (int l = 0; l < nlevels; ++l)
        if (blocks[l] < 3 || blocks[l] > CN_LEVELS_MAX_BLOCK) return CN_ERR_INVALID_ARG;
    cn_desc d = *desc;
    d.block = 0;
    d.level_block = 0;
    d.level1_block = 0;
    cn_status v = validate_desc(&d, true);
    if (v != CN_OK) return v;
    cn_plan p = new (std::nothrow) cn_plan_s();
    if (!p) return CN_ERR_OOM;
    p->lvl_m.assign(blocks, blocks + nlevels);
    v = create_engine(p, &d, std::vector<int64_t>{d.n}, std::vector<double>{d.x_min}, d.cos_a);
    if (v != CN_OK) {
        destroy_engine(p);
        delete p;
        return v;
    }
    *out = p;
    return CN_OK;
}

cn_status cn_plan_destroy(cn_plan p) {
    if (!p) return CN_OK;
    destroy_engine(p);
    delete p;
    return CN_OK;
}

cn_status cn_step(cn_plan p, const void* psi_in, void* psi_out, const double* E_mid, int64_t nsteps, void* stream) {
    if (!p) return CN_ERR_INVALID_ARG;
    return run_steps(p, psi_in, psi_out, E_mid, nsteps, stream);
}

cn_status cn_step_states(cn_plan p, const void* psi_in, void* states_out, const double* E_mid, int64_t nsteps,
                         void* stream) {
    if (!p || !states_out) return CN_ERR_INVALID_ARG;
    return run_steps(p, psi_in, nullptr, E_mid, nsteps, stream, states_out);
}

cn_status cn_step_host(cn_plan p, const void* psi_in_host, void* psi_out_host, const double* E_mid_host,
                       int64_t nsteps, void* stream) {
    if (!p || !psi_in_host || !psi_out_host || nsteps < 0) return CN_ERR_INVALID_ARG;
    if (p->slab) return CN_ERR_UNSUPPORTED;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t bytes = sizeof(double2) * (size_t)p->desc.n;
    cudaError_t e = cudaSuccess;
    if (!p->h_in) e = cudaMalloc(&p->h_in, bytes);
    if (e == cudaSuccess && !p->h_out) e = cudaMalloc(&p->h_out, bytes);
    if (e == cudaSuccess && E_mid_host && p->h_E_cap < nsteps) {
        cudaFree(p->h_E);
        p->h_E = nullptr;
        p->h_E_cap = 0;
        e = cudaMalloc(&p->h_E, sizeof(double) * (size_t)nsteps);
        if (e == cudaSuccess) p->h_E_cap = nsteps;
    }
    if (e != cudaSuccess) return alloc_status(e);
    e = cudaMemcpyAsync(p->h_in, psi_in_host, bytes, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && E_mid_host && nsteps > 0)
        e = cudaMemcpyAsync(p->h_E, E_mid_host, sizeof(double) * (size_t)nsteps, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return CN_ERR_CUDA;
    cn_status s = cn_step(p, p->h_in, p->h_out, E_mid_host ? p->h_E : nullptr, nsteps, stream);
    if (s != CN_OK) return s;
    e = cudaMemcpyAsync(psi_out_host, p->h_out, bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return cuda_status(e);
}

cn_status cn_solve_tridiag(cn_plan p, const void* b, const void* a, const void* c, const void* d, void* x, int64_t n,
                           void* stream) {
    if (!p || !b || !a || !c || !d || !x) return CN_ERR_INVALID_ARG;
    if (p->slab) return CN_ERR_UNSUPPORTED;
    if (n != p->desc.n) return CN_ERR_INVALID_ARG;
    if (!aligned16(b) || !aligned16(a) || !aligned16(c) || !aligned16(d) || !aligned16(x)) return CN_ERR_INVALID_ARG;
    if (x == b || x == a || x == c) return CN_ERR_INVALID_ARG;
    ArraySource s;
    s.b = static_cast<const double2*>(b);
    s.a = static_cast<const double2*>(a);
    s.c = static_cast<const double2*>(c);
    s.d = static_cast<const double2*>(d);
    s.n = n;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t vb = sizeof(double2) * (size_t)n;
    cudaError_t e = dbg_register(p, st, {{b, vb}, {a, vb}, {c, vb}, {d, vb}, {x, vb}});
    if (e == cudaSuccess)
        e = (p->desc.arith == CN_ARITH_DF64) ? solve_arrays<df>(p, s, static_cast<double2*>(x), st)
                                             : solve_arrays<double>(p, s, static_cast<double2*>(x), st);
    return cuda_status(e);
}

cn_status cn_adjoint_step(cn_plan p, const void* psi_n, const void* psi_np1, const void* lam_np1, void* lam_n,
                          const double* E_mid, double* dLdE, void* stream) {
    if (!p || !psi_n || !psi_np1 || !lam_np1 || !lam_n || !dLdE) return CN_ERR_INVALID_ARG;
    if (p->slab) return CN_ERR_UNSUPPORTED;
    if (!aligned16(psi_n) || !aligned16(psi_np1) || !aligned16(lam_np1) || !aligned16(lam_n)) return CN_ERR_INVALID_ARG;
    if (!aligned8(dLdE) || (E_mid && !aligned8(E_mid))) return CN_ERR_INVALID_ARG;
    const int nparts = 148 * 4;
    cudaError_t e = cudaSuccess;
    if (!p->mu) e = cudaMalloc(&p->mu, sizeof(double2) * (size_t)p->desc.n);
    if (e == cudaSuccess && !p->part) {
        // partials, then the ticket counter of k_adjoint_finish (zero between launches)
        e = cudaMalloc(&p->part, 16 * (size_t)nparts + 16);
        if (e == cudaSuccess) e = cudaMemset(p->part, 0, 16 * (size_t)nparts + 16);
        if (e == cudaSuccess) {
            p->part_n = nparts;
            p->ticket = reinterpret_cast<unsigned int*>(static_cast<char*>(p->part) + 16 * (size_t)nparts);
        } else {
            cudaFree(p->part);
            p->part = nullptr;
        }
    }
    if (e != cudaSuccess) return alloc_status(e);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // The adjoint step launches in plain stream order: with programmatic launches
    // it measured 17 us per step slower on B300 (N = 2^20: backward 394 vs 359 ms
    // over 2000 steps) while the forward step loop gains from them.
    struct PlainLaunches {
        Engine* q;
        explicit PlainLaunches(Engine* e) : q(e) { q->pdl = false; }
        ~PlainLaunches() { q->pdl = true; }
    } plain(p);
    CNStep s;
    s.p = p->cnp;
    s.psi = static_cast<const double2*>(lam_np1);
    s.s = -1;  // implicit matrix T^dagger = 1 - i dt/2 H
    s.e = 0;   // right-hand side lam_{n+1} itself
    s.E = E_mid;
    s.tab = p->tab;
    s.own_last = 1;
    const bool dfm = p->desc.arith == CN_ARITH_DF64;
    const size_t vb = sizeof(double2) * (size_t)p->desc.n;
    e = dbg_register(p, st, {{psi_n, vb}, {psi_np1, vb}, {lam_np1, vb}, {lam_n, vb}, {E_mid, sizeof(double)},
                             {dLdE, sizeof(double)}});
    if (e != cudaSuccess) return cuda_status(e);
    e = dfm ? cn_solve<df>(p, s, p->mu, st) : cn_solve<double>(p, s, p->mu, st);
    if (e != cudaSuccess) return CN_ERR_CUDA;
    const SysGrid& g = p->grid[0];
    const int64_t n = p->desc.n;
    const double2* l1 = static_cast<const double2*>(lam_np1);
    const double2* pn = static_cast<const double2*>(psi_n);
    const double2* pn1 = static_cast<const double2*>(psi_np1);
    double2* ln = static_cast<double2*>(lam_n);
    const double2* mu = p->mu;
    if (dfm)
        e = launch(p->pdl, k_adjoint_finish<df>, (unsigned)p->part_n, kAdjThreads, 0, st, p->cnp, g, n, mu, l1, pn,
                   pn1, ln, static_cast<df*>(p->part), p->ticket, p->desc.dt, dLdE);
    else
        e = launch(p->pdl, k_adjoint_finish<double>, (unsigned)p->part_n, kAdjThreads, 0, st, p->cnp, g, n, mu, l1,
                   pn, pn1, ln, static_cast<double*>(p->part), p->ticket, p->desc.dt, dLdE);
    return cuda_status(e);
}

cn_status cn_field_from_controls(const double* u, int64_t n_controls, double t_final, double t0, double dt,
                                 int64_t nsteps, double* E_mid, void* stream) {
    if (!u || !E_mid || n_controls < 2 || nsteps < 0 || !(t_final > 0.0) || !std::isfinite(t0) ||
        !std::isfinite(dt) || dt == 0.0)
        return CN_ERR_INVALID_ARG;
    if (nsteps == 0) return CN_OK;
    cudaError_t e = dbg_register(nullptr, static_cast<cudaStream_t>(stream),
                                 {{u, sizeof(double) * (size_t)n_controls}, {E_mid, sizeof(double) * (size_t)nsteps}});
    if (e != cudaSuccess) return cuda_status(e);
    k_hat_field<<<(unsigned)ceil_div(nsteps, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        u, n_controls, t_final, t0, dt, nsteps, E_mid);
    return cuda_status(cudaGetLastError());
}

cn_status cn_field_grad_to_controls(const double* dLdE, int64_t nsteps, double t_final, double t0, double dt,
                                    int64_t n_controls, double* grad_u, void* stream) {
    if (!dLdE || !grad_u || n_controls < 2 || nsteps < 0 || !(t_final > 0.0) || !std::isfinite(t0) ||
        !(dt > 0.0))
        return CN_ERR_INVALID_ARG;
    cudaError_t e = dbg_register(nullptr, static_cast<cudaStream_t>(stream),
                                 {{dLdE, sizeof(double) * (size_t)nsteps}, {grad_u, sizeof(double) * (size_t)n_controls}});
    if (e != cudaSuccess) return cuda_status(e);
    k_hat_field_grad<<<(unsigned)ceil_div(n_controls, 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        dLdE, nsteps, t_final, t0, dt, n_controls, grad_u);
    return cuda_status(cudaGetLastError());
}

cn_status cn_plan_query(cn_plan p, cn_plan_info* out) {
    if (!p || !out) return CN_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = p->desc.n;
    out->levels = p->base_level[0];
    for (int l = 0; l <= out->levels; ++l) {
        out->level_rows[l] = p->lv[(size_t)l].sys[0].n;
        out->level_block[l] = (l < out->levels) ? p->lv[(size_t)l].m : 0;
    }
    out->launches_per_step = p->persistent ? 3 : 2 * out->levels + 1;
    out->workspace_bytes = p->workspace_bytes;
    out->level0_lanes = p->scan0 ? scan_threads(p->lv[0].m) : 1;
    return CN_OK;
}

cn_status cn_plan_profile(cn_plan p, int enable) {
    if (!p) return CN_ERR_INVALID_ARG;
    p->profiling = enable != 0;
    return CN_OK;
}

cn_status cn_plan_profile_read(cn_plan p, double* ms, int64_t* launches, int32_t cap) {
    if (!p || cap < 0 || (cap > 0 && (!ms || !launches))) return CN_ERR_INVALID_ARG;
    for (int c = 0; c < cap && c < CN_PROFILE_CLASSES; ++c) { ms[c] = 0.0; launches[c] = 0; }
    cn_status st = CN_OK;
    if (p->ev_used > 0 && cudaEventSynchronize(p->ev_pool[p->ev_used - 1]) != cudaSuccess) st = CN_ERR_CUDA;
    for (size_t r = 0; st == CN_OK && r < p->rec_class.size(); ++r) {
        float t = 0.f;
        if (cudaEventElapsedTime(&t, p->ev_pool[2 * r], p->ev_pool[2 * r + 1]) != cudaSuccess) { st = CN_ERR_CUDA; break; }
        int c = p->rec_class[r];
        if (c < cap) { ms[c] += (double)t; launches[c] += 1; }
    }
    p->rec_class.clear();
    p->ev_used = 0;
    return st;
}

cn_status cn_plan_status(cn_plan p) {
    if (!p) return CN_ERR_INVALID_ARG;
    return read_status(p);
}

cn_status cn_plan_fill_workspace(cn_plan p, int32_t byte) {
    if (!p) return CN_ERR_INVALID_ARG;
    return fill_workspace(p, byte);
}

cn_status cn_plan_set_wait_limit(cn_plan p, int64_t timeout_ns, int32_t missing_ctas) {
    if (!p || timeout_ns <= 0 || missing_ctas < 0) return CN_ERR_INVALID_ARG;
    p->wait_ns = timeout_ns;
    p->wait_missing = (unsigned)missing_ctas;
    return CN_OK;
}

// ------------------------------------------------------------------ slabs of a sharded grid
cn_status cn_slab_create(const cn_desc* desc, int32_t nslabs, int32_t rank, const int64_t* joints, cn_plan* out) {
    if (!out) return CN_ERR_INVALID_ARG;
    *out = nullptr;
    cn_status v = validate_desc(desc, true);
    if (v != CN_OK) return v;
    if (nslabs < 1 || nslabs > CN_SLAB_MAX || rank < 0 || rank >= nslabs) return CN_ERR_INVALID_ARG;
    const int64_t n = desc->n;
    std::vector<int64_t> J((size_t)nslabs + 1);
    for (int r = 0; r <= nslabs; ++r) {
        J[(size_t)r] = joints ? joints[r] : (int64_t)(((__int128)r * (n - 1)) / nslabs);
        if (r > 0 && J[(size_t)r] - J[(size_t)r - 1] < 2) return CN_ERR_INVALID_ARG;
    }
    if (J[0] != 0 || J[(size_t)nslabs] != n - 1) return CN_ERR_INVALID_ARG;
    const int64_t lo = J[(size_t)rank], hi = J[(size_t)rank + 1];
    cn_desc d = *desc;
    d.n = hi - lo + 1;
    d.x_min = desc->x_min + (double)lo * desc->dx;  // informational: the grid below is the global one
    if (d.pot == CN_POT_ARRAY) d.V0 = desc->V0 + lo;
    // the global grid's coordinates x_j = x_o + (j - j_o) dx, j counted from this slab's row 0
    SysGrid g = make_grid(desc->x_min, desc->dx, n);
    g.j_o -= lo;
    cn_plan p = new (std::nothrow) cn_plan_s();
    if (!p) return CN_ERR_OOM;
    p->slab = true;
    p->own_last = rank == nslabs - 1;
    p->nslabs = nslabs;
    p->slab_rank = rank;
    p->slab_lo = lo;
    p->slab_hi = hi;
    v = create_engine(p, &d, std::vector<int64_t>{d.n}, std::vector<double>{d.x_min}, d.cos_a, &g);
    if (v == CN_OK) {
        p->workspace_bytes += (int64_t)(2 * sizeof(double2) * ((size_t)nslabs + 1));
        if (cudaMalloc(&p->joint_work, 2 * sizeof(double2) * ((size_t)nslabs + 1)) != cudaSuccess)
            v = alloc_status(cudaErrorMemoryAllocation);
    }
    if (v != CN_OK) {
        destroy_engine(p);
        delete p;
        return v;
    }
    *out = p;
    return CN_OK;
}

cn_status cn_slab_range(cn_plan p, int64_t* lo, int64_t* hi) {
    if (!p || !p->slab || !lo || !hi) return CN_ERR_INVALID_ARG;
    *lo = p->slab_lo;
    *hi = p->slab_hi;
    return CN_OK;
}

}  // extern "C"

namespace {
template <class R>
cudaError_t slab_reduce(Engine* p, const double2* psi, const double* E_mid, double2* share, cudaStream_t st) {
    CNStep s;
    s.p = p->cnp;
    s.psi = psi;
    s.s = 1;
    s.e = -1;
    s.E = E_mid;
    s.tab = p->tab;
    s.own_last = p->own_last ? 1 : 0;
    cudaError_t e = cn_reduce0<R>(p, s, st);
    if (e == cudaSuccess) e = reduce_levels<R>(p, st);
    if (e == cudaSuccess) {
        const LevelData& B = p->lv.back();
        e = launch(p->pdl, k_slab_export<R>, 1, 32, 0, st, level_source<R>(B).bind(B.sys[0]), share);
    }
    return e;
}

template <class R>
cudaError_t slab_finish(Engine* p, const double2* shares, double2* psi_out, cudaStream_t st) {
    const LevelData& B = p->lv.back();
    cudaError_t e = launch(p->pdl, k_slab_joints<R>, 1, 32, 0, st, shares, p->nslabs, p->slab_rank, p->joint_work,
                           p->joint_work + p->nslabs + 1, x_of<R>(B), p->status);
    if (e == cudaSuccess) e = substitute_levels<R>(p, st);
    if (e == cudaSuccess) {
        CNStep s;
        s.p = p->cnp;
        s.psi = nullptr;
        s.s = 1;
        s.e = -1;
        s.E = nullptr;
        s.tab = p->tab;
        s.own_last = p->own_last ? 1 : 0;
        e = cn_subst0<R>(p, s, psi_out, st);
    }
    return e;
}
}  // namespace

extern "C" {

cn_status cn_slab_reduce(cn_plan p, const void* psi_local, const double* E_mid, void* share_out, void* stream) {
    if (!p || !p->slab || !psi_local || !share_out) return CN_ERR_INVALID_ARG;
    if (!p->keep) return CN_ERR_UNSUPPORTED;  // recompute mode keeps no right-hand sides
    if (!aligned16(psi_local) || !aligned16(share_out) || (E_mid && !aligned8(E_mid))) return CN_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double2* in = static_cast<const double2*>(psi_local);
    double2* sh = static_cast<double2*>(share_out);
    cudaError_t e = dbg_register(p, st, {{psi_local, sizeof(double2) * (size_t)p->desc.n}, {E_mid, sizeof(double)},
                                         {share_out, 6 * sizeof(double2)}});
    if (e == cudaSuccess)
        e = (p->desc.arith == CN_ARITH_DF64) ? slab_reduce<df>(p, in, E_mid, sh, st)
                                             : slab_reduce<double>(p, in, E_mid, sh, st);
    return cuda_status(e);
}

cn_status cn_slab_finish(cn_plan p, const void* shares, void* psi_local_out, void* stream) {
    if (!p || !p->slab || !shares || !psi_local_out) return CN_ERR_INVALID_ARG;
    if (!p->keep) return CN_ERR_UNSUPPORTED;
    if (!aligned16(shares) || !aligned16(psi_local_out)) return CN_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double2* sh = static_cast<const double2*>(shares);
    double2* out = static_cast<double2*>(psi_local_out);
    cudaError_t e = dbg_register(p, st, {{shares, 6 * sizeof(double2) * (size_t)p->nslabs},
                                         {psi_local_out, sizeof(double2) * (size_t)p->desc.n}});
    if (e == cudaSuccess)
        e = (p->desc.arith == CN_ARITH_DF64) ? slab_finish<df>(p, sh, out, st)
                                             : slab_finish<double>(p, sh, out, st);
    return cuda_status(e);
}

// ------------------------------------------------------------------ batches
cn_status cn_batch_create(const cn_desc* common, int64_t nsys, const int64_t* sizes, const double* x_min,
                          const double* cos_a, cn_batch* out) {
    if (!out) return CN_ERR_INVALID_ARG;
    *out = nullptr;
    cn_status v = validate_desc(common, false);
    if (v != CN_OK) return v;
    if (nsys < 1 || nsys > kMaxBatch || !sizes) return CN_ERR_INVALID_ARG;
    if (common->pot == CN_POT_COSSERIES && common->n_cos > 0 && !cos_a) return CN_ERR_INVALID_ARG;
    std::vector<int64_t> sz((size_t)nsys);
    std::vector<double> xm((size_t)nsys);
    cn_desc d = *common;
    d.n = 0;
    for (int64_t s = 0; s < nsys; ++s) {
        if (sizes[s] < 3 || sizes[s] > (INT64_C(1) << 40)) return CN_ERR_INVALID_ARG;
        sz[(size_t)s] = sizes[s];
        xm[(size_t)s] = x_min ? x_min[s] : -(double)(sizes[s] / 2) * common->dx;
        if (!std::isfinite(xm[(size_t)s])) return CN_ERR_INVALID_ARG;
        d.n += sizes[s];
    }
    if (common->pot == CN_POT_COSSERIES && common->n_cos > 0) {
        for (int64_t i = 0; i < nsys * common->n_cos; ++i)
            if (!std::isfinite(cos_a[i])) return CN_ERR_INVALID_ARG;
    }
    cn_batch p = new (std::nothrow) cn_batch_s();
    if (!p) return CN_ERR_OOM;
    p->batched = true;
    v = create_engine(p, &d, sz, xm, cos_a);
    if (v != CN_OK) {
        destroy_engine(p);
        delete p;
        return v;
    }
    *out = p;
    return CN_OK;
}

cn_status cn_batch_destroy(cn_batch p) {
    if (!p) return CN_OK;
    destroy_engine(p);
    delete p;
    return CN_OK;
}

cn_status cn_batch_offsets(cn_batch p, int64_t* offsets) {
    if (!p || !offsets) return CN_ERR_INVALID_ARG;
    for (int s = 0; s < p->nsys; ++s) offsets[s] = p->lv[0].sys[(size_t)s].row_off;
    offsets[p->nsys] = p->lv[0].rows_total;
    return CN_OK;
}

cn_status cn_batch_step(cn_batch p, const void* psi_in, void* psi_out, const double* E_mid, int64_t nsteps,
                        void* stream) {
    if (!p) return CN_ERR_INVALID_ARG;
    return run_steps(p, psi_in, psi_out, E_mid, nsteps, stream);
}

cn_status cn_batch_status(cn_batch p) {
    if (!p) return CN_ERR_INVALID_ARG;
    return read_status(p);
}

cn_status cn_batch_fill_workspace(cn_batch p, int32_t byte) {
    if (!p) return CN_ERR_INVALID_ARG;
    return fill_workspace(p, byte);
}

}  // extern "C"
