// cn_api.cu -- C ABI (include/cn.h): plans, argument validation, and the launch
// sequence of the nested N-shaped solve (Eq. iteration of the paper).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/cn.h"
#include "cn_kernels.cuh"

using namespace cnb;

namespace {

constexpr int kDefaultLevelBlock = 8;  // rows per block on the reduced levels (>= 1)
constexpr int kDefaultBlock = 8;       // rows per level-0 block unless the descriptor says otherwise
constexpr int kMaxBlockRows = 32;      // shared memory of the substitution: 2 x 32 x 128 x 16 B

struct Level {
    int64_t n = 0;         // rows
    int64_t P = 0;         // blocks (joint lines 0..P)
    int m = 0;             // block size
    void* rows = nullptr;  // LevelRow<R>[n] (levels >= 1)
    void* slot = nullptr;  // LevelSlot<R>[CTAs of the level below + 1]
    void* x = nullptr;     // Store<R>::T[n]: solution of this level (levels >= 1)
};

}  // namespace

struct cn_plan_s {
    cn_desc desc;
    int device = 0;
    std::vector<Level> lv;     // lv[0]: the system itself; lv[L]: solved by the RS stage
    double2* state = nullptr;  // n complex128 scratch for the step ping-pong (recompute mode)
    void* keep = nullptr;      // 2 n Store<R>::T: explicit rhs and pivot per point (store mode)
    void* tab = nullptr;       // bt0 table (compute type) or NULL
    int* status = nullptr;     // device status word
    CNParams cnp;
    std::vector<double> cos_a;
    // cn_step_host staging (allocated on first use)
    double2* h_in = nullptr;
    double2* h_out = nullptr;
    double* h_E = nullptr;
    int64_t h_E_cap = 0;
    // adjoint (allocated on first use)
    double2* mu = nullptr;
    void* part = nullptr;
    int part_n = 0;
    // kernel timing (cn_plan_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;  // events owned by the plan
    size_t ev_used = 0;                // events handed out since the last read
    std::vector<int> rec_class;        // class of record r (events 2r, 2r+1)
    int64_t workspace_bytes = 0;
};

namespace {

cn_status cuda_status(cudaError_t e) { return e == cudaSuccess ? CN_OK : CN_ERR_CUDA; }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

cn_status validate_desc(const cn_desc* d) {
    if (!d) return CN_ERR_INVALID_ARG;
    if (d->n < 3) return CN_ERR_INVALID_ARG;
    if (!(d->dx > 0.0) || !std::isfinite(d->dx)) return CN_ERR_INVALID_ARG;
    if (!std::isfinite(d->dt) || d->dt == 0.0 || !std::isfinite(d->x_min)) return CN_ERR_INVALID_ARG;
    if (d->pot < CN_POT_NONE || d->pot > CN_POT_COSSERIES) return CN_ERR_INVALID_ARG;
    if (d->pot == CN_POT_ARRAY && (!d->V0 || (reinterpret_cast<uintptr_t>(d->V0) & 7u))) return CN_ERR_INVALID_ARG;
    if (d->pot == CN_POT_SOFTCOULOMB && !(d->soft_s > 0.0)) return CN_ERR_INVALID_ARG;
    if (d->pot == CN_POT_COSSERIES) {
        if (d->n_cos < 0 || d->n_cos > kMaxCos || (d->n_cos > 0 && !d->cos_a) || !(d->L > 0.0))
            return CN_ERR_INVALID_ARG;
    }
    if (d->block != 0 && (d->block < 3 || d->block > kMaxBlockRows)) return CN_ERR_INVALID_ARG;
    if (d->level_block != 0 && (d->level_block < 3 || d->level_block > kMaxBlockRows)) return CN_ERR_INVALID_ARG;
    if (d->arith != CN_ARITH_F64 && d->arith != CN_ARITH_DF64) return CN_ERR_INVALID_ARG;
    if ((d->flags & ~(CN_FLAG_COEFF_TABLE | CN_FLAG_RECOMPUTE)) != 0) return CN_ERR_INVALID_ARG;
    return CN_OK;
}

void free_plan_memory(cn_plan p) {
    for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
    p->ev_pool.clear();
    for (Level& L : p->lv) {
        cudaFree(L.rows);
        cudaFree(L.slot);
        cudaFree(L.x);
    }
    cudaFree(p->state);
    cudaFree(p->keep);
    cudaFree(p->tab);
    cudaFree(p->status);
    cudaFree(p->h_in);
    cudaFree(p->h_out);
    cudaFree(p->h_E);
    cudaFree(p->mu);
    cudaFree(p->part);
}

int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

unsigned grid_for(int64_t P) { return (unsigned)ceil_div(P, kThreads); }

// --------------------------------------------------------------- kernel timing
enum { kProfReduce0 = 0, kProfSubst0 = 1, kProfReduceL = 2, kProfSubstL = 3, kProfBase = 4 };

// Two events per record; the pool grows on demand and is reused after a read.
bool reserve_events(cn_plan p, size_t k) {
    while (p->ev_pool.size() < p->ev_used + k) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        p->ev_pool.push_back(e);
    }
    return true;
}

struct ProfScope {
    cn_plan p;
    cudaStream_t st;
    cudaEvent_t stop = nullptr;
    ProfScope(cn_plan p_, int cls, cudaStream_t st_) : p(p_), st(st_) {
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

template <class R> LevelRow<R>* rows_of(const Level& L) { return static_cast<LevelRow<R>*>(L.rows); }
template <class R> LevelSlot<R>* slot_of(const Level& L) { return static_cast<LevelSlot<R>*>(L.slot); }
template <class R> typename Store<R>::T* x_of(const Level& L) { return static_cast<typename Store<R>::T*>(L.x); }

template <class R> LevelSource<R> level_source(const Level& L) {
    LevelSource<R> s;
    s.rows = rows_of<R>(L);
    s.slot = slot_of<R>(L);
    s.n = L.n;
    s.slot_stride = kThreads;
    return s;
}

// --------------------------------------------------------------- launch helpers
// Shared memory of the substitution kernels: per thread, one (kept) or two
// complex values per block row.
size_t subst_smem(int m, int arrays) { return (size_t)arrays * (size_t)m * kThreads * 16; }
size_t kept_smem(int m) { return (size_t)m * kTileStride * 16; }

template <class R, class Src>
cudaError_t launch_reduce(const Src& src, const Level& L, const Level& next, int* status, cudaStream_t st) {
    k_reduce<R, Src><<<grid_for(L.P), kThreads, 0, st>>>(src, L.n, L.P, L.m, rows_of<R>(next), slot_of<R>(next),
                                                         status);
    return cudaGetLastError();
}

template <class R, class Src, class XT>
cudaError_t launch_substitute(const Src& src, const Level& L, const Level& next, XT* x, int* status, cudaStream_t st) {
    k_substitute<R, Src, XT><<<grid_for(L.P), kThreads, subst_smem(L.m, 2), st>>>(src, L.n, L.P, L.m, x_of<R>(next),
                                                                                  x, status);
    return cudaGetLastError();
}

// Opt every substitution kernel into the dynamic shared memory its largest block needs.
template <class R>
cudaError_t set_smem_limits(int m0, int ml) {
    cudaError_t e = cudaFuncSetAttribute(k_substitute<R, ArraySource, double2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)subst_smem(m0, 2));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_substitute<R, LevelSource<R>, typename Store<R>::T>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)subst_smem(ml, 2));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cn_substitute<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)subst_smem(m0, 2));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_cn_substitute_kept<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)kept_smem(m0));
    return e;
}

// Levels 1..L of the nested solve: reductions down, RS, substitutions up.
template <class R>
cudaError_t solve_levels(cn_plan p, cudaStream_t st) {
    const int L = (int)p->lv.size() - 1;
    cudaError_t e = cudaSuccess;
    for (int l = 1; l < L; ++l) {
        ProfScope ps(p, kProfReduceL, st);
        e = launch_reduce<R>(level_source<R>(p->lv[l]), p->lv[l], p->lv[l + 1], p->status, st);
        if (e != cudaSuccess) return e;
    }
    {
        ProfScope ps(p, kProfBase, st);
        k_base<R><<<1, 32, 0, st>>>(level_source<R>(p->lv[L]), p->lv[L].n, x_of<R>(p->lv[L]), p->status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    for (int l = L - 1; l >= 1; --l) {
        ProfScope ps(p, kProfSubstL, st);
        e = launch_substitute<R>(level_source<R>(p->lv[l]), p->lv[l], p->lv[l + 1], x_of<R>(p->lv[l]), p->status, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// General tridiagonal solve (arrays at level 0).
template <class R>
cudaError_t solve_arrays(cn_plan p, const ArraySource& src, double2* x, cudaStream_t st) {
    cudaError_t e;
    {
        ProfScope ps(p, kProfReduce0, st);
        e = launch_reduce<R>(src, p->lv[0], p->lv[1], p->status, st);
    }
    if (e != cudaSuccess) return e;
    if ((e = solve_levels<R>(p, st)) != cudaSuccess) return e;
    ProfScope ps(p, kProfSubst0, st);
    return launch_substitute<R>(src, p->lv[0], p->lv[1], x, p->status, st);
}

// One CN-type step (level 0 generated on the fly), result in x.
template <class R>
cudaError_t cn_solve(cn_plan p, const CNStep& s, double2* x, cudaStream_t st) {
    const Level& L0 = p->lv[0];
    const Level& L1 = p->lv[1];
    const unsigned grid = grid_for(L0.P);
    typedef typename Store<R>::T ST;
    ST* keep = static_cast<ST*>(p->keep);
    cudaError_t e;
    {
        ProfScope ps(p, kProfReduce0, st);
        k_cn_reduce<R><<<grid, kThreads, 0, st>>>(s, L0.P, L0.m, rows_of<R>(L1), slot_of<R>(L1), keep, p->status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if ((e = solve_levels<R>(p, st)) != cudaSuccess) return e;
    ProfScope ps(p, kProfSubst0, st);
    if (keep)
        k_cn_substitute_kept<R><<<grid, kThreads, kept_smem(L0.m), st>>>(L0.n, L0.P, L0.m, keep, x_of<R>(L1), x);
    else
        k_cn_substitute<R><<<grid, kThreads, subst_smem(L0.m, 2), st>>>(s, L0.P, L0.m, x_of<R>(L1), x, p->status);
    return cudaGetLastError();
}

template <class R>
cudaError_t cn_steps(cn_plan p, const double2* in, double2* out, const double* E_mid, int64_t nsteps,
                     cudaStream_t st) {
    const size_t bytes = sizeof(double2) * (size_t)p->desc.n;
    if (nsteps == 0) {
        if (in == out) return cudaSuccess;
        return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
    }
    const bool kept = p->keep != nullptr;
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
        CNStep s;
        s.p = p->cnp;
        s.psi = src;
        s.s = 1;
        s.e = -1;
        s.E_t = E_mid ? E_mid + k : nullptr;
        s.E_e = s.E_t;
        s.tab = p->tab;
        cudaError_t e = cn_solve<R>(p, s, dst, st);
        if (e != cudaSuccess) return e;
        src = dst;
    }
    return cudaSuccess;
}

size_t real_size(int arith) { return arith == CN_ARITH_DF64 ? sizeof(df) : sizeof(double); }

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
    default: return "unknown status";
    }
}

const char* cn_version(void) { return "cn_b300 0.4 sm_103a"; }

cn_status cn_plan_create(const cn_desc* desc, cn_plan* out) {
    if (!out) return CN_ERR_INVALID_ARG;
    *out = nullptr;
    cn_status v = validate_desc(desc);
    if (v != CN_OK) return v;
    cn_plan p = new (std::nothrow) cn_plan_s();
    if (!p) return CN_ERR_OOM;
    p->desc = *desc;
    if (p->desc.block == 0) p->desc.block = kDefaultBlock;
    if (p->desc.level_block == 0) p->desc.level_block = kDefaultLevelBlock;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return CN_ERR_CUDA; }
    if (desc->pot == CN_POT_COSSERIES && desc->n_cos > 0) p->cos_a.assign(desc->cos_a, desc->cos_a + desc->n_cos);
    p->desc.cos_a = nullptr;
    const bool df_mode = desc->arith == CN_ARITH_DF64;
    const bool use_table = (desc->flags & CN_FLAG_COEFF_TABLE) ||
                           (df_mode && (desc->pot == CN_POT_ARRAY || desc->pot == CN_POT_COSSERIES));

    // levels: level l has n_l rows in P_l blocks of m_l rows; n_{l+1} = P_l + 1
    int64_t n = desc->n;
    int m = p->desc.block;
    for (;;) {
        Level L;
        L.n = n;
        L.m = m;
        L.P = ceil_div(n - 1, m);
        p->lv.push_back(L);
        n = L.P + 1;
        m = p->desc.level_block;
        if (n <= kBaseMax) {
            Level B;
            B.n = n;
            p->lv.push_back(B);
            break;
        }
    }
    const size_t cplx = 16;  // bytes per complex in either compute type
    cudaError_t e = cudaSuccess;
    for (size_t l = 1; l < p->lv.size() && e == cudaSuccess; ++l) {
        Level& L = p->lv[l];
        const size_t nslot = grid_for(p->lv[l - 1].P) + 1;
        p->workspace_bytes += (int64_t)(5 * cplx * L.n + 3 * cplx * nslot);
        e = cudaMalloc(&L.rows, 4 * cplx * (size_t)L.n);
        if (e == cudaSuccess) e = cudaMalloc(&L.slot, 3 * cplx * nslot);
        if (e == cudaSuccess) e = cudaMalloc(&L.x, cplx * (size_t)L.n);
        if (e == cudaSuccess) e = cudaMemset(L.slot, 0, 3 * cplx * nslot);
    }
    const bool recompute = (desc->flags & CN_FLAG_RECOMPUTE) != 0;
    // keep: entries (2k) P + t and (2k+1) P + t for block rows k = 1..m-1
    const size_t keep_entries = 2 * (size_t)p->lv[0].m * (size_t)p->lv[0].P;
    p->workspace_bytes += (int64_t)(recompute ? cplx * desc->n : cplx * keep_entries) + (int64_t)sizeof(int);
    if (e == cudaSuccess && recompute) e = cudaMalloc(&p->state, cplx * (size_t)desc->n);
    if (e == cudaSuccess && !recompute) e = cudaMalloc(&p->keep, cplx * keep_entries);
    if (e == cudaSuccess) e = cudaMalloc(&p->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(int));
    if (e == cudaSuccess && use_table) {
        p->workspace_bytes += (int64_t)(real_size(desc->arith) * desc->n);
        e = cudaMalloc(&p->tab, real_size(desc->arith) * (size_t)desc->n);
    }
    CNParams& c = p->cnp;
    std::memset(&c, 0, sizeof(c));
    c.n = desc->n;
    c.dx = desc->dx;
    c.x_min = desc->x_min;
    c.c1 = 2.0 * desc->dx * desc->dx;
    c.gt = 4.0 * desc->dx * desc->dx / desc->dt;
    c.pot = desc->pot;
    c.V0 = desc->V0;
    c.soft_s = desc->soft_s;
    c.n_cos = desc->pot == CN_POT_COSSERIES ? desc->n_cos : 0;
    c.two_pi_over_L = desc->pot == CN_POT_COSSERIES ? 2.0 * 3.14159265358979323846 / desc->L : 0.0;
    for (int k = 0; k < c.n_cos; ++k) c.cos_a[k] = p->cos_a[(size_t)k];
    auto split = [](double v) { df d = df_from_double(v); DFc r; r.hi = d.hi; r.lo = d.lo; return r; };
    c.dx_f = split(c.dx);
    c.c1_f = split(c.c1);
    c.gt_f = split(c.gt);
    c.soft_f = split(c.soft_s);
    {
        double jo = std::nearbyint(-desc->x_min / desc->dx);
        if (jo < 0) jo = 0;
        if (jo > (double)(desc->n - 1)) jo = (double)(desc->n - 1);
        c.j_o = (int64_t)jo;
        c.x_o = desc->x_min + (double)c.j_o * desc->dx;
        c.xo_f = split(c.x_o);
    }
    if (e == cudaSuccess && use_table) {
        const unsigned grid = (unsigned)ceil_div(desc->n, 256);
        if (df_mode) k_beta0_table<df><<<grid, 256>>>(c, static_cast<df*>(p->tab));
        else k_beta0_table<double><<<grid, 256>>>(c, static_cast<double*>(p->tab));
        e = cudaGetLastError();
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e == cudaSuccess)
        e = df_mode ? set_smem_limits<df>(p->desc.block, p->desc.level_block)
                    : set_smem_limits<double>(p->desc.block, p->desc.level_block);
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan_memory(p);
        delete p;
        return e == cudaErrorMemoryAllocation ? CN_ERR_OOM : CN_ERR_CUDA;
    }
    *out = p;
    return CN_OK;
}

cn_status cn_plan_destroy(cn_plan p) {
    if (!p) return CN_OK;
    cudaDeviceSynchronize();
    free_plan_memory(p);
    delete p;
    return CN_OK;
}

cn_status cn_step(cn_plan p, const void* psi_in, void* psi_out, const double* E_mid, int64_t nsteps, void* stream) {
    if (!p || !psi_in || !psi_out || nsteps < 0) return CN_ERR_INVALID_ARG;
    if (!aligned16(psi_in) || !aligned16(psi_out)) return CN_ERR_INVALID_ARG;
    if (E_mid && (reinterpret_cast<uintptr_t>(E_mid) & 7u)) return CN_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const double2* in = static_cast<const double2*>(psi_in);
    double2* out = static_cast<double2*>(psi_out);
    cudaError_t e = (p->desc.arith == CN_ARITH_DF64) ? cn_steps<df>(p, in, out, E_mid, nsteps, st)
                                                     : cn_steps<double>(p, in, out, E_mid, nsteps, st);
    return cuda_status(e);
}

cn_status cn_step_host(cn_plan p, const void* psi_in_host, void* psi_out_host, const double* E_mid_host,
                       int64_t nsteps, void* stream) {
    if (!p || !psi_in_host || !psi_out_host || nsteps < 0) return CN_ERR_INVALID_ARG;
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
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CN_ERR_OOM : CN_ERR_CUDA;
    }
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
    cudaError_t e = (p->desc.arith == CN_ARITH_DF64) ? solve_arrays<df>(p, s, static_cast<double2*>(x), st)
                                                     : solve_arrays<double>(p, s, static_cast<double2*>(x), st);
    return cuda_status(e);
}

cn_status cn_adjoint_step(cn_plan p, const void* psi_n, const void* psi_np1, const void* lam_np1, void* lam_n,
                          const double* E_mid, double* dLdE, void* stream) {
    if (!p || !psi_n || !psi_np1 || !lam_np1 || !lam_n || !dLdE) return CN_ERR_INVALID_ARG;
    if (!aligned16(psi_n) || !aligned16(psi_np1) || !aligned16(lam_np1) || !aligned16(lam_n)) return CN_ERR_INVALID_ARG;
    if ((reinterpret_cast<uintptr_t>(dLdE) & 7u) || (E_mid && (reinterpret_cast<uintptr_t>(E_mid) & 7u)))
        return CN_ERR_INVALID_ARG;
    const int nparts = 148 * 4;
    cudaError_t e = cudaSuccess;
    if (!p->mu) e = cudaMalloc(&p->mu, sizeof(double2) * (size_t)p->desc.n);
    if (e == cudaSuccess && !p->part) {
        e = cudaMalloc(&p->part, 16 * (size_t)nparts);
        p->part_n = nparts;
    }
    if (e != cudaSuccess) {
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? CN_ERR_OOM : CN_ERR_CUDA;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    CNStep s;
    s.p = p->cnp;
    s.psi = static_cast<const double2*>(lam_np1);
    s.s = -1;  // implicit matrix T^dagger = 1 - i dt/2 H
    s.e = 0;   // right-hand side lam_{n+1} itself
    s.E_t = E_mid;
    s.E_e = E_mid;
    s.tab = p->tab;
    const bool dfm = p->desc.arith == CN_ARITH_DF64;
    e = dfm ? cn_solve<df>(p, s, p->mu, st) : cn_solve<double>(p, s, p->mu, st);
    if (e != cudaSuccess) return CN_ERR_CUDA;
    if (dfm) {
        k_adjoint_finish<df><<<p->part_n, kAdjThreads, 0, st>>>(
            p->cnp, p->mu, static_cast<const double2*>(lam_np1), static_cast<const double2*>(psi_n),
            static_cast<const double2*>(psi_np1), static_cast<double2*>(lam_n), static_cast<df*>(p->part));
        k_adjoint_sum<df><<<1, 32, 0, st>>>(static_cast<const df*>(p->part), p->part_n, p->desc.dt, dLdE);
    } else {
        k_adjoint_finish<double><<<p->part_n, kAdjThreads, 0, st>>>(
            p->cnp, p->mu, static_cast<const double2*>(lam_np1), static_cast<const double2*>(psi_n),
            static_cast<const double2*>(psi_np1), static_cast<double2*>(lam_n), static_cast<double*>(p->part));
        k_adjoint_sum<double><<<1, 32, 0, st>>>(static_cast<const double*>(p->part), p->part_n, p->desc.dt, dLdE);
    }
    return cuda_status(cudaGetLastError());
}

cn_status cn_field_from_controls(const double* u, int64_t n_controls, double t_final, double t0, double dt,
                                 int64_t nsteps, double* E_mid, void* stream) {
    if (!u || !E_mid || n_controls < 2 || nsteps < 0 || !(t_final > 0.0) || !std::isfinite(t0) ||
        !std::isfinite(dt) || dt == 0.0)
        return CN_ERR_INVALID_ARG;
    if (nsteps == 0) return CN_OK;
    k_hat_field<<<(unsigned)ceil_div(nsteps, 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        u, n_controls, t_final, t0, dt, nsteps, E_mid);
    return cuda_status(cudaGetLastError());
}

cn_status cn_field_grad_to_controls(const double* dLdE, int64_t nsteps, double t_final, double t0, double dt,
                                    int64_t n_controls, double* grad_u, void* stream) {
    if (!dLdE || !grad_u || n_controls < 2 || nsteps < 0 || !(t_final > 0.0) || !std::isfinite(t0) ||
        !(dt > 0.0))
        return CN_ERR_INVALID_ARG;
    k_hat_field_grad<<<(unsigned)ceil_div(n_controls, 128), 128, 0, static_cast<cudaStream_t>(stream)>>>(
        dLdE, nsteps, t_final, t0, dt, n_controls, grad_u);
    return cuda_status(cudaGetLastError());
}

cn_status cn_plan_query(cn_plan p, cn_plan_info* out) {
    if (!p || !out) return CN_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof(*out));
    out->n = p->desc.n;
    out->levels = (int32_t)p->lv.size() - 1;
    if (out->levels + 1 > CN_MAX_LEVELS) return CN_ERR_UNSUPPORTED;
    for (size_t l = 0; l < p->lv.size(); ++l) {
        out->level_rows[l] = p->lv[l].n;
        out->level_block[l] = (l + 1 < p->lv.size()) ? p->lv[l].m : 0;
    }
    out->launches_per_step = 2 * out->levels + 1;
    out->workspace_bytes = p->workspace_bytes;
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
    if (cudaDeviceSynchronize() != cudaSuccess) return CN_ERR_CUDA;
    int h = 0;
    if (cudaMemcpy(&h, p->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CN_ERR_CUDA;
    if (h != 0 && cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return CN_ERR_CUDA;
    return static_cast<cn_status>(h);
}

}  // extern "C"
