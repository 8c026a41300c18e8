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

constexpr int kLevelBlock = 8;  // rows per block on the reduced levels (>= 1)

struct Level {
    int64_t n = 0;            // rows
    int64_t P = 0;            // blocks (joint lines 0..P)
    int m = 0;                // block size
    LevelRow* rows = nullptr; // rows of this level (levels >= 1)
    LevelSlot* slot = nullptr;
    double2* x = nullptr;     // solution of this level (levels >= 1)
};

}  // namespace

struct cn_plan_s {
    cn_desc desc;
    int device = 0;
    std::vector<Level> lv;    // lv[0]: the system itself; lv[L]: solved by the RS stage
    double2* state = nullptr; // n complex128 scratch for the step ping-pong
    int* status = nullptr;    // device status word
    CNParams cnp;
    std::vector<double> cos_a;
    // cn_step_host staging (allocated on first use)
    double2* h_in = nullptr;
    double2* h_out = nullptr;
    double* h_E = nullptr;
    int64_t h_E_cap = 0;
    // kernel timing (cn_plan_profile)
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;   // events owned by the plan
    size_t ev_used = 0;                 // events handed out since the last read
    std::vector<int> rec_class;         // class of record r (events 2r, 2r+1)
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
    if (d->block != 0 && d->block != 4 && d->block != 8 && d->block != 16) return CN_ERR_INVALID_ARG;
    if (d->arith != CN_ARITH_F64 && d->arith != CN_ARITH_DF64) return CN_ERR_INVALID_ARG;
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
    cudaFree(p->status);
    cudaFree(p->h_in);
    cudaFree(p->h_out);
    cudaFree(p->h_E);
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

LevelSource level_source(const Level& L) {
    LevelSource s;
    s.rows = L.rows;
    s.slot = L.slot;
    s.n = L.n;
    s.slot_stride = kThreads;
    return s;
}

// --------------------------------------------------------------- launch helpers
template <class R, class Src>
cudaError_t launch_reduce(const Src& src, const Level& L, const Level& next, int* status, cudaStream_t st) {
    const unsigned grid = grid_for(L.P);
    switch (L.m) {
    case 4: k_reduce<R, 4, Src><<<grid, kThreads, 0, st>>>(src, L.n, L.P, L.m, next.rows, next.slot, status); break;
    case 8: k_reduce<R, 8, Src><<<grid, kThreads, 0, st>>>(src, L.n, L.P, L.m, next.rows, next.slot, status); break;
    case 16: k_reduce<R, 16, Src><<<grid, kThreads, 0, st>>>(src, L.n, L.P, L.m, next.rows, next.slot, status); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

template <class R, class Src>
cudaError_t launch_substitute(const Src& src, const Level& L, const Level& next, double2* x, int* status,
                              cudaStream_t st) {
    const unsigned grid = grid_for(L.P);
    switch (L.m) {
    case 4: k_substitute<R, 4, Src><<<grid, kThreads, 0, st>>>(src, L.n, L.P, L.m, next.x, x, status); break;
    case 8: k_substitute<R, 8, Src><<<grid, kThreads, 0, st>>>(src, L.n, L.P, L.m, next.x, x, status); break;
    case 16: k_substitute<R, 16, Src><<<grid, kThreads, 0, st>>>(src, L.n, L.P, L.m, next.x, x, status); break;
    default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

// The nested N-shaped solve of one system whose level-0 rows come from src0;
// the solution of level 0 is written to x0.
template <class R, class Src0>
cudaError_t nshape_solve(cn_plan p, const Src0& src0, double2* x0, cudaStream_t st) {
    const int L = (int)p->lv.size() - 1;
    cudaError_t e;
    {
        ProfScope ps(p, kProfReduce0, st);
        e = launch_reduce<R>(src0, p->lv[0], p->lv[1], p->status, st);
    }
    if (e != cudaSuccess) return e;
    for (int l = 1; l < L; ++l) {
        ProfScope ps(p, kProfReduceL, st);
        e = launch_reduce<R>(level_source(p->lv[l]), p->lv[l], p->lv[l + 1], p->status, st);
        if (e != cudaSuccess) return e;
    }
    {
        ProfScope ps(p, kProfBase, st);
        k_base<R><<<1, 32, 0, st>>>(level_source(p->lv[L]), p->lv[L].n, p->lv[L].x, p->status);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    for (int l = L - 1; l >= 1; --l) {
        ProfScope ps(p, kProfSubstL, st);
        e = launch_substitute<R>(level_source(p->lv[l]), p->lv[l], p->lv[l + 1], p->lv[l].x, p->status, st);
        if (e != cudaSuccess) return e;
    }
    ProfScope ps(p, kProfSubst0, st);
    return launch_substitute<R>(src0, p->lv[0], p->lv[1], x0, p->status, st);
}

template <class R>
cudaError_t cn_steps(cn_plan p, const double2* in, double2* out, const double* E_mid, int64_t nsteps,
                     cudaStream_t st) {
    const size_t bytes = sizeof(double2) * (size_t)p->desc.n;
    if (nsteps == 0) {
        if (in == out) return cudaSuccess;
        return cudaMemcpyAsync(out, in, bytes, cudaMemcpyDeviceToDevice, st);
    }
    // Step k writes dest(k); the last step writes out; in is never written
    // unless it is out.  Destinations alternate between out and the scratch.
    const double2* src = in;
    bool first_to_out = ((nsteps - 1) % 2) == 0;
    if (in == out && first_to_out) {
        cudaError_t e = cudaMemcpyAsync(p->state, in, bytes, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
        src = p->state;
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        double2* dst = (((nsteps - 1 - k) % 2) == 0) ? out : p->state;
        CNSource s;
        s.p = p->cnp;
        s.psi = src;
        s.sgn_t = 1.0;
        s.sgn_e = -1.0;
        s.E_t = E_mid ? E_mid + k : nullptr;
        s.E_e = s.E_t;
        cudaError_t e = nshape_solve<R>(p, s, dst, st);
        if (e != cudaSuccess) return e;
        src = dst;
    }
    return cudaSuccess;
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
    default: return "unknown status";
    }
}

const char* cn_version(void) { return "cn_b300 0.1 sm_103a"; }

cn_status cn_plan_create(const cn_desc* desc, cn_plan* out) {
    if (!out) return CN_ERR_INVALID_ARG;
    *out = nullptr;
    cn_status v = validate_desc(desc);
    if (v != CN_OK) return v;
    cn_plan p = new (std::nothrow) cn_plan_s();
    if (!p) return CN_ERR_OOM;
    p->desc = *desc;
    if (p->desc.block == 0) p->desc.block = 8;
    if (cudaGetDevice(&p->device) != cudaSuccess) { delete p; return CN_ERR_CUDA; }
    if (desc->pot == CN_POT_COSSERIES && desc->n_cos > 0) p->cos_a.assign(desc->cos_a, desc->cos_a + desc->n_cos);
    p->desc.cos_a = nullptr;

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
        m = kLevelBlock;
        if (n <= kBaseMax) {
            Level B;
            B.n = n;
            p->lv.push_back(B);
            break;
        }
    }
    cudaError_t e = cudaSuccess;
    for (size_t l = 1; l < p->lv.size() && e == cudaSuccess; ++l) {
        Level& L = p->lv[l];
        p->workspace_bytes += (int64_t)(sizeof(LevelRow) + sizeof(double2)) * L.n +
                              (int64_t)sizeof(LevelSlot) * (grid_for(p->lv[l - 1].P) + 1);
        e = cudaMalloc(&L.rows, sizeof(LevelRow) * (size_t)L.n);
        if (e == cudaSuccess) e = cudaMalloc(&L.slot, sizeof(LevelSlot) * (size_t)(grid_for(p->lv[l - 1].P) + 1));
        if (e == cudaSuccess) e = cudaMalloc(&L.x, sizeof(double2) * (size_t)L.n);
        if (e == cudaSuccess) e = cudaMemset(L.slot, 0, sizeof(LevelSlot) * (size_t)(grid_for(p->lv[l - 1].P) + 1));
    }
    p->workspace_bytes += (int64_t)sizeof(double2) * desc->n + (int64_t)sizeof(int);
    if (e == cudaSuccess) e = cudaMalloc(&p->state, sizeof(double2) * (size_t)desc->n);
    if (e == cudaSuccess) e = cudaMalloc(&p->status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(p->status, 0, sizeof(int));
    if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan_memory(p);
        delete p;
        return e == cudaErrorMemoryAllocation ? CN_ERR_OOM : CN_ERR_CUDA;
    }
    CNParams& c = p->cnp;
    std::memset(&c, 0, sizeof(c));
    c.n = desc->n;
    c.dx = desc->dx;
    c.x_min = desc->x_min;
    c.half_dt = 0.5 * desc->dt;
    c.inv_dx2 = 1.0 / (desc->dx * desc->dx);
    c.gamma = desc->dt / (4.0 * desc->dx * desc->dx);
    c.pot = desc->pot;
    c.V0 = desc->V0;
    c.soft_s = desc->soft_s;
    c.n_cos = desc->pot == CN_POT_COSSERIES ? desc->n_cos : 0;
    c.two_pi_over_L = desc->pot == CN_POT_COSSERIES ? 2.0 * 3.14159265358979323846 / desc->L : 0.0;
    for (int k = 0; k < c.n_cos; ++k) c.cos_a[k] = p->cos_a[(size_t)k];
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

cn_status cn_step(cn_plan p, const void* psi_in, void* psi_out, const double* E_mid, int64_t nsteps,
                  void* stream) {
    if (!p || !psi_in || !psi_out || nsteps < 0) return CN_ERR_INVALID_ARG;
    if (!aligned16(psi_in) || !aligned16(psi_out)) return CN_ERR_INVALID_ARG;
    if (E_mid && (reinterpret_cast<uintptr_t>(E_mid) & 7u)) return CN_ERR_INVALID_ARG;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (p->desc.arith == CN_ARITH_DF64)
        e = cn_steps<df>(p, static_cast<const double2*>(psi_in), static_cast<double2*>(psi_out), E_mid, nsteps, st);
    else
        e = cn_steps<double>(p, static_cast<const double2*>(psi_in), static_cast<double2*>(psi_out), E_mid, nsteps, st);
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
    if (e != cudaSuccess) { cudaGetLastError(); return e == cudaErrorMemoryAllocation ? CN_ERR_OOM : CN_ERR_CUDA; }
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

cn_status cn_solve_tridiag(cn_plan p, const void* b, const void* a, const void* c, const void* d, void* x,
                           int64_t n, void* stream) {
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
    cudaError_t e = (p->desc.arith == CN_ARITH_DF64) ? nshape_solve<df>(p, s, static_cast<double2*>(x), st)
                                                     : nshape_solve<double>(p, s, static_cast<double2*>(x), st);
    return cuda_status(e);
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
    if (h != 0) {
        if (cudaMemset(p->status, 0, sizeof(int)) != cudaSuccess) return CN_ERR_CUDA;
    }
    return static_cast<cn_status>(h);
}

}  // extern "C"
