// Level 0 of few long blocks: one CTA per block, prefix scans.
//
// The paper's own partition of its small case (n = 4096 in P = 16 blocks of 256
// rows, Sec. 4.1.1) walks each block with one thread.  On B300 every dependent
// binary64 operation costs a warp ~64 clocks, so a 256-row walk is ~0.7 M clocks
// per step however few blocks there are.  Here the threads of a CTA share one
// block's rows (about kScanRowsPerThread consecutive rows each) and every
// recurrence of Table 1's RD/RU on the block and of its SS becomes a prefix scan:
//   pivots       w_k = 1 / (a~_k - w_{k-1}), w_0 = 0: a Moebius map of w_{k-1},
//                composed as the 2x2 matrices F_k = [[0, 1], [-1, a~_k]]
//                (w_k = num / den of F_k ... F_1 (0, 1)^T);
//   RD's d       d_k = d^_k + w_{k-1} d_{k-1}: affine maps y -> w_{k-1} y + d^_k;
//   RU's Q       Q_k = Q_{k-1} w_k (k >= 2, Q_1 = 1): products;
//   RU's sums    S = sum_{k>=2} Q_k Q_{k-1},  d_1 + sum_{k>=2} Q_k d_k: reductions;
//   SS           z_k = (d^_k + z_{k-1}) w_k from z_0 = x_L, then
//                x_k = z_k + w_k x_{k+1} from x_{g-1} = z_{g-1}: affine maps.
// Each thread composes the maps of its rows, a Kogge-Stone scan over the lanes of
// each warp and one over the warps' totals give every thread the composition of
// the rows before its own (after them, for the backward sweep), and each thread
// then re-runs its rows' recurrences from that start value exactly as the
// one-thread kernels do.  The results are those of the one-thread elimination up
// to rounding (the start values of the threads' chains are formed in a different
// order).  Projective matrix products are rescaled by powers of two (exact) so
// that they neither overflow nor vanish.  The level-1 rows take this block's JU
// part; its JD part goes to slot t + 1, one slot per block (the level's
// slot_shift 0), and the reader adds it.  The RS stage of an explicit-depth plan
// runs on one warp when short: parallel cyclic reduction up to 32 rows
// (k_base_pcr), Thomas' recurrences as scans up to 512 (k_base_scan, binary64).
#pragma once
#include "cn_kernels.cuh"

namespace cnb {

constexpr int kScanMinRows = 64;     // level-0 blocks at least this long take the scan kernels
constexpr int kScanMaxRows = 1024;   // ... and at most this long (shared memory per CTA)
constexpr int64_t kScanMaxBlocks = 4096;  // latency regime only: few blocks

template <class T> __device__ __forceinline__ T shfl_word_up(const T& v, int d) {
    static_assert(sizeof(T) % sizeof(int) == 0, "shuffled in 32-bit words");
    constexpr int nw = (int)(sizeof(T) / sizeof(int));
    int w[nw];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < nw; ++i) w[i] = __shfl_up_sync(0xffffffffu, w[i], d);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}
template <class T> __device__ __forceinline__ T shfl_word_down(const T& v, int d) {
    constexpr int nw = (int)(sizeof(T) / sizeof(int));
    int w[nw];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < nw; ++i) w[i] = __shfl_down_sync(0xffffffffu, w[i], d);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}
template <class T> __device__ __forceinline__ T shfl_word_xor(const T& v, int d) {
    constexpr int nw = (int)(sizeof(T) / sizeof(int));
    int w[nw];
    memcpy(w, &v, sizeof(T));
#pragma unroll
    for (int i = 0; i < nw; ++i) w[i] = __shfl_xor_sync(0xffffffffu, w[i], d);
    T r;
    memcpy(&r, w, sizeof(T));
    return r;
}

// magnitude exponent of a complex number and exact scaling by 2^e
__device__ __forceinline__ double mx2(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float mx2(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double cmag(cx<double> z) { return fmax(fabs(z.re), fabs(z.im)); }
__device__ __forceinline__ int mag_exp(double m) { return m > 0.0 ? ilogb(m) : 0; }
__device__ __forceinline__ cx<double> cscale(cx<double> z, int e) { return mk(scalbn(z.re, e), scalbn(z.im, e)); }
__device__ __forceinline__ float cmag(cx<df> z) { return fmaxf(fabsf(z.re.hi), fabsf(z.im.hi)); }
__device__ __forceinline__ int mag_exp(float m) { return m > 0.0f ? ilogbf(m) : 0; }
__device__ __forceinline__ df dscale(df a, int e) { return df_make(ldexpf(a.hi, e), ldexpf(a.lo, e)); }
__device__ __forceinline__ cx<df> cscale(cx<df> z, int e) { return mk(dscale(z.re, e), dscale(z.im, e)); }

// 2x2 complex matrix [[a, b], [c, d]] acting on (w, 1): a projective (Moebius) map
template <class R> struct Mob {
    cx<R> a, b, c, d;
};
template <class R> __device__ __forceinline__ Mob<R> mob_identity() {
    Mob<R> m;
    m.a = m.d = cfrom<R>(1.0, 0.0);
    m.b = m.c = czero<R>();
    return m;
}
// the same map with its entries scaled to a largest magnitude in [1, 2)
template <class R> __device__ __forceinline__ Mob<R> mob_normalize(Mob<R> m) {
    const auto mx = mx2(mx2(cmag(m.a), cmag(m.b)), mx2(cmag(m.c), cmag(m.d)));
    const int e = -mag_exp(mx);
    m.a = cscale(m.a, e);
    m.b = cscale(m.b, e);
    m.c = cscale(m.c, e);
    m.d = cscale(m.d, e);
    return m;
}
// binary64: the largest exponent field and the scaling by integer operations only
// (no binary64 operation: each would cost a warp ~64 clocks of the FP64 pipe)
__device__ __forceinline__ int efield(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }
__device__ __forceinline__ int efield(cx<double> z) { return max(efield(z.re), efield(z.im)); }
// v 2^k by an integer add to the exponent field, exact; zeros, subnormals and
// values that would leave the normal range become signed zeros (entries 2^-1022
// below the matrix's largest, which it then leaves at ~1, contribute nothing)
__device__ __forceinline__ double scale_exp(double v, int k) {
    const uint64_t b = d_bits_opaque(v);
    const int e = (int)((b >> 52) & 0x7ff), e2 = e + k;
    const uint64_t sgn = b & 0x8000000000000000ull;
    if (e == 0 || e2 <= 0) return __longlong_as_double((long long)sgn);
    return __longlong_as_double((long long)((b & 0x800FFFFFFFFFFFFFull) | ((uint64_t)e2 << 52)));
}
template <> __device__ __forceinline__ Mob<double> mob_normalize(Mob<double> m) {
    const int em = min(max(max(efield(m.a), efield(m.b)), max(efield(m.c), efield(m.d))), 2045);
    const int k = 1023 - em;  // the largest entry to [1, 2)
    m.a = mk(scale_exp(m.a.re, k), scale_exp(m.a.im, k));
    m.b = mk(scale_exp(m.b.re, k), scale_exp(m.b.im, k));
    m.c = mk(scale_exp(m.c.re, k), scale_exp(m.c.im, k));
    m.d = mk(scale_exp(m.d.re, k), scale_exp(m.d.im, k));
    return m;
}
// later o earlier: the matrix product L E
template <class R> __device__ __forceinline__ Mob<R> mob_after(const Mob<R>& L, const Mob<R>& E) {
    Mob<R> r;
    r.a = cfma(cmul(L.a, E.a), L.b, E.c);
    r.b = cfma(cmul(L.a, E.b), L.b, E.d);
    r.c = cfma(cmul(L.c, E.a), L.d, E.c);
    r.d = cfma(cmul(L.c, E.b), L.d, E.d);
    return mob_normalize(r);
}
// F_k M, F_k = [[0, 1], [-1, a~_k]]: row k's pivot map after M
template <class R> __device__ __forceinline__ Mob<R> mob_pivot_after(cx<R> at, const Mob<R>& M) {
    Mob<R> r;
    r.a = M.c;
    r.b = M.d;
    r.c = csub(cmul(at, M.c), M.a);
    r.d = csub(cmul(at, M.d), M.b);
    return r;
}

// affine map y -> m y + a
template <class R> struct Aff {
    cx<R> m, a;
};
template <class R> __device__ __forceinline__ Aff<R> aff_identity() {
    Aff<R> f;
    f.m = cfrom<R>(1.0, 0.0);
    f.a = czero<R>();
    return f;
}
template <class R> __device__ __forceinline__ Aff<R> aff_after(const Aff<R>& L, const Aff<R>& E) {
    Aff<R> r;
    r.m = cmul(L.m, E.m);
    r.a = cfma(L.a, L.m, E.a);
    return r;
}
// products of complex numbers, earlier factor first
template <class R> struct Prod {
    cx<R> v;
};
// "L after E" for the three kinds of map, and their identities
template <class R> __device__ __forceinline__ Mob<R> after(const Mob<R>& L, const Mob<R>& E) { return mob_after(L, E); }
template <class R> __device__ __forceinline__ Aff<R> after(const Aff<R>& L, const Aff<R>& E) { return aff_after(L, E); }
template <class R> __device__ __forceinline__ Prod<R> after(const Prod<R>& L, const Prod<R>& E) {
    Prod<R> r;
    r.v = cmul(E.v, L.v);
    return r;
}
template <class R> __device__ __forceinline__ void set_identity(Mob<R>& v) { v = mob_identity<R>(); }
template <class R> __device__ __forceinline__ void set_identity(Aff<R>& v) { v = aff_identity<R>(); }
template <class R> __device__ __forceinline__ void set_identity(Prod<R>& v) { v.v = cfrom<R>(1.0, 0.0); }

// Kogge-Stone scans over the lanes 0 .. width-1 of a warp: "up" composes lane l
// with every lane below it (forward recurrences), "down" with every lane above it
// (backward ones); the exclusive forms give each lane the composition of the
// others' maps only.  The rounds stay a loop: few CTAs run these kernels, each
// fetching its code cold, and unrolled rounds cost more in instruction fetch than
// the loop's few integer instructions (double-float P = 16 step 40 -> 36 us on
// B300, binary64 unchanged).
template <class V> __device__ __forceinline__ V warp_inclusive_up(V v, int lane, int width) {
#pragma unroll 1
    for (int d = 1; d < width; d <<= 1) {
        const V o = shfl_word_up(v, d);
        if (lane >= d) v = after(v, o);
    }
    return v;
}
template <class V> __device__ __forceinline__ V warp_inclusive_down(V v, int lane, int width) {
#pragma unroll 1
    for (int d = 1; d < width; d <<= 1) {
        const V o = shfl_word_down(v, d);
        if (lane + d < width) v = after(v, o);
    }
    return v;
}
template <class V> __device__ __forceinline__ V scan_up_exclusive(V v, int lane) {
    v = warp_inclusive_up(v, lane, 32);
    V x = shfl_word_up(v, 1);
    if (lane == 0) set_identity(x);
    return x;
}
template <class V> __device__ __forceinline__ V scan_down_exclusive(V v, int lane) {
    v = warp_inclusive_down(v, lane, 32);
    V x = shfl_word_down(v, 1);
    if (lane == 31) set_identity(x);
    return x;
}
// The same over the whole CTA (blockDim.x a multiple of 32, a few warps): each
// warp scans its lanes, then composes its exclusive result with the totals of the
// warps before its own, nearest first (after it, for "down").  tot: 32 entries of
// shared memory, free again on return.
template <class V> __device__ __forceinline__ V block_up_exclusive(V v, V* tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_inclusive_up(v, lane, 32);
    V x = shfl_word_up(v, 1);
    if (lane == 0) set_identity(x);
    if (nw == 1) return x;
    if (lane == 31) tot[wid] = v;
    __syncthreads();
    for (int i = wid - 1; i >= 0; --i) x = after(x, tot[i]);  // one composition site
    __syncthreads();
    return x;
}
template <class V> __device__ __forceinline__ V block_down_exclusive(V v, V* tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    v = warp_inclusive_down(v, lane, 32);
    V x = shfl_word_down(v, 1);
    if (lane == 31) set_identity(x);
    if (nw == 1) return x;
    if (lane == 0) tot[wid] = v;
    __syncthreads();
    for (int i = wid + 1; i < nw; ++i) x = after(x, tot[i]);
    __syncthreads();
    return x;
}
template <class R> __device__ __forceinline__ cx<R> warp_sum(cx<R> v) {
#pragma unroll
    for (int d = 16; d >= 1; d >>= 1) v = cadd(v, shfl_word_xor(v, d));
    return v;
}
// two CTA-wide sums, valid in warp 0; tot: 64 entries of shared memory
template <class R> __device__ __forceinline__ void block_sum2(cx<R>& s, cx<R>& u, cx<R>* tot) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    s = warp_sum(s);
    u = warp_sum(u);
    if (nw == 1) return;
    if (lane == 0) {
        tot[wid] = s;
        tot[32 + wid] = u;
    }
    __syncthreads();
    if (wid == 0) {
        s = tot[0];
        u = tot[32];
        for (int i = 1; i < nw; ++i) {
            s = cadd(s, tot[i]);
            u = cadd(u, tot[32 + i]);
        }
    }
}

// Block t's rows 1..g-1 are dealt to the CTA's nt threads in runs of
// c = ceil((g - 1) / nt): thread i takes rows k0 = 1 + i c .. k1 - 1 (none if
// k0 >= g).  Row k's entry in the CTA's shared arrays: thread-interleaved (the
// j-th row of every thread's run side by side), so that a warp's access to its
// threads' rows is conflict-free; row 0 after them.  Arrays hold m + nt entries.
struct ScanRows {
    int gap, c, k0, k1, tid, nt;
    __device__ __forceinline__ explicit ScanRows(int g) : gap(g), tid((int)threadIdx.x), nt((int)blockDim.x) {
        c = (g - 1 + nt - 1) / nt;
        k0 = 1 + tid * c;
        k1 = min(g, k0 + c);
    }
    // any row
    __device__ __forceinline__ int pos(int k) const {
        if (k == 0) return nt * c;
        const int l = (k - 1) / c;
        return (k - 1 - l * c) * nt + l;
    }
    // one of the thread's own rows k0 .. k1 - 1
    __device__ __forceinline__ int own(int k) const { return (k - k0) * nt + tid; }
};
// threads of the CTA that takes one level-0 block of m rows: about kScanRowsPerThread
// rows each, whole warps, at most kScanMaxThreads.  A warp on B300 issues a binary64
// instruction every ~64 clocks whatever its other warps do, and an SM takes about
// four at a time (one per scheduler): the scans' cost is their depth in binary64
// instructions, so four warps, each with its own scheduler, and runs of two rows
// (m = 256 on B300: 59 us a step at 2 rows and 4 warps, 74 at 1 row and 8 warps,
// 70 at 4 rows and 2 warps; m = 512: 72 at 4 warps, 82 at 8, 113 at 16)
constexpr int kScanRowsPerThread = 2;
constexpr int kScanMaxThreads = 128;
__host__ __device__ constexpr int scan_threads(int m) {
    const int t = ((m - 1 + kScanRowsPerThread - 1) / kScanRowsPerThread + 31) / 32 * 32;
    return t < 32 ? 32 : (t > kScanMaxThreads ? kScanMaxThreads : t);
}
// entries of one shared array / one kept field per block
__host__ __device__ constexpr size_t scan_ld(int m) { return (size_t)m + (size_t)scan_threads(m); }
// shared memory of the scan kernels, in storage entries: a~, d^, w, d^RD, Q (reduction)
// or d^, w, z (substitution)
__host__ __device__ constexpr size_t scan_reduce_entries(int m) { return 5 * scan_ld(m); }
__host__ __device__ constexpr size_t scan_subst_entries(int m) { return 3 * scan_ld(m); }
// kept (d^, w) of block t: field j at keep0 + (2 t + j) ld, row k at its shared position
__host__ __device__ constexpr size_t scan_keep_entries(int m, int64_t blocks) { return 2 * scan_ld(m) * (size_t)blocks; }

// Level-0 reduction of block t = blockIdx.x by one CTA: coefficients and explicit
// rows, RD/JD with RU/JU (the scans above), the kept (d^, w) of every interior row,
// and the block's JU part of level-1 row t (JD part to slot t + 1; the system's last
// block writes row P whole).  Same arithmetic per row as cn_reduce_block.
template <class R, int ES>
__global__ void __launch_bounds__(kScanMaxThreads)
k_cn_reduce_scan(CNStep st, OneSys sys, OneSys next, OneGrid grid, int m, int m_next, LevelPlanes<R> out,
                 LevelSlot<R>* out_slot, typename Store<R>::T* keep0, int* status) {
    grid_dep_enter();
    typedef typename Store<R>::T ST;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) unsigned char tot_raw[32 * sizeof(Mob<R>)];
    const int ld = (int)scan_ld(m);
    ST* const sA = reinterpret_cast<ST*>(smem_raw);  // a~_k
    ST* const sD = sA + ld;                           // d^_k
    ST* const sW = sD + ld;                           // w_k, w_0 = 0
    ST* const sR = sW + ld;                           // RD's d_k
    ST* const sQ = sR + ld;                           // RU's Q_k
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x;
    const LvlSys& e = sys.at(0);
    const int64_t n = e.n, P = e.P;
    const int64_t J0 = joint_line(t, P, m, n);
    const ScanRows rw((int)(joint_line(t + 1, P, m, n) - J0));
    const int gap = rw.gap, k0 = rw.k0, k1 = rw.k1;
    ST* const keep = keep0 + 2 * t * ld;
    bool ok = true;
    // scaled rows: a~_k and d^_k (row k0's stencil takes psi_{k0 - 1}: not a joint row)
    if (k0 < k1) {
        CNRowStream<R, ES> rs;
        rs.init(st, e, grid.at(0), J0 + k0);
        rs.pm = rs.ld(J0 + k0 - 1);
        for (int k = k0; k < k1; ++k) {
            cx<R> a, d;
            rs.next(a, d);
            sstore(sA + rw.own(k), a);
            sstore(sD + rw.own(k), d);
        }
    }
    if (tid == 0) sstore(sW + rw.pos(0), czero<R>());
    __syncthreads();
    // RD pivots: w_k = 1 / (a~_k - w_{k-1})
    {
        Mob<R> M = mob_identity<R>();
        for (int k = k0; k < k1; ++k) {
            M = mob_pivot_after(sload(sA + rw.own(k)), M);
            if (((k - k0) & 7) == 7) M = mob_normalize(M);
        }
        const Mob<R> X = block_up_exclusive(mob_normalize(M), reinterpret_cast<Mob<R>*>(tot_raw));
        cx<R> w = cmul(X.b, crcp(X.d, ok));  // w_{k0 - 1}: X applied to (w_0, 1) = (0, 1)
        for (int k = k0; k < k1; ++k) {
            w = crcp(csub(sload(sA + rw.own(k)), w), ok);
            sstore(sW + rw.own(k), w);
        }
    }
    __syncthreads();
    // RD right-hand side: d_k = d^_k + w_{k-1} d_{k-1}
    {
        const cx<R> wk0 = k0 < k1 ? sload(sW + rw.pos(k0 - 1)) : czero<R>();  // w_{k0 - 1}
        Aff<R> F = aff_identity<R>();
        cx<R> wp = wk0;
        for (int k = k0; k < k1; ++k) {
            Aff<R> f;
            f.m = wp;
            f.a = sload(sD + rw.own(k));
            F = aff_after(f, F);
            wp = sload(sW + rw.own(k));
        }
        cx<R> y = block_up_exclusive(F, reinterpret_cast<Aff<R>*>(tot_raw)).a;  // d_{k0 - 1} (d_0 = 0)
        wp = wk0;
        for (int k = k0; k < k1; ++k) {
            y = k == 1 ? sload(sD + rw.own(1)) : cfma(sload(sD + rw.own(k)), wp, y);
            sstore(sR + rw.own(k), y);
            wp = sload(sW + rw.own(k));
        }
    }
    // RU products: Q_1 = 1, Q_k = Q_{k-1} w_k
    {
        Prod<R> F;
        F.v = cfrom<R>(1.0, 0.0);
        for (int k = max(k0, 2); k < k1; ++k) F.v = cmul(F.v, sload(sW + rw.own(k)));
        cx<R> q = block_up_exclusive(F, reinterpret_cast<Prod<R>*>(tot_raw)).v;  // Q_{k0 - 1}
        for (int k = k0; k < k1; ++k) {
            q = k == 1 ? cfrom<R>(1.0, 0.0) : cmul(q, sload(sW + rw.own(k)));
            sstore(sQ + rw.own(k), q);
        }
    }
    __syncthreads();
    // RU sums: S = sum_{k>=2} Q_k Q_{k-1},  nd = d_1 + sum_{k>=2} Q_k d_k
    cx<R> S = czero<R>(), ND = czero<R>();
    {
        cx<R> qp = k0 > 1 && k0 < k1 ? sload(sQ + rw.pos(k0 - 1)) : czero<R>();  // Q_{k0 - 1}
        for (int k = k0; k < k1; ++k) {
            const cx<R> Qk = sload(sQ + rw.own(k));
            if (k == 1) {
                ND = sload(sR + rw.own(1));
            } else {
                S = cfma(S, Qk, qp);
                ND = cfma(ND, Qk, sload(sR + rw.own(k)));
            }
            qp = Qk;
        }
    }
    block_sum2(S, ND, reinterpret_cast<cx<R>*>(tot_raw));
    // the kept values of the substitution
    for (int k = k0; k < k1; ++k) {
        dbg_st(keep + rw.own(k), sD[rw.own(k)]);
        dbg_st(keep + ld + rw.own(k), sW[rw.own(k)]);
    }
    if (!ok) flag_error(status, kStatusNonfinite);
    if (tid != 0) return;
    // JD on row J_{t+1}, JU on row J_t (as cn_reduce_block)
    const cx<R> one = cfrom<R>(1.0, 0.0);
    const cx<R> w1 = sload(sW + rw.pos(1)), wl = sload(sW + rw.pos(gap - 1));
    const cx<R> dl = sload(sR + rw.pos(gap - 1)), Ql = sload(sQ + rw.pos(gap - 1));
    CNRowStream<R, ES> r0;  // row J_t, its own share (psi_{J_t - 1} is the block above's)
    r0.init(st, e, grid.at(0), J0);
    cx<R> A0, D0;
    r0.next(A0, D0);
    const cx<R> wQ = cneg(cmul(w1, Ql));
    JDPart<R> jd;
    jd.b = wQ;
    jd.a = cneg(wl);
    jd.d = cmul(wl, dl);
    if constexpr (ES != 0) {  // this block's part of row J_{t+1}'s term in psi_{J_{t+1} - 1}
        const cx<R> pm = r0.ld(J0 + gap - 1);
        jd.d = ES > 0 ? csub(jd.d, pm) : cadd(jd.d, pm);
    }
    const cx<R> JUc = wQ;
    const cx<R> JUa = cneg(cmul(w1, cfma(one, w1, S)));
    const cx<R> JUd = cmul(w1, ND);
    const RowSink<R> sink(out, next.at(0), m_next);
    sink.put(t, czero<R>(), cadd(A0, JUa), JUc, cadd(D0, JUd));
    if (t == P - 1) {
        cx<R> Ag = czero<R>(), Dg = czero<R>();
        if (st.own_last) {  // row J_P, the system's last: its own share
            CNRowStream<R, ES> rg;
            rg.init(st, e, grid.at(0), J0 + gap);
            rg.next(Ag, Dg);
        }
        sink.put(P, jd.b, cadd(Ag, jd.a), czero<R>(), cadd(Dg, jd.d));
    } else {
        LevelSlot<R> sl;
        sstore(&sl.b, jd.b);
        sstore(&sl.a, jd.a);
        sstore(&sl.d, jd.d);
        dbg_st(&out_slot[t + 1], sl);
    }
}

// Level-0 substitution of block t = blockIdx.x by one CTA from the kept (d^, w):
//   z_k = (d^_k + z_{k-1}) w_k from z_0 = x_L (row g-1 also adds x_R), then
//   x_k = z_k + w_k x_{k+1} from x_{g-1} = z_{g-1}
// (the forward and backward sweeps of k_cn_substitute_kept, as scans).
template <class R>
__global__ void __launch_bounds__(kScanMaxThreads)
k_cn_substitute_scan(OneSys sys, OneSys next, int m, const typename Store<R>::T* keep0,
                     const typename Store<R>::T* x_next0, double2* x_out) {
    grid_dep_enter();
    typedef typename Store<R>::T ST;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(16) unsigned char tot_raw[32 * sizeof(Aff<R>)];
    Aff<R>* const tot = reinterpret_cast<Aff<R>*>(tot_raw);
    const int ld = (int)scan_ld(m);
    ST* const sD = reinterpret_cast<ST*>(smem_raw);
    ST* const sW = sD + ld;
    ST* const sZ = sW + ld;
    const int tid = threadIdx.x;
    const int64_t t = blockIdx.x;
    const LvlSys& e = sys.at(0);
    const int64_t n = e.n, P = e.P;
    const int64_t J0 = joint_line(t, P, m, n);
    const ScanRows rw((int)(joint_line(t + 1, P, m, n) - J0));
    const int gap = rw.gap, k0 = rw.k0, k1 = rw.k1;
    const ST* const keep = keep0 + 2 * t * ld;
    const ST* x_next = x_next0 + next.at(0).row_off;
    const cx<R> xL = sload(x_next + t), xR = sload(x_next + t + 1);
    for (int k = k0; k < k1; ++k) {
        sD[rw.own(k)] = dbg_ld(keep + rw.own(k));
        sW[rw.own(k)] = dbg_ld(keep + ld + rw.own(k));
    }
    // forward sweep
    {
        Aff<R> F = aff_identity<R>();
        for (int k = k0; k < k1; ++k) {
            const cx<R> w = sload(sW + rw.own(k));
            const cx<R> dd = k == gap - 1 ? cadd(sload(sD + rw.own(k)), xR) : sload(sD + rw.own(k));
            Aff<R> f;  // z -> w z + w (d^ (+ x_R))
            f.m = w;
            f.a = cmul(dd, w);
            F = aff_after(f, F);
        }
        const Aff<R> Z = block_up_exclusive(F, tot);
        cx<R> z = cfma(Z.a, Z.m, xL);  // z_{k0 - 1}
        for (int k = k0; k < k1; ++k) {
            const cx<R> w = sload(sW + rw.own(k)), d = sload(sD + rw.own(k));
            z = k == gap - 1 ? cmul(cadd(cadd(d, z), xR), w) : cmul(cadd(d, z), w);
            sstore(sZ + rw.own(k), z);
        }
    }
    __syncthreads();
    // backward sweep over rows g-2 .. 1
    const cx<R> ztop = sload(sZ + rw.pos(gap - 1));
    const int b1 = min(k1, gap - 1);  // the thread's rows below g - 1: k0 .. b1 - 1
    Aff<R> B = aff_identity<R>();
    for (int k = b1 - 1; k >= k0; --k) {
        Aff<R> f;  // y -> w_k y + z_k
        f.m = sload(sW + rw.own(k));
        f.a = sload(sZ + rw.own(k));
        B = aff_after(f, B);
    }
    const Aff<R> Yb = block_down_exclusive(B, tot);
    double2* x = x_out + e.row_off;
    cx<R> y = cfma(Yb.a, Yb.m, ztop);  // x_{b1}
    for (int k = b1 - 1; k >= k0; --k) {
        y = cfma(sload(sZ + rw.own(k)), sload(sW + rw.own(k)), y);
        store128(x + J0 + k, y);
    }
    if (k0 <= gap - 1 && gap - 1 < k1) store128(x + J0 + gap - 1, ztop);
    if (tid == 0) store128(x + J0, xL);
    if (tid == 0 && t == P - 1) store128(x + J0 + gap, xR);
}

}  // namespace cnb

namespace cnb {

// The RS stage of an explicit-depth plan whose last reduced system has at most
// kPcrMax rows: parallel cyclic reduction (Hockney, J. ACM 12(1), 1965) on one
// warp, one row per lane.  In the step with stride s every row eliminates its
// couplings to rows i - s and i + s with those rows' equations,
//   k1 = b_i / a_{i-s},  k2 = c_i / a_{i+s},
//   a_i -= k1 c_{i-s} + k2 b_{i+s},  d_i -= k1 d_{i-s} + k2 d_{i+s},
//   b_i = -k1 b_{i-s},  c_i = -k2 c_{i+s},
// after which it couples to i -+ 2s (a row beyond the system contributes
// nothing); once 2s >= n every row stands alone and x_i = d_i / a_i.  Five steps
// for 17 rows, each ~39 binary64 operations in every lane at once, where Thomas'
// recurrences walk the rows one after another.  Lanes beyond the system hold the
// identity row.
constexpr int kPcrMax = 32;
template <class R> struct PcrRow {
    cx<R> q, b, c, d;  // q = 1 / a
};
template <class R>
__global__ void __launch_bounds__(32)
k_base_pcr(LevelSource<R> src, typename Store<R>::T* x, int* status) {
    grid_dep_enter();
    const int n = (int)src.n, i = threadIdx.x;
    bool ok = true;
    cx<R> a = cfrom<R>(1.0, 0.0), b = czero<R>(), c = czero<R>(), d = czero<R>();
    if (i < n) {
        const Row<R> r = src.template row_at<R>(i);
        a = r.a;
        b = i > 0 ? r.b : czero<R>();
        c = i < n - 1 ? r.c : czero<R>();
        d = r.d;
    }
    for (int s = 1; s < n; s <<= 1) {
        PcrRow<R> me;
        me.q = crcp(a, ok);
        me.b = b;
        me.c = c;
        me.d = d;
        const PcrRow<R> lo = shfl_word_up(me, s), hi = shfl_word_down(me, s);
        const bool has_lo = i >= s, has_hi = i + s < n;
        const cx<R> k1 = has_lo ? cmul(b, lo.q) : czero<R>();
        const cx<R> k2 = has_hi ? cmul(c, hi.q) : czero<R>();
        const cx<R> lb = has_lo ? lo.b : czero<R>(), lc = has_lo ? lo.c : czero<R>();
        const cx<R> ld = has_lo ? lo.d : czero<R>();
        const cx<R> hb = has_hi ? hi.b : czero<R>(), hc = has_hi ? hi.c : czero<R>();
        const cx<R> hd = has_hi ? hi.d : czero<R>();
        a = csub2mul(a, k1, lc, k2, hb);
        d = csub2mul(d, k1, ld, k2, hd);
        b = cneg(cmul(k1, lb));
        c = cneg(cmul(k2, hc));
    }
    const cx<R> xi = cmul(d, crcp(a, ok));
    if (i < n) sstore(x + i, xi);
    if (!ok) flag_error(status, kStatusNonfinite);
}

// The RS stage of a plan whose level 0 runs on warps (explicit depth, last reduced
// system of at most kScanRsMax rows): Thomas' recurrences as warp scans, one warp
//   c'_k = c_k / (a_k - b_k c'_{k-1}):  Moebius maps [[0, c_k], [-b_k, a_k]] of c'_{k-1}
//   z_k = (d_k - b_k z_{k-1}) / m_k:    affine maps;   x_k = z_k - c'_k x_{k+1}: affine maps
// with each lane re-running its rows as k_base_serial does.  Taken in binary64;
// in double-float the one-thread walk is the faster (its dependent operations
// cost a few clocks, not ~64).
constexpr int kScanRsMax = 512;
__host__ __device__ constexpr size_t scan_rs_entries(int n) { return 7 * (size_t)n; }

template <class R>
__global__ void __launch_bounds__(32)
k_base_scan(LevelSource<R> src, typename Store<R>::T* x, int* status) {
    grid_dep_enter();
    typedef typename Store<R>::T ST;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int n = (int)src.n;
    ST* const sa = reinterpret_cast<ST*>(smem_raw);
    ST* const sb = sa + n;
    ST* const sc = sb + n;
    ST* const sd = sc + n;
    ST* const si = sd + n;  // 1 / m_k
    ST* const sp = si + n;  // c'_k
    ST* const sz = sp + n;  // z_k
    const int lane = threadIdx.x;
    const int c = (n + 31) / 32;
    const int k0 = min(n, lane * c), k1 = min(n, k0 + c);
    bool ok = true;
    for (int k = k0; k < k1; ++k) {
        const Row<R> r = src.template row_at<R>(k);
        sstore(sa + k, r.a);
        sstore(sb + k, r.b);
        sstore(sc + k, r.c);
        sstore(sd + k, r.d);
    }
    // pivots and c'
    {
        Mob<R> M = mob_identity<R>();
        for (int k = k0; k < k1; ++k) {
            const cx<R> a = sload(sa + k), b = sload(sb + k), cc = sload(sc + k);
            Mob<R> r;  // [[0, c], [-b, a]] M
            r.a = cmul(cc, M.c);
            r.b = cmul(cc, M.d);
            r.c = csub(cmul(a, M.c), cmul(b, M.a));
            r.d = csub(cmul(a, M.d), cmul(b, M.b));
            M = ((k - k0) & 7) == 7 ? mob_normalize(r) : r;
        }
        const Mob<R> X = scan_up_exclusive(mob_normalize(M), lane);
        cx<R> cp = cmul(X.b, crcp(X.d, ok));  // c'_{k0 - 1} (c'_{-1} = 0)
        for (int k = k0; k < k1; ++k) {
            const cx<R> a = sload(sa + k);
            const cx<R> piv = k == 0 ? a : csub(a, cmul(sload(sb + k), cp));
            const cx<R> iv = crcp(piv, ok);
            cp = cmul(sload(sc + k), iv);
            sstore(si + k, iv);
            sstore(sp + k, cp);
        }
    }
    __syncwarp();
    // z
    {
        Aff<R> F = aff_identity<R>();
        for (int k = k0; k < k1; ++k) {
            const cx<R> iv = sload(si + k);
            Aff<R> f;  // z -> -b iv z + d iv
            f.m = k == 0 ? czero<R>() : cneg(cmul(sload(sb + k), iv));
            f.a = cmul(sload(sd + k), iv);
            F = aff_after(f, F);
        }
        cx<R> z = scan_up_exclusive(F, lane).a;  // z_{k0 - 1}
        for (int k = k0; k < k1; ++k) {
            const cx<R> d = sload(sd + k), iv = sload(si + k);
            z = k == 0 ? cmul(d, iv) : cmul(csub(d, cmul(sload(sb + k), z)), iv);
            sstore(sz + k, z);
        }
    }
    __syncwarp();
    // x, backward from x_{n-1} = z_{n-1}
    const cx<R> ztop = sload(sz + n - 1);
    const int b1 = min(k1, n - 1);
    Aff<R> B = aff_identity<R>();
    for (int k = b1 - 1; k >= k0; --k) {
        Aff<R> f;  // y -> -c' y + z
        f.m = cneg(sload(sp + k));
        f.a = sload(sz + k);
        B = aff_after(f, B);
    }
    const Aff<R> Yb = scan_down_exclusive(B, lane);
    cx<R> y = cfma(Yb.a, Yb.m, ztop);
    for (int k = b1 - 1; k >= k0; --k) {
        y = csub(sload(sz + k), cmul(sload(sp + k), y));
        sstore(x + k, y);
    }
    if (k0 <= n - 1 && n - 1 < k1) sstore(x + n - 1, ztop);
    if (!ok) flag_error(status, kStatusNonfinite);
}

}  // namespace cnb
