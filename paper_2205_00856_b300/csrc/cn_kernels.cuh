// cn_kernels.cuh -- N-shaped partition method kernels (reduction, substitution,
// RS stage) for complex tridiagonal systems and for the Crank-Nicolson step of
// the 1D TDSE.
//
// Method (Lutsyshyn, Navarrete, Bauer, "The N-shaped partition method", Sec. 4):
// the rows 0..n-1 of a level are cut into blocks by the joint lines
//   J_t = min(t m, n - 1 - 2 (P - t)),  t = 0..P,  P = ceil((n - 1) / m),
// so every block spans 2..m rows between its joint lines (at least one
// interior row).  One GPU thread owns one block and runs Table 1 on it in
// registers, in the order (RD + JD) + (RU + JU) of Sec. 5.2.1.  The two
// contributions every joint line receives (the paper's atomic additions) are
// exchanged through shared memory, or through a per-CTA slot in global memory
// for the first row of each CTA range, and added in a fixed order (the "two
// extra memory elements per joint line" of Sec. 4.1.3), so every result is
// deterministic.  The joint lines form the reduced tridiagonal system of the
// next level, which is reduced again by the same kernels (Eq. iteration) until
// it is small enough for the serial RS stage (Table 1).  The SS stage then
// returns level by level.  Instead of keeping the RD/RU fill-in columns in
// memory between the two passes (the paper keeps all 5 n vectors in place),
// the substitution kernel re-solves each block's interior rows with its two
// support values as Dirichlet data (the same equations SS evaluates, Fig. 1f).
//
// Level 0 of a Crank-Nicolson step never reads a matrix: it regenerates the
// diagonal of T = 1 + i dt/2 H(t + dt/2) from V(x) and E(t + dt/2) and forms the
// explicit half-step d = T^dagger psi (Eq. ForwardStep) while it walks its block
// (Sec. 5.3: the explicit step fused into RD).  Its rows are divided by the
// off-diagonal value, which leaves -1 on both off-diagonals:
//   -psi_{j-1} + a~_j psi_j - psi_{j+1} = d^_j,
//   a~_j = bt_j - i s g~,  bt_j = 2 + 2 dx^2 V_j,  g~ = 4 dx^2 / dt,
// for T_s = 1 + i s dt/2 H (s = +1: T; s = -1: T^dagger); any row scaling leaves
// the solution unchanged.
#pragma once
#include "cn_arith.cuh"

namespace cnb {

constexpr int kThreads = 128;  // threads per CTA of the reduce / substitute kernels
constexpr int kMaxCos = 16;    // cos-series terms held in the kernel parameters
constexpr int kBaseMax = 16;   // largest reduced system solved by the serial RS stage

// joint line t of a level with n rows, block size m and P blocks
__host__ __device__ __forceinline__ int64_t joint_line(int64_t t, int64_t P, int64_t m, int64_t n) {
    int64_t a = t * m, b = n - 1 - 2 * (P - t);
    return a < b ? a : b;
}

constexpr int kStatusNonfinite = 6;  // cn_status CN_ERR_NONFINITE

// Row predicates of a block with gap g (rows 0..g) as bit masks.  Loops over
// the rows are fully unrolled and test bits instead of comparing k with g: a
// comparison lets the compiler shorten the loop to a run-time trip count,
// which stops the unrolling and moves the per-row arrays to local memory.
struct RowMask {
    unsigned all;      // rows 0..g
    unsigned inner;    // interior rows 1..g-1
    unsigned last_in;  // row g-1
    unsigned ru;       // rows 1..g-2 (RU rows)
    unsigned joint1;   // row g
    __device__ __forceinline__ explicit RowMask(int g)
        : all((2u << g) - 1u), inner((1u << g) - 2u), last_in(1u << (g - 1)), ru((1u << (g - 1)) - 2u),
          joint1(1u << g) {}
};
__device__ __forceinline__ bool bit(unsigned m, int k) { return (m >> k) & 1u; }

__device__ __forceinline__ void flag_error(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ reduced rows
// Row {b, a, c, d} of a reduced system (levels >= 1), stored in the compute type.
template <class R> struct LevelRow {
    typename Store<R>::T b, a, c, d;
};
template <class R> struct LevelSlot {
    typename Store<R>::T b, a, d;
};
template <class R> struct JDPart {
    cx<R> b, a, d;
};

// ------------------------------------------------------------------ generic sources
// A source yields rows k = k0..k1 (k0 = 0 or 1, k1 = g or g-1) of the block
// starting at J0: lower b_k, diagonal a_k, upper c_k, rhs d_k, with b = 0 on
// row 0 of the level and c = 0 on its last row.

// General tridiagonal system in four complex128 arrays (cn_solve_tridiag).
struct ArraySource {
    const double2 *b, *a, *c, *d;
    int64_t n;
    template <class R, int M, bool kInterior>
    __device__ __forceinline__ void load(int64_t J0, int g, cx<R>* B, cx<R>* A, cx<R>* C, cx<R>* D) const {
        const RowMask rm(g);
        const unsigned use = kInterior ? rm.inner : rm.all;
#pragma unroll
        for (int k = kInterior ? 1 : 0; k <= M; ++k) {
            if (bit(use, k)) {
                int64_t i = J0 + k;
                B[k] = (i > 0) ? load128<R>(b + i) : czero<R>();
                A[k] = load128<R>(a + i);
                C[k] = (i < n - 1) ? load128<R>(c + i) : czero<R>();
                D[k] = load128<R>(d + i);
            }
        }
    }
};

// Reduced system of a level >= 1, plus the contribution of the previous CTA's
// last block to the first row of every CTA range (slot).
template <class R> struct LevelSource {
    const LevelRow<R>* rows;
    const LevelSlot<R>* slot;
    int64_t n;            // rows of this level
    int64_t slot_stride;  // rows per CTA range of the producing kernel
    template <class RR, int M, bool kInterior>
    __device__ __forceinline__ void load(int64_t J0, int g, cx<R>* B, cx<R>* A, cx<R>* C, cx<R>* D) const {
        const unsigned use = (M == 0) ? 1u : (kInterior ? RowMask(g).inner : RowMask(g).all);
#pragma unroll
        for (int k = kInterior ? 1 : 0; k <= M; ++k) {
            if (bit(use, k)) {
                int64_t i = J0 + k;
                const LevelRow<R>* r = rows + i;
                B[k] = sload(&r->b);
                A[k] = sload(&r->a);
                C[k] = sload(&r->c);
                D[k] = sload(&r->d);
                if (i > 0 && i < n - 1 && (i % slot_stride) == 0) {
                    const LevelSlot<R>* s = slot + i / slot_stride;
                    B[k] = sload(&s->b);
                    A[k] = cadd(A[k], sload(&s->a));
                    D[k] = cadd(D[k], sload(&s->d));
                }
            }
        }
    }
};

// ------------------------------------------------------------------ output of a block
// Writes row t of the next level from this block's JU part and (via shared
// memory or the CTA slot) the previous block's JD part; the last block also
// writes row P.
template <class R>
__device__ __forceinline__ void write_reduced_row(bool active, int64_t t, int64_t P, JDPart<R> jd, cx<R> A0, cx<R> D0,
                                                  cx<R> JUa, cx<R> JUc, cx<R> JUd, cx<R> Ag, cx<R> Dg,
                                                  LevelRow<R>* out, LevelSlot<R>* out_slot) {
    __shared__ JDPart<R> xch[kThreads];
    const int tid = threadIdx.x;
    xch[tid] = jd;
    __syncthreads();
    if (!active) return;
    LevelRow<R> row;
    if (tid > 0) {
        JDPart<R> pj = xch[tid - 1];
        sstore(&row.b, pj.b);
        sstore(&row.a, cadd(A0, cadd(pj.a, JUa)));
        sstore(&row.d, cadd(D0, cadd(pj.d, JUd)));
    } else {
        // t == 0: no block above; otherwise the previous CTA's slot completes the row
        sstore(&row.b, czero<R>());
        sstore(&row.a, cadd(A0, JUa));
        sstore(&row.d, cadd(D0, JUd));
    }
    sstore(&row.c, JUc);
    out[t] = row;
    if (t == P - 1) {
        LevelRow<R> last;
        sstore(&last.b, jd.b);
        sstore(&last.a, cadd(Ag, jd.a));
        sstore(&last.c, czero<R>());
        sstore(&last.d, cadd(Dg, jd.d));
        out[P] = last;
    } else if (tid == kThreads - 1) {
        LevelSlot<R> s;
        sstore(&s.b, jd.b);
        sstore(&s.a, jd.a);
        sstore(&s.d, jd.d);
        out_slot[blockIdx.x + 1] = s;
    }
}

// ------------------------------------------------------------------ generic reduction
// One thread per block: Table 1 RD + JD, then RU + JU.
template <class R, int M, class Src>
__global__ void __launch_bounds__(kThreads)
k_reduce(Src src, int64_t n, int64_t P, int m, LevelRow<R>* out, LevelSlot<R>* out_slot, int* status) {
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = t < P;
    bool ok = true;
    cx<R> JUa = czero<R>(), JUc = czero<R>(), JUd = czero<R>(), A0 = czero<R>(), D0 = czero<R>();
    cx<R> Ag = czero<R>(), Dg = czero<R>();
    JDPart<R> jd;
    jd.b = czero<R>(); jd.a = czero<R>(); jd.d = czero<R>();
    if (active) {
        const int64_t J0 = joint_line(t, P, m, n);
        const int g = (int)(joint_line(t + 1, P, m, n) - J0);
        const RowMask rm(g);
        cx<R> B[M + 1], A[M + 1], C[M + 1], D[M + 1], W[M + 1];
        src.template load<R, M, false>(J0, g, B, A, C, D);
        A0 = A[0];
        D0 = D[0];
        // RD: r_k = -b_k / a_{k-1}; b_k = r b_{k-1}; a_k += r c_{k-1}; d_k += r d_{k-1}
        W[1] = crcp(A[1], ok);
#pragma unroll
        for (int k = 2; k < M; ++k) {
            if (bit(rm.inner, k)) {
                cx<R> r = cneg(cmul(B[k], W[k - 1]));
                B[k] = cmul(r, B[k - 1]);
                A[k] = cfma(A[k], r, C[k - 1]);
                D[k] = cfma(D[k], r, D[k - 1]);
                W[k] = crcp(A[k], ok);
            }
        }
        // JD on row J_{t+1} (k = g)
#pragma unroll
        for (int k = 2; k <= M; ++k) {
            if (bit(rm.joint1, k)) {
                cx<R> r = cneg(cmul(B[k], W[k - 1]));
                jd.b = cmul(r, B[k - 1]);
                jd.a = cmul(r, C[k - 1]);
                jd.d = cmul(r, D[k - 1]);
                Ag = A[k];
                Dg = D[k];
            }
        }
        // RU: r_k = -c_k / a_{k+1}; b_k += r b_{k+1}; c_k = r c_{k+1}; d_k += r d_{k+1}
        cx<R> nb = czero<R>(), nc = czero<R>(), nd = czero<R>();
#pragma unroll
        for (int k = M - 1; k >= 1; --k) {
            if (bit(rm.last_in, k)) {
                nb = B[k]; nc = C[k]; nd = D[k];
            } else if (bit(rm.ru, k)) {
                cx<R> r = cneg(cmul(C[k], W[k + 1]));
                nb = cfma(B[k], r, nb);
                nc = cmul(r, nc);
                nd = cfma(D[k], r, nd);
            }
        }
        // JU on row J_t (k = 0) with row 1 after RU
        cx<R> r = cneg(cmul(C[0], W[1]));
        JUc = cmul(r, nc);
        JUa = cmul(r, nb);
        JUd = cmul(r, nd);
    }
    write_reduced_row<R>(active, t, P, jd, A0, D0, JUa, JUc, JUd, Ag, Dg, out, out_slot);
    if (!ok) flag_error(status, kStatusNonfinite);
}

// ------------------------------------------------------------------ generic substitution
// One thread per block: the interior rows with the support values xL (row 0)
// and xR (row g) known form a tridiagonal system, solved by Thomas (Sec. 2).
template <class XT, class R> __device__ __forceinline__ void put(XT* p, cx<R> z);
template <> __device__ __forceinline__ void put<double2, double>(double2* p, cx<double> z) { store128(p, z); }
template <> __device__ __forceinline__ void put<double2, df>(double2* p, cx<df> z) { store128(p, z); }
template <> __device__ __forceinline__ void put<float4, df>(float4* p, cx<df> z) { sstore(p, z); }

template <class R, int M, class Src, class XT>
__global__ void __launch_bounds__(kThreads)
k_substitute(Src src, int64_t n, int64_t P, int m, const typename Store<R>::T* x_next, XT* x, int* status) {
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= P) return;
    bool ok = true;
    const int64_t J0 = joint_line(t, P, m, n);
    const int g = (int)(joint_line(t + 1, P, m, n) - J0);
    const RowMask rm(g);
    cx<R> B[M + 1], A[M + 1], C[M + 1], D[M + 1];
    src.template load<R, M, true>(J0, g, B, A, C, D);
    const cx<R> xL = sload(x_next + t);
    const cx<R> xR = sload(x_next + t + 1);
    cx<R> Z[M + 1], CP[M + 1];
    cx<R> zp = czero<R>(), cpp = czero<R>();
#pragma unroll
    for (int k = 1; k < M + 1; ++k) {
        if (bit(rm.inner, k)) {
            cx<R> rhs = D[k];
            if (k == 1) rhs = csub(rhs, cmul(B[1], xL));
            if (bit(rm.last_in, k)) rhs = csub(rhs, cmul(C[k], xR));
            cx<R> piv = (k == 1) ? A[1] : csub(A[k], cmul(B[k], cpp));
            cx<R> w = crcp(piv, ok);
            cx<R> z = (k == 1) ? cmul(rhs, w) : cmul(csub(rhs, cmul(B[k], zp)), w);
            cx<R> cp = cmul(C[k], w);
            Z[k] = z;
            CP[k] = cp;
            zp = z;
            cpp = cp;
        }
    }
    cx<R> y = czero<R>();
#pragma unroll
    for (int k = M; k >= 1; --k) {
        if (bit(rm.last_in, k)) {
            y = Z[k];
            put<XT, R>(x + J0 + k, y);
        } else if (bit(rm.ru, k)) {
            y = csub(Z[k], cmul(CP[k], y));
            put<XT, R>(x + J0 + k, y);
        }
    }
    put<XT, R>(x + J0, xL);
    if (t == P - 1) put<XT, R>(x + J0 + g, xR);
    if (!ok) flag_error(status, kStatusNonfinite);
}

// ------------------------------------------------------------------ RS stage
// Serial Thomas elimination of the last reduced system (Table 1, RS), one thread.
template <class R>
__global__ void k_base(LevelSource<R> src, int64_t n, typename Store<R>::T* x, int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool ok = true;
    cx<R> a_prev = czero<R>(), c_prev = czero<R>(), d_prev = czero<R>();
    cx<R> A[kBaseMax], C[kBaseMax], D[kBaseMax];
    for (int64_t w = 0; w < n; ++w) {
        cx<R> b, a, c, d;
        src.template load<R, 0, false>(w, 0, &b, &a, &c, &d);
        if (w > 0) {
            // r = -b_w / a_{w-1};  a_w += r c_{w-1};  d_w += r d_{w-1}
            cx<R> r = cneg(cmul(b, crcp(a_prev, ok)));
            a = cfma(a, r, c_prev);
            d = cfma(d, r, d_prev);
        }
        A[w] = a; C[w] = c; D[w] = d;
        a_prev = a; c_prev = c; d_prev = d;
    }
    cx<R> y = cmul(D[n - 1], crcp(A[n - 1], ok));
    sstore(x + n - 1, y);
    for (int64_t w = n - 2; w >= 0; --w) {
        y = cmul(csub(D[w], cmul(C[w], y)), crcp(A[w], ok));
        sstore(x + w, y);
    }
    if (!ok) flag_error(status, kStatusNonfinite);
}

// ------------------------------------------------------------------ CN level 0
struct CNParams {
    int64_t n;
    double dx, x_min;
    double c1;             // 2 dx^2:  bt_j = 2 + c1 V_j
    double gt;             // 4 dx^2 / dt
    int pot;               // cn_pot_kind
    int n_cos;
    const double* V0;      // CN_POT_ARRAY (on-the-fly FP64 path)
    double soft_s;
    double two_pi_over_L;
    double cos_a[kMaxCos];
};

// Static potential Vs(x_j) in binary64 (the FP64 path and the table builder).
__device__ __forceinline__ double static_potential_d(const CNParams& p, int64_t j, double x) {
    switch (p.pot) {
    case 1: return p.V0[j];
    case 2: return -rsqrt(fma(x, x, p.soft_s));
    case 3: {
        double v = 0.0;
        for (int k = 0; k < p.n_cos; ++k) v = fma(p.cos_a[k], cos(p.two_pi_over_L * (double)(k + 1) * x), v);
        return v;
    }
    default: return 0.0;
    }
}

// bt0_j = 2 + c1 Vs(x_j): the static part of the scaled diagonal, tabulated once
// per plan when the potential is not regenerated on the fly.
template <class R>
__global__ void k_beta0_table(CNParams p, R* tab) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= p.n) return;
    double x = fma((double)j, p.dx, p.x_min);
    tab[j] = RealOps<R>::from_d(fma(p.c1, static_potential_d(p, j, x), 2.0));
}

// Per-thread coefficient generator walking rows J0, J0+1, ...: returns bt_j for
// the field values E_t (implicit matrix) and E_e (explicit matrix).
template <class R> struct CoefGen;

template <> struct CoefGen<double> {
    const CNParams* p;
    const double* tab;
    double c1Et, c1Ee, x;
    int64_t j;
    __device__ __forceinline__ void init(const CNParams& pp, const double* tb, double Et, double Ee, int64_t j0) {
        p = &pp; tab = tb; j = j0;
        c1Et = pp.c1 * Et; c1Ee = pp.c1 * Ee;
        x = fma((double)j0, pp.dx, pp.x_min);
    }
    // bt for row j (then advance)
    __device__ __forceinline__ void next(double& bt_t, double& bt_e) {
        double b0 = tab ? tab[j] : fma(p->c1, static_potential_d(*p, j, x), 2.0);
        bt_t = fma(c1Et, x, b0);
        bt_e = (c1Ee == c1Et) ? bt_t : fma(c1Ee, x, b0);
        ++j;
        x = fma((double)j, p->dx, p->x_min);
    }
    __device__ __forceinline__ void skip() { ++j; x = fma((double)j, p->dx, p->x_min); }
};

template <> struct CoefGen<df> {
    const df* tab;
    df c1Et, c1Ee, x, dx, c1, soft_s;
    int pot;
    bool same;  // E_e == E_t: one diagonal serves both matrices
    int64_t j;
    __device__ __forceinline__ void init(const CNParams& pp, const df* tb, double Et, double Ee, int64_t j0) {
        tab = tb; j = j0; pot = pp.pot;
        same = (Et == Ee);
        c1Et = df_from_double(pp.c1 * Et);
        c1Ee = df_from_double(pp.c1 * Ee);
        dx = df_from_double(pp.dx);
        c1 = df_from_double(pp.c1);
        soft_s = df_from_double(pp.soft_s);
        // x_j0 = x_min + j0 dx with j0 = hi 2^16 + lo split into exact binary32 parts
        df xm = df_from_double(pp.x_min);
        float jh = (float)(j0 >> 16), jl = (float)(j0 & 0xFFFF);
        x = df_add(xm, df_add(df_mul_f(df_mul_f(dx, jh), 65536.0f), df_mul_f(dx, jl)));
    }
    __device__ __forceinline__ void next(df& bt_t, df& bt_e) {
        df b0;
        if (tab) {
            b0 = tab[j];
        } else if (pot == 2) {
            // bt0 = 2 - c1 / sqrt(x^2 + s)
            df q = df_add(df_mul(x, x), soft_s);
            b0 = df_add_f(df_neg(df_mul(c1, df_rsqrt(q))), 2.0f);
        } else {
            b0 = df_make(2.0f, 0.0f);
        }
        bt_t = df_add(b0, df_mul(c1Et, x));
        bt_e = same ? bt_t : df_add(b0, df_mul(c1Ee, x));
        ++j;
        x = df_add(x, dx);
    }
    __device__ __forceinline__ void skip() { ++j; x = df_add(x, dx); }
};

// Scaled explicit row: d^ = (e s)(bt_e psi - sigma) - i s g~ psi, sigma = psi_{j-1} + psi_{j+1}.
__device__ __forceinline__ cx<double> explicit_row(cx<double> pm, cx<double> p0, cx<double> pp, double bte,
                                                   double es, double sg) {
    double sr = pm.re + pp.re, si = pm.im + pp.im;
    double eb = es * bte;
    return mk(fma(eb, p0.re, fma(sg, p0.im, -es * sr)), fma(eb, p0.im, fma(-sg, p0.re, -es * si)));
}
__device__ __forceinline__ cx<df> explicit_row(cx<df> pm, cx<df> p0, cx<df> pp, df bte, double es, df sg) {
    df sr = df_add(pm.re, pp.re), si = df_add(pm.im, pp.im);
    df eb = es > 0 ? bte : df_neg(bte);
    df nsr = es > 0 ? df_neg(sr) : sr;
    df nsi = es > 0 ? df_neg(si) : si;
    return mk(df_dot2_add(nsr, eb, p0.re, sg, p0.im), df_dot2_add(nsi, eb, p0.im, df_neg(sg), p0.re));
}

template <class R> struct CNTypes;
template <> struct CNTypes<double> { typedef double real; };
template <> struct CNTypes<df> { typedef df real; };

// Level-0 CN source: sign s of the implicit matrix, sign e of the explicit one,
// fields read from device memory (NULL: 0).
struct CNStep {
    CNParams p;
    const double2* psi;   // state the explicit half-step is applied to
    double s, e;          // T_s = 1 + i s dt/2 H(E_t);  explicit S_e = 1 + i e dt/2 H(E_e)
    const double* E_t;
    const double* E_e;
    const void* tab;      // bt0 table in the compute type, or NULL (regenerate)
};

template <class R>
__device__ __forceinline__ R rconst(double v);
template <> __device__ __forceinline__ double rconst<double>(double v) { return v; }
template <> __device__ __forceinline__ df rconst<df>(double v) { return df_from_double(v); }

// One thread per block at level 0 of a CN step: coefficients + explicit
// half-step + Table 1 (RD + JD, RU + JU) on the scaled rows (off-diagonals -1).
template <class R, int M>
__global__ void __launch_bounds__(kThreads)
k_cn_reduce(CNStep st, int64_t P, int m, LevelRow<R>* out, LevelSlot<R>* out_slot, int* status) {
    const int64_t n = st.p.n;
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    const bool active = t < P;
    bool ok = true;
    cx<R> JUa = czero<R>(), JUc = czero<R>(), JUd = czero<R>(), A0 = czero<R>(), D0 = czero<R>();
    cx<R> Ag = czero<R>(), Dg = czero<R>();
    JDPart<R> jd;
    jd.b = czero<R>(); jd.a = czero<R>(); jd.d = czero<R>();
    if (active) {
        const int64_t J0 = joint_line(t, P, m, n);
        const int g = (int)(joint_line(t + 1, P, m, n) - J0);
        const bool last = (t == P - 1);
        const double Et = st.E_t ? *st.E_t : 0.0, Ee = st.E_e ? *st.E_e : 0.0;
        const R sg = rconst<R>(st.s * st.p.gt);        // s g~
        const R msg = rconst<R>(-st.s * st.p.gt);      // imaginary part of a~
        const double es = st.e * st.s;
        CoefGen<R> cg;
        cg.init(st.p, (const R*)st.tab, Et, Ee, J0);
        cx<R> pm = (J0 > 0) ? load128<R>(st.psi + J0 - 1) : czero<R>();
        cx<R> p0 = load128<R>(st.psi + J0);
        const RowMask rm(g);
        const unsigned need = last ? rm.all : (rm.all & ~rm.joint1);  // rows with coefficients
        cx<R> D[M + 1], W[M + 1], BT[M + 1];
        R AT[M + 1];  // real part of a~ (bt_t)
#pragma unroll
        for (int k = 0; k <= M; ++k) {
            if (bit(rm.all, k)) {
                cx<R> pp = (J0 + k + 1 < n) ? load128<R>(st.psi + J0 + k + 1) : czero<R>();
                if (bit(need, k)) {
                    R bt, be;
                    cg.next(bt, be);
                    AT[k] = bt;
                    D[k] = explicit_row(pm, p0, pp, be, es, sg);
                }
                pm = p0;
                p0 = pp;
            }
        }
        A0 = mk(AT[0], msg);
        D0 = D[0];
        // RD (b_k = c_k = -1): w = 1/a; a_k -= w_{k-1}; d_k += w_{k-1} d_{k-1}; b~_k = w_{k-1} b~_{k-1}
        W[1] = crcp(mk(AT[1], msg), ok);
#pragma unroll
        for (int k = 2; k < M; ++k) {
            if (bit(rm.inner, k)) {
                cx<R> a = csub(mk(AT[k], msg), W[k - 1]);
                W[k] = crcp(a, ok);
                D[k] = cfma(D[k], W[k - 1], D[k - 1]);
                BT[k] = (k == 2) ? W[1] : cmul(W[k - 1], BT[k - 1]);
            }
        }
        // JD on row J_{t+1}: b = -w_{g-1} b~_{g-1}, a += -w_{g-1}, d += w_{g-1} d_{g-1}
#pragma unroll
        for (int k = 2; k <= M; ++k) {
            if (bit(rm.joint1, k)) {
                jd.b = (k == 2) ? cneg(W[1]) : cneg(cmul(W[k - 1], BT[k - 1]));
                jd.a = cneg(W[k - 1]);
                jd.d = cmul(W[k - 1], D[k - 1]);
                if (last) {
                    Ag = mk(AT[k], msg);
                    Dg = D[k];
                }
            }
        }
        // RU: b~_k += w_{k+1} b~_{k+1}; c~_k = w_{k+1} c~_{k+1}; d_k += w_{k+1} d_{k+1}
        const cx<R> one = cfrom<R>(1.0, 0.0);
        cx<R> nb = one, nc = one, nd = czero<R>();
#pragma unroll
        for (int k = M - 1; k >= 1; --k) {
            if (bit(rm.last_in, k)) {
                nb = (k == 1) ? one : BT[k];
                nc = one;
                nd = D[k];
            } else if (bit(rm.ru, k)) {
                nb = (k == 1) ? cfma(one, W[k + 1], nb) : cfma(BT[k], W[k + 1], nb);
                nc = bit(rm.last_in, k + 1) ? W[k + 1] : cmul(W[k + 1], nc);
                nd = cfma(D[k], W[k + 1], nd);
            }
        }
        // JU on row J_t with row 1 after RU: c = -w_1 c~_1, a += -w_1 b~_1, d += w_1 d_1
        JUc = cneg(cmul(W[1], nc));
        JUa = cneg(cmul(W[1], nb));
        JUd = cmul(W[1], nd);
    }
    write_reduced_row<R>(active, t, P, jd, A0, D0, JUa, JUc, JUd, Ag, Dg, out, out_slot);
    if (!ok) flag_error(status, kStatusNonfinite);
}

// One thread per block at level 0: the interior rows with the support values
// from level 1 as Dirichlet data, by Thomas on the scaled rows:
//   a_1 = a~_1, a_k = a~_k - w_{k-1}, w = 1/a, z_k = (d^_k + z_{k-1}) w_k
//   (z_0 = xL, xR added on the last interior row), y_k = z_k + w_k y_{k+1}.
template <class R, int M>
__global__ void __launch_bounds__(kThreads)
k_cn_substitute(CNStep st, int64_t P, int m, const typename Store<R>::T* x_next, double2* x, int* status) {
    const int64_t n = st.p.n;
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= P) return;
    bool ok = true;
    const int64_t J0 = joint_line(t, P, m, n);
    const int g = (int)(joint_line(t + 1, P, m, n) - J0);
    const double Et = st.E_t ? *st.E_t : 0.0, Ee = st.E_e ? *st.E_e : 0.0;
    const R sg = rconst<R>(st.s * st.p.gt);
    const R msg = rconst<R>(-st.s * st.p.gt);
    const double es = st.e * st.s;
    const cx<R> xL = sload(x_next + t);
    const cx<R> xR = sload(x_next + t + 1);
    CoefGen<R> cg;
    cg.init(st.p, (const R*)st.tab, Et, Ee, J0);
    cg.skip();
    cx<R> pm = load128<R>(st.psi + J0);
    cx<R> p0 = load128<R>(st.psi + J0 + 1);
    const RowMask rm(g);
    cx<R> W[M + 1], Z[M + 1];
    cx<R> zp = xL;
#pragma unroll
    for (int k = 1; k < M; ++k) {
        if (bit(rm.inner, k)) {
            cx<R> pp = load128<R>(st.psi + J0 + k + 1);  // row J0+g exists
            R bt, be;
            cg.next(bt, be);
            cx<R> d = explicit_row(pm, p0, pp, be, es, sg);
            cx<R> a = (k == 1) ? mk(bt, msg) : csub(mk(bt, msg), W[k - 1]);
            W[k] = crcp(a, ok);
            cx<R> rhs = cadd(d, zp);
            if (bit(rm.last_in, k)) rhs = cadd(rhs, xR);
            zp = cmul(rhs, W[k]);
            Z[k] = zp;
            pm = p0;
            p0 = pp;
        }
    }
    cx<R> y = czero<R>();
#pragma unroll
    for (int k = M - 1; k >= 1; --k) {
        if (bit(rm.last_in, k)) {
            y = Z[k];
            store128(x + J0 + k, y);
        } else if (bit(rm.ru, k)) {
            y = cfma(Z[k], W[k], y);
            store128(x + J0 + k, y);
        }
    }
    store128(x + J0, xL);
    if (t == P - 1) store128(x + J0 + g, xR);
    if (!ok) flag_error(status, kStatusNonfinite);
}

}  // namespace cnb
