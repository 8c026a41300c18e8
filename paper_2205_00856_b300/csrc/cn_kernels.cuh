// cn_kernels.cuh -- N-shaped partition method kernels (reduction, substitution,
// reduced-system solve) for complex tridiagonal systems and the Crank-Nicolson
// step of the 1D TDSE.
//
// Method (Lutsyshyn, Navarrete, Bauer, "The N-shaped partition method", Sec. 4):
// the rows 0..n-1 of a level are cut into blocks by joint lines
//   J_t = min(t m, n - 1 - 2 (P - t)),  t = 0..P,  P = ceil((n - 1) / m),
// so every block has 2..m rows between its joint lines (gap >= 2: at least one
// interior row).  One GPU thread owns one block and runs Table 1 on it in
// registers:
//   RD + JD  (downward elimination, then the contribution to row J_{t+1}),
//   RU + JU  (upward elimination, then the contribution to row J_t),
// in the reordered form (RD + JD) + (RU + JU) of Sec. 5.2.1.  The two
// contributions every joint line receives (the paper's atomic additions) are
// exchanged through shared memory, or through a per-CTA slot in global memory
// for the first row of a CTA, and added in a fixed order (the "two extra memory
// elements per joint line" of Sec. 4.1.3), so results are deterministic.
// The joint lines form the reduced tridiagonal system of the next level, which
// is reduced again by the same kernel (Eq. iteration) until it is small enough
// for the serial RS stage (Table 1, RS).  The SS stage then returns level by
// level: every block's interior rows satisfy a tridiagonal system whose two
// support values are now known; the kernel solves that Dirichlet block system
// directly (the same equations the paper's SS evaluates after RD + RU, Fig. 1f),
// which is cheaper than rebuilding the fill-in columns.
//
// Level 0 of a Crank-Nicolson step regenerates the coefficients of
// T = 1 + i dt/2 H(t + dt/2) from V(x) and E(t + dt/2) and forms the explicit
// half-step d = T^dagger psi (Eq. ForwardStep) while loading, so only psi is
// read from HBM (Sec. 5.3: the explicit step fused into RD).
#pragma once
#include "cn_arith.cuh"

namespace cnb {

constexpr int kThreads = 128;       // threads per CTA of the reduce / substitute kernels
constexpr int kMaxCos = 16;         // cos-series terms held in the kernel parameters
constexpr int kBaseMax = 16;        // largest reduced system solved by the serial RS stage

// joint line t of a level with n rows, block size m and P blocks
__host__ __device__ __forceinline__ int64_t joint_line(int64_t t, int64_t P, int64_t m, int64_t n) {
    int64_t a = t * m, b = n - 1 - 2 * (P - t);
    return a < b ? a : b;
}

// Device status word values (match cn_status).
constexpr int kStatusNonfinite = 6;

__device__ __forceinline__ void flag_error(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// ------------------------------------------------------------------ row sources
// A source yields the rows k = 0..g (g <= M) of the block starting at row J0:
// lower b_k, diagonal a_k, upper c_k, rhs d_k, with b = 0 on row 0 of the
// level and c = 0 on its last row.

// General tridiagonal system held in four complex128 arrays (cn_solve_tridiag).
struct ArraySource {
    const double2 *b, *a, *c, *d;
    int64_t n;
    template <class R, int M, bool kInterior>
    __device__ __forceinline__ void load(int64_t J0, int g, cx<R>* B, cx<R>* A, cx<R>* C, cx<R>* D) const {
#pragma unroll
        for (int k = kInterior ? 1 : 0; k <= M; ++k) {
            if (kInterior ? (k <= g - 1) : (k <= g)) {
                int64_t i = J0 + k;
                B[k] = (i > 0) ? cload<R>(b + i) : czero<R>();
                A[k] = cload<R>(a + i);
                C[k] = (i < n - 1) ? cload<R>(c + i) : czero<R>();
                D[k] = cload<R>(d + i);
            }
        }
    }
};

// Reduced system of a level >= 1: rows written by the reduce kernel of the
// level below as {b, a, c, d} (four complex128), plus the contribution of the
// previous CTA's last block to the first row of every CTA range (slot).
struct LevelRow {
    double2 b, a, c, d;
};
struct LevelSlot {
    double2 b, a, d;
};
struct LevelSource {
    const LevelRow* rows;
    const LevelSlot* slot;
    int64_t n;            // rows of this level
    int64_t slot_stride;  // rows per CTA range of the producing kernel
    template <class R, int M, bool kInterior>
    __device__ __forceinline__ void load(int64_t J0, int g, cx<R>* B, cx<R>* A, cx<R>* C, cx<R>* D) const {
#pragma unroll
        for (int k = kInterior ? 1 : 0; k <= M; ++k) {
            if (kInterior ? (k <= g - 1) : (k <= g)) {
                int64_t i = J0 + k;
                const LevelRow* r = rows + i;
                B[k] = cload<R>(&r->b);
                A[k] = cload<R>(&r->a);
                C[k] = cload<R>(&r->c);
                D[k] = cload<R>(&r->d);
                if (i > 0 && i < n - 1 && (i % slot_stride) == 0) {
                    const LevelSlot* s = slot + i / slot_stride;
                    B[k] = cload<R>(&s->b);
                    A[k] = A[k] + cload<R>(&s->a);
                    D[k] = D[k] + cload<R>(&s->d);
                }
            }
        }
    }
};

// Crank-Nicolson level 0: T = 1 + i dt/2 H, H = -1/2 d^2/dx^2 + Vs(x) + x E,
// 3-point stencil (Sec. 2).  sgn_t = +1 builds T; the explicit matrix is the
// conjugate transpose with sgn_e = -1 (Eq. ForwardStep).  The adjoint sweep uses
// the opposite signs.  a_j = 1 + i s (dt/2)(1/dx^2 + V_j), b = c = -i s dt/(4 dx^2).
struct CNParams {
    int64_t n;
    double dx, x_min;
    double half_dt;        // dt / 2
    double inv_dx2;        // 1 / dx^2
    double gamma;          // dt / (4 dx^2)
    int pot;               // cn_pot_kind
    int n_cos;
    const double* V0;      // CN_POT_ARRAY
    double soft_s;
    double two_pi_over_L;
    double cos_a[kMaxCos];
};

template <class R>
__device__ __forceinline__ double cn_potential(const CNParams& p, int64_t j, double E) {
    double x = fma((double)j, p.dx, p.x_min);
    double v;
    switch (p.pot) {
    case 1: v = p.V0[j]; break;
    case 2: v = -rsqrt(fma(x, x, p.soft_s)); break;
    case 3: {
        v = 0.0;
        for (int k = 0; k < p.n_cos; ++k) v = fma(p.cos_a[k], cos(p.two_pi_over_L * (double)(k + 1) * x), v);
        break;
    }
    default: v = 0.0;
    }
    return fma(x, E, v);
}

struct CNSource {
    CNParams p;
    const double2* psi;   // state the explicit half-step is applied to
    double sgn_t, sgn_e;  // +1 / -1: sign of i dt/2 H in the implicit / explicit matrix
    const double* E_t;    // device pointer to the field in the implicit matrix (NULL: 0)
    const double* E_e;    // device pointer to the field in the explicit matrix (NULL: 0)
    template <class R, int M, bool kInterior>
    __device__ __forceinline__ void load(int64_t J0, int g, cx<R>* B, cx<R>* A, cx<R>* C, cx<R>* D) const {
        typedef RealOps<R> O;
        const int64_t n = p.n;
        const double Et = E_t ? *E_t : 0.0;
        const double Ee = E_e ? *E_e : 0.0;
        // psi_{J0-1} .. psi_{J0+g+1}, zero outside the grid
        cx<R> prev = (J0 > 0) ? cload<R>(psi + J0 - 1) : czero<R>();
        cx<R> cur = cload<R>(psi + J0);
        const R g_t = O::from_d(-sgn_t * p.gamma);  // b = c = i g_t
        const R g_e = O::from_d(-sgn_e * p.gamma);
        const cx<R> bc = mk<R>(O::from_d(0.0), g_t);
#pragma unroll
        for (int k = 0; k <= M; ++k) {
            if (k <= g) {
                int64_t i = J0 + k;
                cx<R> next = (i + 1 < n) ? cload<R>(psi + i + 1) : czero<R>();
                if (kInterior && (k == 0 || k == g)) {  // joint rows are not needed
                    prev = cur;
                    cur = next;
                    continue;
                }
                double h_t = p.inv_dx2 + cn_potential<R>(p, i, Et);
                double h_e = (Ee == Et) ? h_t : p.inv_dx2 + cn_potential<R>(p, i, Ee);
                R beta_t = O::from_d(sgn_t * p.half_dt * h_t);
                R beta_e = O::from_d(sgn_e * p.half_dt * h_e);
                // explicit row: d = (1 + i beta_e) psi_i + i g_e (psi_{i-1} + psi_{i+1})
                cx<R> s = prev + next;
                D[k] = cur + cmul_i(cscale(cur, beta_e) + cscale(s, g_e));
                A[k] = mk<R>(O::from_d(1.0), beta_t);
                B[k] = (i > 0) ? bc : czero<R>();
                C[k] = (i < n - 1) ? bc : czero<R>();
                prev = cur;
                cur = next;
            }
        }
    }
};

// ------------------------------------------------------------------ reduction
// One thread per block: Table 1 RD + JD, then RU + JU (Sec. 5.2.1 order).
// Writes the reduced system rows {b, a, c, d} of the next level.
template <class R>
struct JDPart {
    cx<R> b, a, d;
};

template <class R, int M, class Src>
__global__ void __launch_bounds__(kThreads)
k_reduce(Src src, int64_t n, int64_t P, int m, LevelRow* out, LevelSlot* out_slot, int* status) {
    __shared__ JDPart<R> xch[kThreads];
    const int tid = threadIdx.x;
    const int64_t t = (int64_t)blockIdx.x * kThreads + tid;
    const bool active = t < P;
    bool ok = true;
    cx<R> JUa = czero<R>(), JUc = czero<R>(), JUd = czero<R>();
    cx<R> A0 = czero<R>(), D0 = czero<R>();
    JDPart<R> jd;
    jd.b = czero<R>(); jd.a = czero<R>(); jd.d = czero<R>();
    cx<R> Ag = czero<R>(), Dg = czero<R>();
    int64_t J0 = 0;
    if (active) {
        J0 = joint_line(t, P, m, n);
        const int g = (int)(joint_line(t + 1, P, m, n) - J0);
        cx<R> B[M + 1], A[M + 1], C[M + 1], D[M + 1], W[M + 1];
        src.template load<R, M, false>(J0, g, B, A, C, D);
        A0 = A[0];
        D0 = D[0];
        // RD: i = J0+2 .. J1-1 ; W[k] = 1 / a_k (after RD) for interior rows
        W[1] = crcp(A[1], ok);
#pragma unroll
        for (int k = 2; k < M; ++k) {
            if (k <= g - 1) {
                cx<R> r = -(B[k] * W[k - 1]);
                B[k] = r * B[k - 1];
                A[k] = A[k] + r * C[k - 1];
                D[k] = D[k] + r * D[k - 1];
                W[k] = crcp(A[k], ok);
            }
        }
        // JD on row J1 (k = g): r = -b_g / a_{g-1}
#pragma unroll
        for (int k = 2; k <= M; ++k) {
            if (k == g) {
                cx<R> r = -(B[k] * W[k - 1]);
                jd.b = r * B[k - 1];
                jd.a = r * C[k - 1];
                jd.d = r * D[k - 1];
                Ag = A[k];
                Dg = D[k];
            }
        }
        // RU: i = J1-2 down to J0+1 ; carried row below (nb, nc, nd)
        cx<R> nb = czero<R>(), nc = czero<R>(), nd = czero<R>();
#pragma unroll
        for (int k = M - 1; k >= 1; --k) {
            if (k == g - 1) {
                nb = B[k]; nc = C[k]; nd = D[k];
            } else if (k < g - 1) {
                cx<R> r = -(C[k] * W[k + 1]);
                nb = B[k] + r * nb;
                nc = r * nc;
                nd = D[k] + r * nd;
            }
        }
        // JU on row J0 (k = 0): r = -c_0 / a_1 with row 1 after RU
        cx<R> r = -(C[0] * W[1]);
        JUc = r * nc;
        JUa = r * nb;
        JUd = r * nd;
    }
    xch[tid] = jd;
    __syncthreads();
    if (!active) return;
    // row t of the next level: b = JD of block t-1, a = a_J + (JD + JU), c = JU, d likewise
    LevelRow row;
    if (tid > 0) {
        JDPart<R> pj = xch[tid - 1];
        cstore(&row.b, pj.b);
        cstore(&row.a, A0 + (pj.a + JUa));
        cstore(&row.d, D0 + (pj.d + JUd));
    } else {
        // t == 0: no block above; otherwise the previous CTA delivers its part via the slot
        cstore(&row.b, czero<R>());
        cstore(&row.a, A0 + JUa);
        cstore(&row.d, D0 + JUd);
    }
    cstore(&row.c, JUc);
    out[t] = row;
    if (t == P - 1) {
        // last joint line: only the JD contribution of this block
        LevelRow last;
        cstore(&last.b, jd.b);
        cstore(&last.a, Ag + jd.a);
        cstore(&last.c, czero<R>());
        cstore(&last.d, Dg + jd.d);
        out[P] = last;
    } else if (tid == kThreads - 1) {
        LevelSlot s;
        cstore(&s.b, jd.b);
        cstore(&s.a, jd.a);
        cstore(&s.d, jd.d);
        out_slot[blockIdx.x + 1] = s;
    }
    if (!ok) flag_error(status, kStatusNonfinite);
}

// ------------------------------------------------------------------ substitution
// One thread per block: the interior rows 1..g-1 with the support values xL
// (row 0) and xR (row g) known form a tridiagonal system, solved by Thomas.
template <class R, int M, class Src>
__global__ void __launch_bounds__(kThreads)
k_substitute(Src src, int64_t n, int64_t P, int m, const double2* x_next, double2* x, int* status) {
    const int64_t t = (int64_t)blockIdx.x * kThreads + threadIdx.x;
    if (t >= P) return;
    bool ok = true;
    const int64_t J0 = joint_line(t, P, m, n);
    const int g = (int)(joint_line(t + 1, P, m, n) - J0);
    cx<R> B[M + 1], A[M + 1], C[M + 1], D[M + 1];
    src.template load<R, M, true>(J0, g, B, A, C, D);
    const cx<R> xL = cload<R>(x_next + t);
    const cx<R> xR = cload<R>(x_next + t + 1);
    cx<R> Z[M + 1], CP[M + 1];
    cx<R> zp = czero<R>(), cpp = czero<R>();
#pragma unroll
    for (int k = 1; k < M + 1; ++k) {
        if (k <= g - 1) {
            cx<R> rhs = D[k];
            if (k == 1) rhs = rhs - B[1] * xL;
            if (k == g - 1) rhs = rhs - C[k] * xR;
            cx<R> mk_ = (k == 1) ? A[1] : A[k] - B[k] * cpp;
            cx<R> w = crcp(mk_, ok);
            cx<R> z = (k == 1) ? rhs * w : (rhs - B[k] * zp) * w;
            cx<R> cp = C[k] * w;
            Z[k] = z;
            CP[k] = cp;
            zp = z;
            cpp = cp;
        }
    }
    cx<R> y = czero<R>();
#pragma unroll
    for (int k = M; k >= 1; --k) {
        if (k == g - 1) {
            y = Z[k];
            cstore(x + J0 + k, y);
        } else if (k < g - 1) {
            y = Z[k] - CP[k] * y;
            cstore(x + J0 + k, y);
        }
    }
    cstore(x + J0, xL);
    if (t == P - 1) cstore(x + J0 + g, xR);
    if (!ok) flag_error(status, kStatusNonfinite);
}

// ------------------------------------------------------------------ RS stage
// Serial Thomas elimination of the last reduced system (Table 1, RS), one thread.
template <class R>
__global__ void k_base(LevelSource src, int64_t n, double2* x, int* status) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    bool ok = true;
    cx<R> a_prev = czero<R>(), c_prev = czero<R>(), d_prev = czero<R>();
    cx<R> A[kBaseMax], C[kBaseMax], D[kBaseMax];
    for (int64_t w = 0; w < n; ++w) {
        cx<R> b, a, c, d;
        src.template load<R, 0, false>(w, 0, &b, &a, &c, &d);
        if (w > 0) {
            // r = -b_w / a_{w-1};  a_w += r c_{w-1};  d_w += r d_{w-1}
            cx<R> r = -(b * crcp(a_prev, ok));
            a = a + r * c_prev;
            d = d + r * d_prev;
        }
        A[w] = a; C[w] = c; D[w] = d;
        a_prev = a; c_prev = c; d_prev = d;
    }
    cx<R> y = D[n - 1] * crcp(A[n - 1], ok);
    cstore(x + n - 1, y);
    for (int64_t w = n - 2; w >= 0; --w) {
        y = (D[w] - C[w] * y) * crcp(A[w], ok);
        cstore(x + w, y);
    }
    if (!ok) flag_error(status, kStatusNonfinite);
}

}  // namespace cnb
