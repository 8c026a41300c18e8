/*
 * cn_oracle.h -- serial FP64 CPU oracle for the Crank-Nicolson / N-shaped
 * partition method (Lutsyshyn, Navarrete, Bauer, "The N-shaped partition
 * method: A novel parallel implementation of the Crank Nicolson algorithm").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may include, link or
 * call this library: only tests/, __graft_entry__.smoke() and the CPU-baseline
 * leg of bench.py use it.  It shares no code, header, table or helper with the
 * CUDA path.
 *
 * Conventions (all functions):
 *   - complex numbers are C99 `double _Complex`, stored as interleaved
 *     (re, im) pairs of doubles, i.e. the same bytes as numpy complex128;
 *   - indices are 0-based, rows j = 0..n-1; the paper's 1-based rows
 *     1..n_tot map to 0..n-1 (Sec. 4);
 *   - a tridiagonal matrix is given by its three diagonals b (lower,
 *     b[j] = T[j][j-1]), a (centre) and c (upper, c[j] = T[j][j+1]);
 *     b[0] and c[n-1] are ignored (taken as 0), Eq. (algorithm);
 *   - return 0 on success, negative on bad arguments, positive when a pivot
 *     is exactly zero.
 *
 * Parity status: every function here is pinned by tests under tests/ marked
 * "not gpu" (dense LU, DST-I eigen-decomposition, closed-form Gaussian,
 * invariants, finite differences).  None is "parity unpinned".
 */
#ifndef CN_ORACLE_H
#define CN_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Potential kinds of the 1D TDSE Hamiltonian H = -1/2 d^2/dx^2 + V(x, t). */
enum { OR_POT_NONE = 0, OR_POT_ARRAY = 1, OR_POT_SOFTCOULOMB = 2, OR_POT_COSSERIES = 3 };

/* A 1D TDSE problem on the uniform grid x_j = x_min + j dx, j = 0..n-1, with
 * psi = 0 outside the grid (Sec. 4: psi_0 = psi_{n_tot+1} = 0).
 * V(x, t) = Vs(x) + x E(t), where the static part Vs is
 *   NONE:        0
 *   ARRAY:       V0[j]
 *   SOFTCOULOMB: -1 / sqrt(x^2 + soft_s)
 *   COSSERIES:   sum_{k=1..n_cos} cos_a[k-1] cos(2 pi k x / L)           */
typedef struct {
    int64_t n;
    double dx, dt, x_min;
    int32_t pot;
    const double* V0;
    double soft_s;
    const double* cos_a;
    int32_t n_cos;
    double L;
} or_problem;

/* Thomas algorithm (Sec. 2): solve T x = d for tridiagonal T (b, a, c). */
int or_thomas(int64_t n, const double* b, const double* a, const double* c,
              const double* d, double* x);

/* y = T x for tridiagonal T (b, a, c). */
int or_tridiag_apply(int64_t n, const double* b, const double* a, const double* c,
                     const double* x, double* y);

/* The diagonals of T = 1 + i (dt/2) H(t_mid) (Sec. 2) for field value E at
 * t_mid; with dt_sign = -1 the diagonals of the conjugate-transpose
 * T^dagger = 1 - i (dt/2) H are returned instead.  b, a, c have n entries. */
int or_cn_matrix(const or_problem* p, double E, int dt_sign,
                 double* b, double* a, double* c);

/* nsteps Crank-Nicolson steps (Eq. Cn_both_steps): for k = 0..nsteps-1,
 * d = T_k^dagger psi (Eq. ForwardStep), then T_k psi' = d solved by Thomas
 * (Eq. BackwardStep), with T_k built at t_k + dt/2 from E_mid[k]
 * (E_mid may be NULL: E = 0).  psi0 and psi_out may alias. */
int or_cn_run(const or_problem* p, const double* psi0, const double* E_mid,
              int64_t nsteps, double* psi_out);

/* --- Literal restatement of Table 1 (Sec. 4) ------------------------------ */

/* RD+JD+RU+JU on the blocks delimited by the joint lines J[0..P]
 * (J[0] = 0, J[P] = n-1, J[w+1] - J[w] >= 2).  The four working vectors
 * (bw, aw, cw, dw), which on entry hold b, a, c, d, are modified in place as
 * Table 1 prescribes; the two "atomic" additions on every joint line are kept
 * in two separate slots and folded afterwards in a fixed order
 * (a_J += from_left + from_right), as Sec. 4.1.3 allows.
 * order = 0: stages in the order RD, RU, JU, JD (Table 1);
 * order = 1: (RD + JD) + (RU + JU) (Sec. 5.2.1).
 * On return the joint lines J[w] of (bw, aw, cw, dw) hold the reduced
 * tridiagonal system (Fig. 1e): lower = bw[J[w]] (column J[w-1]),
 * centre = aw[J[w]], upper = cw[J[w]] (column J[w+1]), rhs = dw[J[w]]. */
int or_nshape_reduce(int64_t n, double* bw, double* aw, double* cw, double* dw,
                     int64_t P, const int64_t* J, int order);

/* SS stage: given the support values psi_J[0..P] on the joint lines and the
 * vectors produced by or_nshape_reduce, fill x[0..n-1]. */
int or_nshape_substitute(int64_t n, const double* bw, const double* aw, const double* cw,
                         const double* dw, int64_t P, const int64_t* J,
                         const double* psi_J, double* x);

/* RS stage: Thomas-like elimination restricted to the joint lines (Table 1,
 * RS).  Operates in place on the joint-line entries; writes psi_J[0..P]. */
int or_nshape_rs(double* bw, double* aw, double* cw, double* dw,
                 int64_t P, const int64_t* J, double* psi_J);

/* Full N-shaped solve of T x = d, nested as in Eq. (iteration):
 * level 0 uses the joint lines J[0..P]; the reduced system of every level l
 * is again solved by the N-shaped method with nested_P[l] blocks placed by
 * the default rule J_w = floor(w (n_l - 1) / P_l), for l < n_nested; the
 * last reduced system is solved by the RS stage. */
int or_nshape_solve(int64_t n, const double* b, const double* a, const double* c,
                    const double* d, int64_t P, const int64_t* J,
                    int64_t n_nested, const int64_t* nested_P, int order, double* x);

/* Default joint-line placement J_w = floor(w (n-1) / P), w = 0..P. */
int or_default_joints(int64_t n, int64_t P, int64_t* J);

/* --- Adjoint (gradient of a final-state population w.r.t. E) -------------- */

/* Loss L = sum_j wgt[j] |psi_{nsteps, j}|^2 after or_cn_run.  Computes L and
 * dLdE[k] = dL / dE_mid[k] for k = 0..nsteps-1 by the discrete adjoint of
 * the Crank-Nicolson recursion, storing every forward state.  lam0 (may be
 * NULL) receives the adjoint state lambda_0 with dL = 2 Re(lambda_0^H dpsi_0)
 * for a perturbation of the initial state.  E_mid may be NULL (E = 0). */
int or_adjoint_run(const or_problem* p, const double* psi0, const double* E_mid,
                   int64_t nsteps, const double* wgt, double* loss, double* dLdE,
                   double* lam0);

#ifdef __cplusplus
}
#endif
#endif
