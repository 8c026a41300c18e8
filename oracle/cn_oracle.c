/*
 * cn_oracle.c -- serial FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * cn_oracle.h).  Plain, slow, obviously-correct restatements of the paper's
 * definitions.  Built without fast-math: C99 complex arithmetic, IEEE double.
 *
 * Paper: Lutsyshyn, Navarrete, Bauer, "The N-shaped partition method".
 *   Sec. 2      : Crank-Nicolson propagator, T = 1 + i dt/2 H(t + dt/2),
 *                 Eq. (Cn_both_steps), (ForwardStep), (BackwardStep);
 *                 Thomas algorithm.
 *   Sec. 4      : tridiagonal notation, Eq. (algorithm); joint lines;
 *                 Table 1 stages RD, RU, JU, JD, RS, SS; Eq. (iteration).
 *   Sec. 5.2.1  : (RD + JD) + (RU + JU) reordering.
 *   Appendix I  : row-operation form of the same stages.
 */
#include "cn_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

typedef double _Complex cplx;

#define CV(p) ((const cplx*)(const void*)(p))
#define MV(p) ((cplx*)(void*)(p))

/* ------------------------------------------------------------------------ */
/* Thomas algorithm (Sec. 2).  Forward elimination with the modified upper
 * diagonal cp and right-hand side dp, then back-substitution:
 *   cp_0 = c_0 / a_0,  dp_0 = d_0 / a_0,
 *   m_j  = a_j - b_j cp_{j-1},  cp_j = c_j / m_j,
 *   dp_j = (d_j - b_j dp_{j-1}) / m_j,
 *   x_{n-1} = dp_{n-1},  x_j = dp_j - cp_j x_{j+1}.                          */
int or_thomas(int64_t n, const double* b_, const double* a_, const double* c_,
              const double* d_, double* x_)
{
    if (n < 1 || !a_ || !d_ || !x_ || (n > 1 && (!b_ || !c_))) return -1;
    const cplx *b = CV(b_), *a = CV(a_), *c = CV(c_), *d = CV(d_);
    cplx* x = MV(x_);
    cplx* cp = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    cplx* dp = (cplx*)malloc(sizeof(cplx) * (size_t)n);
    if (!cp || !dp) { free(cp); free(dp); return -2; }
    int rc = 0;
    if (a[0] == 0) { rc = 1; goto done; }
    cp[0] = (n > 1) ? c[0] / a[0] : 0;
    dp[0] = d[0] / a[0];
    for (int64_t j = 1; j < n; ++j) {
        cplx m = a[j] - b[j] * cp[j - 1];
        if (m == 0) { rc = 1; goto done; }
        cp[j] = (j < n - 1) ? c[j] / m : 0;
        dp[j] = (d[j] - b[j] * dp[j - 1]) / m;
    }
    x[n - 1] = dp[n - 1];
    for (int64_t j = n - 2; j >= 0; --j) x[j] = dp[j] - cp[j] * x[j + 1];
done:
    free(cp);
    free(dp);
    return rc;
}

/* y = T x, Eq. (algorithm) row by row, with psi_{-1} = psi_n = 0. */
int or_tridiag_apply(int64_t n, const double* b_, const double* a_, const double* c_,
                     const double* x_, double* y_)
{
    if (n < 1 || !a_ || !x_ || !y_ || (n > 1 && (!b_ || !c_))) return -1;
    const cplx *b = CV(b_), *a = CV(a_), *c = CV(c_), *x = CV(x_);
    cplx* y = MV(y_);
    for (int64_t j = 0; j < n; ++j) {
        cplx s = a[j] * x[j];
        if (j > 0) s += b[j] * x[j - 1];
        if (j < n - 1) s += c[j] * x[j + 1];
        y[j] = s;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Grid and Hamiltonian (Sec. 2, Sec. 4).  x_j = x_min + j dx.              */
static double grid_x(const or_problem* p, int64_t j) { return p->x_min + (double)j * p->dx; }

static double static_potential(const or_problem* p, int64_t j)
{
    const double x = grid_x(p, j);
    switch (p->pot) {
    case OR_POT_NONE: return 0.0;
    case OR_POT_ARRAY: return p->V0[j];
    case OR_POT_SOFTCOULOMB: return -1.0 / sqrt(x * x + p->soft_s);
    case OR_POT_COSSERIES: {
        const double pi = 3.14159265358979323846;
        double v = 0.0;
        for (int k = 1; k <= p->n_cos; ++k) v += p->cos_a[k - 1] * cos(2.0 * pi * k * x / p->L);
        return v;
    }
    default: return NAN;
    }
}

static int problem_ok(const or_problem* p)
{
    if (!p || p->n < 1 || !(p->dx > 0) || !(p->dt == p->dt)) return 0;
    if (p->pot < OR_POT_NONE || p->pot > OR_POT_COSSERIES) return 0;
    if (p->pot == OR_POT_ARRAY && !p->V0) return 0;
    if (p->pot == OR_POT_COSSERIES && (p->n_cos < 0 || (p->n_cos > 0 && !p->cos_a) || !(p->L > 0))) return 0;
    return 1;
}

/* Finite-difference H = -1/2 d^2/dx^2 + V(x, t) by the 3-point stencil:
 *   H_jj = 1/dx^2 + V_j,   H_{j,j+-1} = -1/(2 dx^2).
 * T = 1 + s i (dt/2) H with s = +1 (implicit matrix T) or s = -1 (the
 * explicit matrix T^dagger of Eq. ForwardStep; H is real symmetric, so the
 * conjugate transpose of T is 1 - i (dt/2) H).                               */
int or_cn_matrix(const or_problem* p, double E, int dt_sign, double* b_, double* a_, double* c_)
{
    if (!problem_ok(p) || !b_ || !a_ || !c_ || (dt_sign != 1 && dt_sign != -1)) return -1;
    cplx *b = MV(b_), *a = MV(a_), *c = MV(c_);
    const double inv_dx2 = 1.0 / (p->dx * p->dx);
    const cplx f = (double)dt_sign * I * (p->dt / 2.0);
    const double h_off = -0.5 * inv_dx2;
    for (int64_t j = 0; j < p->n; ++j) {
        const double V = static_potential(p, j) + grid_x(p, j) * E;
        const double h_diag = inv_dx2 + V;
        a[j] = 1.0 + f * h_diag;
        b[j] = (j > 0) ? f * h_off : 0;
        c[j] = (j < p->n - 1) ? f * h_off : 0;
    }
    return 0;
}

/* One Crank-Nicolson step (Eq. Cn_both_steps): d = T^dagger psi, T psi' = d. */
static int cn_one_step(const or_problem* p, double E, const cplx* psi, cplx* out,
                       cplx* b, cplx* a, cplx* c, cplx* bs, cplx* as, cplx* cs, cplx* d)
{
    int rc = or_cn_matrix(p, E, -1, (double*)bs, (double*)as, (double*)cs);
    if (rc) return rc;
    rc = or_cn_matrix(p, E, +1, (double*)b, (double*)a, (double*)c);
    if (rc) return rc;
    rc = or_tridiag_apply(p->n, (double*)bs, (double*)as, (double*)cs, (const double*)psi, (double*)d);
    if (rc) return rc;
    return or_thomas(p->n, (double*)b, (double*)a, (double*)c, (double*)d, (double*)out);
}

int or_cn_run(const or_problem* p, const double* psi0_, const double* E_mid,
              int64_t nsteps, double* psi_out_)
{
    if (!problem_ok(p) || !psi0_ || !psi_out_ || nsteps < 0) return -1;
    const int64_t n = p->n;
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n * 8);
    if (!buf) return -2;
    cplx *b = buf, *a = buf + n, *c = buf + 2 * n, *bs = buf + 3 * n, *as = buf + 4 * n,
         *cs = buf + 5 * n, *d = buf + 6 * n, *cur = buf + 7 * n;
    memcpy(cur, psi0_, sizeof(cplx) * (size_t)n);
    int rc = 0;
    for (int64_t k = 0; k < nsteps && rc == 0; ++k) {
        const double E = E_mid ? E_mid[k] : 0.0;
        rc = cn_one_step(p, E, cur, cur, b, a, c, bs, as, cs, d);
    }
    if (rc == 0) memcpy(psi_out_, cur, sizeof(cplx) * (size_t)n);
    free(buf);
    return rc;
}

/* ------------------------------------------------------------------------ */
/* Table 1, stage by stage.  Blocks w = 0..P-1 lie between joint lines J[w]
 * and J[w+1]; their interior rows are J[w]+1 .. J[w+1]-1.                   */

static int joints_ok(int64_t n, int64_t P, const int64_t* J)
{
    if (P < 1 || !J || J[0] != 0 || J[P] != n - 1) return 0;
    for (int64_t w = 0; w < P; ++w)
        if (J[w + 1] - J[w] < 2) return 0;  /* every block keeps >= 1 interior row */
    return 1;
}

/* RD stage of block w: i = J_w+2 .. J_{w+1}-1,
 *   r_i = -b_i / a_{i-1};  b_i <- r_i b_{i-1};  a_i <- a_i + r_i c_{i-1};
 *   d_i <- d_i + r_i d_{i-1};  (c_i unchanged).                             */
static void stage_rd(cplx* b, cplx* a, cplx* c, cplx* d, int64_t Jw, int64_t Jw1)
{
    for (int64_t i = Jw + 2; i <= Jw1 - 1; ++i) {
        const cplx r = -b[i] / a[i - 1];
        b[i] = r * b[i - 1];
        a[i] = a[i] + r * c[i - 1];
        d[i] = d[i] + r * d[i - 1];
    }
}

/* RU stage of block w: i = J_{w+1}-2 down to J_w+1,
 *   r_i = -c_i / a_{i+1};  b_i <- b_i + r_i b_{i+1};  c_i <- r_i c_{i+1};
 *   d_i <- d_i + r_i d_{i+1};  (a_i unchanged).                             */
static void stage_ru(cplx* b, cplx* a, cplx* c, cplx* d, int64_t Jw, int64_t Jw1)
{
    for (int64_t i = Jw1 - 2; i >= Jw + 1; --i) {
        const cplx r = -c[i] / a[i + 1];
        b[i] = b[i] + r * b[i + 1];
        c[i] = r * c[i + 1];
        d[i] = d[i] + r * d[i + 1];
    }
}

/* JU stage of block w on row i = J_w:
 *   r_i = -c_i / a_{i+1};  c_i <- r_i c_{i+1};
 *   a_i <-(atomic) a_i + r_i b_{i+1};  d_i <-(atomic) d_i + r_i d_{i+1}.
 * The two atomic additions go to the "from the block below" slot of the
 * joint line (Sec. 4.1.3: two extra memory elements per joint line).        */
static void stage_ju(cplx* b, cplx* a, cplx* c, cplx* d, int64_t Jw, cplx* slot_a, cplx* slot_d)
{
    const int64_t i = Jw;
    const cplx r = -c[i] / a[i + 1];
    c[i] = r * c[i + 1];
    *slot_a = r * b[i + 1];
    *slot_d = r * d[i + 1];
}

/* JD stage of block w on row i = J_{w+1}:
 *   r_i = -b_i / a_{i-1};  b_i <- r_i b_{i-1};
 *   a_i <-(atomic) a_i + r_i c_{i-1};  d_i <-(atomic) d_i + r_i d_{i-1}.    */
static void stage_jd(cplx* b, cplx* a, cplx* c, cplx* d, int64_t Jw1, cplx* slot_a, cplx* slot_d)
{
    const int64_t i = Jw1;
    const cplx r = -b[i] / a[i - 1];
    b[i] = r * b[i - 1];
    *slot_a = r * c[i - 1];
    *slot_d = r * d[i - 1];
}

int or_nshape_reduce(int64_t n, double* b_, double* a_, double* c_, double* d_,
                     int64_t P, const int64_t* J, int order)
{
    if (n < 3 || !b_ || !a_ || !c_ || !d_ || !joints_ok(n, P, J) || (order != 0 && order != 1)) return -1;
    cplx *b = MV(b_), *a = MV(a_), *c = MV(c_), *d = MV(d_);
    /* slot arrays: from_above[w] is written by block w-1 (JD on J_w),
     * from_below[w] by block w (JU on J_w). */
    cplx* slots = (cplx*)calloc((size_t)(P + 1) * 4, sizeof(cplx));
    if (!slots) return -2;
    cplx *above_a = slots, *above_d = slots + (P + 1), *below_a = slots + 2 * (P + 1),
         *below_d = slots + 3 * (P + 1);
    if (order == 0) {
        /* Table 1 order: RD, RU, JU, JD for every block. */
        for (int64_t w = 0; w < P; ++w) stage_rd(b, a, c, d, J[w], J[w + 1]);
        for (int64_t w = 0; w < P; ++w) stage_ru(b, a, c, d, J[w], J[w + 1]);
        for (int64_t w = 0; w < P; ++w) stage_ju(b, a, c, d, J[w], &below_a[w], &below_d[w]);
        for (int64_t w = 0; w < P; ++w) stage_jd(b, a, c, d, J[w + 1], &above_a[w + 1], &above_d[w + 1]);
    } else {
        /* Sec. 5.2.1 order: (RD + JD) + (RU + JU). */
        for (int64_t w = 0; w < P; ++w) {
            stage_rd(b, a, c, d, J[w], J[w + 1]);
            stage_jd(b, a, c, d, J[w + 1], &above_a[w + 1], &above_d[w + 1]);
        }
        for (int64_t w = 0; w < P; ++w) {
            stage_ru(b, a, c, d, J[w], J[w + 1]);
            stage_ju(b, a, c, d, J[w], &below_a[w], &below_d[w]);
        }
    }
    /* Fold the two slots of every joint line in a fixed order. */
    for (int64_t w = 0; w <= P; ++w) {
        const int64_t i = J[w];
        a[i] = a[i] + (above_a[w] + below_a[w]);
        d[i] = d[i] + (above_d[w] + below_d[w]);
    }
    /* The first joint line has no column J_{-1}; the last has no J_{P+1}. */
    b[J[0]] = 0;
    c[J[P]] = 0;
    free(slots);
    return 0;
}

/* RS stage (Table 1), index w over joint lines (the grid indices i-1, i+1 of
 * the table denote the neighbouring joint lines J_{w-1}, J_{w+1}):
 *   w = 1..P:     r = -b_{J_w} / a_{J_{w-1}};  a_{J_w} += r c_{J_{w-1}};
 *                 d_{J_w} += r d_{J_{w-1}};
 *   psi_{J_P} = d_{J_P} / a_{J_P};
 *   w = P-1..0:   psi_{J_w} = (d_{J_w} - c_{J_w} psi_{J_{w+1}}) / a_{J_w}.   */
int or_nshape_rs(double* b_, double* a_, double* c_, double* d_, int64_t P,
                 const int64_t* J, double* psi_J_)
{
    if (P < 1 || !b_ || !a_ || !c_ || !d_ || !J || !psi_J_) return -1;
    cplx *b = MV(b_), *a = MV(a_), *c = MV(c_), *d = MV(d_), *psi = MV(psi_J_);
    for (int64_t w = 1; w <= P; ++w) {
        const int64_t i = J[w], im = J[w - 1];
        if (a[im] == 0) return 1;
        const cplx r = -b[i] / a[im];
        a[i] = a[i] + r * c[im];
        d[i] = d[i] + r * d[im];
    }
    if (a[J[P]] == 0) return 1;
    psi[P] = d[J[P]] / a[J[P]];
    for (int64_t w = P - 1; w >= 0; --w) {
        const int64_t i = J[w];
        if (a[i] == 0) return 1;
        psi[w] = (d[i] - c[i] * psi[w + 1]) / a[i];
    }
    return 0;
}

/* SS stage (Table 1): i = J_w+1 .. J_{w+1}-1,
 *   r_i = 1 / a_i;  psi_i = (d_i - b_i psi_{J_w} - c_i psi_{J_{w+1}}) r_i.   */
int or_nshape_substitute(int64_t n, const double* b_, const double* a_, const double* c_,
                         const double* d_, int64_t P, const int64_t* J,
                         const double* psi_J_, double* x_)
{
    if (n < 3 || !b_ || !a_ || !c_ || !d_ || !psi_J_ || !x_ || !joints_ok(n, P, J)) return -1;
    const cplx *b = CV(b_), *a = CV(a_), *c = CV(c_), *d = CV(d_), *psi = CV(psi_J_);
    cplx* x = MV(x_);
    for (int64_t w = 0; w <= P; ++w) x[J[w]] = psi[w];
    for (int64_t w = 0; w < P; ++w) {
        for (int64_t i = J[w] + 1; i <= J[w + 1] - 1; ++i) {
            if (a[i] == 0) return 1;
            const cplx r = 1.0 / a[i];
            x[i] = (d[i] - b[i] * psi[w] - c[i] * psi[w + 1]) * r;
        }
    }
    return 0;
}

int or_default_joints(int64_t n, int64_t P, int64_t* J)
{
    if (n < 3 || P < 1 || !J || 2 * P > n - 1) return -1;
    for (int64_t w = 0; w <= P; ++w) {
        /* floor(w (n-1) / P) without 64-bit overflow for the sizes used here */
        J[w] = (int64_t)(((__int128)w * (n - 1)) / P);
    }
    return joints_ok(n, P, J) ? 0 : -1;
}

/* Eq. (iteration): N[M_0] = (reduction of M_0) + N[M_1] + SS[M_0], where M_1
 * is the reduced system on the joint lines of M_0.                          */
static int nshape_rec(int64_t n, const cplx* b, const cplx* a, const cplx* c, const cplx* d,
                      int64_t P, const int64_t* J, int64_t n_nested, const int64_t* nested_P,
                      int order, cplx* x)
{
    int rc = 0;
    cplx* w4 = (cplx*)malloc(sizeof(cplx) * (size_t)n * 4);
    cplx* red = (cplx*)malloc(sizeof(cplx) * (size_t)(P + 1) * 5);
    int64_t* Jn = NULL;
    if (!w4 || !red) { rc = -2; goto out; }
    cplx *bw = w4, *aw = w4 + n, *cw = w4 + 2 * n, *dw = w4 + 3 * n;
    memcpy(bw, b, sizeof(cplx) * (size_t)n);
    memcpy(aw, a, sizeof(cplx) * (size_t)n);
    memcpy(cw, c, sizeof(cplx) * (size_t)n);
    memcpy(dw, d, sizeof(cplx) * (size_t)n);
    rc = or_nshape_reduce(n, (double*)bw, (double*)aw, (double*)cw, (double*)dw, P, J, order);
    if (rc) goto out;
    /* M_1: the reduced system on the joint lines, Fig. 1(e). */
    const int64_t m = P + 1;
    cplx *rb = red, *ra = red + m, *rc_ = red + 2 * m, *rd = red + 3 * m, *psiJ = red + 4 * m;
    for (int64_t w = 0; w < m; ++w) {
        rb[w] = bw[J[w]];
        ra[w] = aw[J[w]];
        rc_[w] = cw[J[w]];
        rd[w] = dw[J[w]];
    }
    if (n_nested > 0) {
        if (m < 3 || nested_P[0] < 1 || 2 * nested_P[0] > m - 1) { rc = -1; goto out; }
        Jn = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nested_P[0] + 1));
        if (!Jn) { rc = -2; goto out; }
        rc = or_default_joints(m, nested_P[0], Jn);
        if (rc) goto out;
        rc = nshape_rec(m, rb, ra, rc_, rd, nested_P[0], Jn, n_nested - 1, nested_P + 1, order, psiJ);
    } else {
        /* RS stage on M_1 (the joint lines of M_1 are all of its rows). */
        int64_t* Jid = (int64_t*)malloc(sizeof(int64_t) * (size_t)m);
        if (!Jid) { rc = -2; goto out; }
        for (int64_t w = 0; w < m; ++w) Jid[w] = w;
        rc = or_nshape_rs((double*)rb, (double*)ra, (double*)rc_, (double*)rd, P, Jid, (double*)psiJ);
        free(Jid);
    }
    if (rc) goto out;
    rc = or_nshape_substitute(n, (double*)bw, (double*)aw, (double*)cw, (double*)dw, P, J,
                              (double*)psiJ, (double*)x);
out:
    free(w4);
    free(red);
    free(Jn);
    return rc;
}

int or_nshape_solve(int64_t n, const double* b, const double* a, const double* c,
                    const double* d, int64_t P, const int64_t* J,
                    int64_t n_nested, const int64_t* nested_P, int order, double* x)
{
    if (n < 3 || !b || !a || !c || !d || !x || !joints_ok(n, P, J) || n_nested < 0 ||
        (n_nested > 0 && !nested_P) || (order != 0 && order != 1))
        return -1;
    return nshape_rec(n, CV(b), CV(a), CV(c), CV(d), P, J, n_nested, nested_P, order, MV(x));
}

/* ------------------------------------------------------------------------ */
/* Discrete adjoint of the CN recursion  T_k psi_{k+1} = S_k psi_k,
 * S_k = T_k^dagger (Eq. Cn_both_steps), for L = sum_j wgt_j |psi_{K,j}|^2.
 * With the convention dL = 2 Re(lambda_k^H dpsi_k):
 *   lambda_K = wgt .* psi_K,
 *   mu_k     = T_k^{-H} lambda_{k+1}     (solve with the conjugate transpose),
 *   lambda_k = S_k^H mu_k,
 *   dL/dE_k  = 2 Re( mu_k^H ( dS_k/dE psi_k - dT_k/dE psi_{k+1} ) ),
 * where dT_k/dE = i (dt/2) X and dS_k/dE = -i (dt/2) X, X = diag(x_j), since
 * V = Vs(x) + x E enters H only through its diagonal.                       */

/* conjugate transpose of a tridiagonal (b, a, c): lower'[j] = conj(c[j-1]),
 * centre'[j] = conj(a[j]), upper'[j] = conj(b[j+1]). */
static void tridiag_conj_transpose(int64_t n, const cplx* b, const cplx* a, const cplx* c,
                                   cplx* bh, cplx* ah, cplx* ch)
{
    for (int64_t j = 0; j < n; ++j) {
        ah[j] = conj(a[j]);
        bh[j] = (j > 0) ? conj(c[j - 1]) : 0;
        ch[j] = (j < n - 1) ? conj(b[j + 1]) : 0;
    }
}

int or_adjoint_run(const or_problem* p, const double* psi0_, const double* E_mid,
                   int64_t nsteps, const double* wgt, double* loss, double* dLdE,
                   double* lam0_)
{
    if (!problem_ok(p) || !psi0_ || !wgt || !loss || nsteps < 0 || (nsteps > 0 && !dLdE)) return -1;
    const int64_t n = p->n;
    cplx* states = (cplx*)malloc(sizeof(cplx) * (size_t)n * (size_t)(nsteps + 1));
    cplx* buf = (cplx*)malloc(sizeof(cplx) * (size_t)n * 12);
    if (!states || !buf) { free(states); free(buf); return -2; }
    cplx *b = buf, *a = buf + n, *c = buf + 2 * n, *bs = buf + 3 * n, *as = buf + 4 * n,
         *cs = buf + 5 * n, *d = buf + 6 * n, *bh = buf + 7 * n, *ah = buf + 8 * n,
         *ch = buf + 9 * n, *lam = buf + 10 * n, *mu = buf + 11 * n;
    int rc = 0;
    memcpy(states, psi0_, sizeof(cplx) * (size_t)n);
    for (int64_t k = 0; k < nsteps && rc == 0; ++k) {
        const double E = E_mid ? E_mid[k] : 0.0;
        rc = cn_one_step(p, E, states + k * n, states + (k + 1) * n, b, a, c, bs, as, cs, d);
    }
    if (rc) goto out;
    {
        const cplx* psiK = states + nsteps * n;
        double L = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            L += wgt[j] * (creal(psiK[j]) * creal(psiK[j]) + cimag(psiK[j]) * cimag(psiK[j]));
            lam[j] = wgt[j] * psiK[j];
        }
        *loss = L;
    }
    for (int64_t k = nsteps - 1; k >= 0 && rc == 0; --k) {
        const double E = E_mid ? E_mid[k] : 0.0;
        rc = or_cn_matrix(p, E, +1, (double*)b, (double*)a, (double*)c);     /* T_k */
        if (rc) break;
        rc = or_cn_matrix(p, E, -1, (double*)bs, (double*)as, (double*)cs);  /* S_k */
        if (rc) break;
        tridiag_conj_transpose(n, b, a, c, bh, ah, ch);                       /* T_k^H */
        rc = or_thomas(n, (double*)bh, (double*)ah, (double*)ch, (double*)lam, (double*)mu);
        if (rc) break;
        const cplx* psik = states + k * n;
        const cplx* psik1 = states + (k + 1) * n;
        const cplx dT = I * (p->dt / 2.0), dS = -I * (p->dt / 2.0);
        double g = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            const double xj = grid_x(p, j);
            const cplx v = dS * xj * psik[j] - dT * xj * psik1[j];
            g += 2.0 * creal(conj(mu[j]) * v);
        }
        dLdE[k] = g;
        tridiag_conj_transpose(n, bs, as, cs, bh, ah, ch);                    /* S_k^H */
        rc = or_tridiag_apply(n, (double*)bh, (double*)ah, (double*)ch, (double*)mu, (double*)lam);
    }
    if (rc == 0 && lam0_) memcpy(lam0_, lam, sizeof(cplx) * (size_t)n);
out:
    free(states);
    free(buf);
    return rc;
}
