// Host build of the library's arithmetic (cn_arith.cuh) for the CPU checks in
// test_df_arith.py (double-float) and test_f64_rcp.py (the binary64
// reciprocal).  Compiled with -ffp-contract=off.
#include "../paper_2205_00856_b300/csrc/cn_arith.cuh"
using namespace cnb;

extern "C" {
void shim_from_double(const double* x, float* hl, long n) {
    for (long i = 0; i < n; ++i) { df v = df_from_double(x[i]); hl[2 * i] = v.hi; hl[2 * i + 1] = v.lo; }
}
void shim_to_double(const float* hl, double* x, long n) {
    for (long i = 0; i < n; ++i) x[i] = df_to_double(df_make(hl[2 * i], hl[2 * i + 1]));
}
// op: 0 add, 1 mul, 2 mul_f (b.hi), 3 rcp (a), 4 rsqrt (a), 5 dot2 (a0 b0 + a1 b1), 6 dot2_add (c + a0 b0 + a1 b1)
void shim_op(int op, const float* a, const float* b, const float* c, const float* d, const float* e, float* out, long n) {
    for (long i = 0; i < n; ++i) {
        df A = df_make(a[2 * i], a[2 * i + 1]), B = df_make(b[2 * i], b[2 * i + 1]);
        df C = df_make(c[2 * i], c[2 * i + 1]), D = df_make(d[2 * i], d[2 * i + 1]);
        df E = df_make(e[2 * i], e[2 * i + 1]);
        df r;
        switch (op) {
        case 0: r = df_add(A, B); break;
        case 1: r = df_mul(A, B); break;
        case 2: r = df_mul_f(A, B.hi); break;
        case 3: r = df_rcp(A); break;
        case 4: r = df_rsqrt(A); break;
        case 5: r = df_dot2(A, B, C, D); break;
        default: r = df_dot2_add(E, A, B, C, D); break;
        }
        out[2 * i] = r.hi; out[2 * i + 1] = r.lo;
    }
}
// c + a0 b0 + a1 b1 + a2 b2 + a3 b3 on arrays of df pairs (a, b of length 4 per item)
void shim_dot4(const float* c, const float* a, const float* b, float* out, long n) {
    for (long i = 0; i < n; ++i) {
        df A[4], B[4];
        for (int k = 0; k < 4; ++k) {
            A[k] = df_make(a[8 * i + 2 * k], a[8 * i + 2 * k + 1]);
            B[k] = df_make(b[8 * i + 2 * k], b[8 * i + 2 * k + 1]);
        }
        df r = df_dot4_add(df_make(c[2 * i], c[2 * i + 1]), A[0], B[0], A[1], B[1], A[2], B[2], A[3], B[3]);
        out[2 * i] = r.hi; out[2 * i + 1] = r.lo;
    }
}
// complex c - a b - e f on (re.hi, re.lo, im.hi, im.lo)
void shim_csub2mul(const float* c, const float* a, const float* b, const float* e, const float* f, float* out, long n) {
    auto ld = [](const float* p, long i) { return mk(df_make(p[4 * i], p[4 * i + 1]), df_make(p[4 * i + 2], p[4 * i + 3])); };
    for (long i = 0; i < n; ++i) {
        cx<df> r = csub2mul(ld(c, i), ld(a, i), ld(b, i), ld(e, i), ld(f, i));
        out[4 * i] = r.re.hi; out[4 * i + 1] = r.re.lo; out[4 * i + 2] = r.im.hi; out[4 * i + 3] = r.im.lo;
    }
}
// complex ops on (re.hi, re.lo, im.hi, im.lo): 0 cmul(a,b), 1 cfma(c,a,b) = c + a b, 2 crcp(a)
void shim_cop(int op, const float* a, const float* b, const float* c, float* out, int* ok, long n) {
    for (long i = 0; i < n; ++i) {
        cx<df> A = mk(df_make(a[4 * i], a[4 * i + 1]), df_make(a[4 * i + 2], a[4 * i + 3]));
        cx<df> B = mk(df_make(b[4 * i], b[4 * i + 1]), df_make(b[4 * i + 2], b[4 * i + 3]));
        cx<df> Cc = mk(df_make(c[4 * i], c[4 * i + 1]), df_make(c[4 * i + 2], c[4 * i + 3]));
        bool k = true;
        cx<df> r = op == 0 ? cmul(A, B) : (op == 1 ? cfma(Cc, A, B) : crcp(A, k));
        out[4 * i] = r.re.hi; out[4 * i + 1] = r.re.lo; out[4 * i + 2] = r.im.hi; out[4 * i + 3] = r.im.lo;
        ok[i] = k;
    }
}
// binary64 addition and FMA on the integer pipe
void shim_d_add_int(const double* x, const double* y, double* z, long n) {
    for (long i = 0; i < n; ++i) z[i] = d_add_int(x[i], y[i]);
}
void shim_d_fma_int(const double* x, const double* y, const double* z, double* r, long n) {
    for (long i = 0; i < n; ++i) r[i] = d_fma_int(x[i], y[i], z[i]);
}
void shim_fma(const double* x, const double* y, const double* z, double* r, long n) {
    for (long i = 0; i < n; ++i) r[i] = fma(x[i], y[i], z[i]);
}
// binary64 reciprocal d_rcp and complex reciprocal crcp<double>
void shim_d_rcp(const double* q, double* y, int* ok, long n) {
    for (long i = 0; i < n; ++i) { bool k = true; y[i] = d_rcp(q[i], k); ok[i] = k; }
}
void shim_crcp_d(const double* z, double* w, int* ok, long n) {
    for (long i = 0; i < n; ++i) {
        bool k = true;
        cx<double> r = crcp(mk(z[2 * i], z[2 * i + 1]), k);
        w[2 * i] = r.re; w[2 * i + 1] = r.im; ok[i] = k;
    }
}
}
