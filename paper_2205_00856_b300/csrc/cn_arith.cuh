// cn_arith.cuh -- real and complex arithmetic used by the N-shaped CN kernels.
//
// Two real types share one kernel source:
//   double : native IEEE binary64 (on B300 the FP64 pipe issues ~1.6 FMA per
//            clock per SM, ~74x below FP32);
//   df     : double-float ("double-word") value hi + lo of two binary32 words,
//            |lo| <= ulp(hi)/2, ~48-bit significand.  Its operations are the
//            error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2,
//            TwoSum) and the double-word algorithms of Joldes, Muller and
//            Popescu, "Tight and rigorous error bounds for basic building blocks
//            of double-word arithmetic", ACM TOMS 44(2), 2017 (their Algorithms
//            1-2, 4, 6, 9 and 12 are named where used).  All binary32 steps use
//            __fadd_rn / __fmul_rn / __fmaf_rn so that the compiler can neither
//            contract nor reassociate them.
//
// The complex type cx<R> holds (re, im).  Complex numbers are stored in
// memory as complex128 (two doubles); df values are converted on load/store.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace cnb {

// ---------------------------------------------------------------- double-float
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }

// Fast2Sum (Dekker): exact s + t = a + b when |a| >= |b| (JMP17 Alg. 1).
__device__ __forceinline__ df fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float z = __fadd_rn(s, -a);
    return df_make(s, __fadd_rn(b, -z));
}
// 2Sum (Knuth/Moller): exact s + t = a + b for any a, b (JMP17 Alg. 2).
__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float ap = __fadd_rn(s, -b);
    float bp = __fadd_rn(s, -ap);
    float da = __fadd_rn(a, -ap);
    float db = __fadd_rn(b, -bp);
    return df_make(s, __fadd_rn(da, db));
}
// Fast2Mult: exact p + e = a * b with one FMA.
__device__ __forceinline__ df two_prod(float a, float b) {
    float p = __fmul_rn(a, b);
    return df_make(p, __fmaf_rn(a, b, -p));
}

__device__ __forceinline__ df df_from_double(double x) {
    float h = __double2float_rn(x);
    float l = __double2float_rn(x - (double)h);
    return df_make(h, l);
}
__device__ __forceinline__ double df_to_double(df a) { return (double)a.hi + (double)a.lo; }

// AccurateDWPlusDW (JMP17 Alg. 6): relative error <= 3u^2 + 13u^3.
__device__ __forceinline__ df operator+(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    df t = two_sum(x.lo, y.lo);
    float c = __fadd_rn(s.lo, t.hi);
    df v = fast_two_sum(s.hi, c);
    float w = __fadd_rn(t.lo, v.lo);
    return fast_two_sum(v.hi, w);
}
__device__ __forceinline__ df operator-(df x) { return df_make(-x.hi, -x.lo); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }

// DWTimesDW3 (JMP17 Alg. 12, with FMA): relative error <= 4u^2.
__device__ __forceinline__ df operator*(df x, df y) {
    df c = two_prod(x.hi, y.hi);
    float tl0 = __fmul_rn(x.lo, y.lo);
    float tl1 = __fmaf_rn(x.hi, y.lo, tl0);
    float cl2 = __fmaf_rn(x.lo, y.hi, tl1);
    float cl3 = __fadd_rn(c.lo, cl2);
    return fast_two_sum(c.hi, cl3);
}
// DWTimesFP3 (JMP17 Alg. 9): double-float times a binary32 value, error <= 2u^2.
__device__ __forceinline__ df df_mul_f(df x, float y) {
    df c = two_prod(x.hi, y);
    float cl3 = __fmaf_rn(x.lo, y, c.lo);
    return fast_two_sum(c.hi, cl3);
}
// Reciprocal by one Newton step on the correctly rounded binary32 reciprocal:
// t = RN(1/y_h) has relative error <= u; e = 1 - y t is formed with two FMAs
// (the first is exact); 1/y = t (1 + e + e^2 + ...) ~= t + t e.
__device__ __forceinline__ df df_rcp(df y) {
    float t = __frcp_rn(y.hi);
    float e1 = __fmaf_rn(-y.hi, t, 1.0f);
    float e2 = __fmaf_rn(-y.lo, t, e1);
    return fast_two_sum(t, __fmul_rn(t, e2));
}
__device__ __forceinline__ df df_fma(df a, df b, df c) { return a * b + c; }

// ------------------------------------------------------------- real traits
template <class R> struct RealOps;

template <> struct RealOps<double> {
    static __device__ __forceinline__ double from_d(double x) { return x; }
    static __device__ __forceinline__ double to_d(double x) { return x; }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double fma(double a, double b, double c) { return __fma_rn(a, b, c); }
    static __device__ __forceinline__ bool finite_pos(double x) { return x > 0.0 && x < 1.0e300; }
};
template <> struct RealOps<df> {
    static __device__ __forceinline__ df from_d(double x) { return df_from_double(x); }
    static __device__ __forceinline__ double to_d(df x) { return df_to_double(x); }
    static __device__ __forceinline__ df rcp(df x) { return df_rcp(x); }
    static __device__ __forceinline__ df fma(df a, df b, df c) { return df_fma(a, b, c); }
    static __device__ __forceinline__ bool finite_pos(df x) { return x.hi > 0.0f && x.hi < 1.0e37f; }
};

// ---------------------------------------------------------------- complex
template <class R> struct cx {
    R re, im;
};

template <class R> __device__ __forceinline__ cx<R> mk(R re, R im) { cx<R> z; z.re = re; z.im = im; return z; }
template <class R> __device__ __forceinline__ cx<R> czero() {
    return mk<R>(RealOps<R>::from_d(0.0), RealOps<R>::from_d(0.0));
}
template <class R> __device__ __forceinline__ cx<R> operator+(cx<R> a, cx<R> b) { return mk<R>(a.re + b.re, a.im + b.im); }
template <class R> __device__ __forceinline__ cx<R> operator-(cx<R> a, cx<R> b) { return mk<R>(a.re - b.re, a.im - b.im); }
template <class R> __device__ __forceinline__ cx<R> operator-(cx<R> a) { return mk<R>(-a.re, -a.im); }
// (a + ib)(c + id) = (ac - bd) + i(ad + bc)
template <class R> __device__ __forceinline__ cx<R> operator*(cx<R> a, cx<R> b) {
    return mk<R>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <class R> __device__ __forceinline__ cx<R> cscale(cx<R> a, R s) { return mk<R>(a.re * s, a.im * s); }
// i * z
template <class R> __device__ __forceinline__ cx<R> cmul_i(cx<R> z) { return mk<R>(-z.im, z.re); }
template <class R> __device__ __forceinline__ R cabs2(cx<R> z) { return z.re * z.re + z.im * z.im; }
// 1/z = conj(z) / |z|^2 (one real reciprocal); ok <- false when |z|^2 is 0, inf or NaN
template <class R> __device__ __forceinline__ cx<R> crcp(cx<R> z, bool& ok) {
    R m2 = cabs2(z);
    ok = ok && RealOps<R>::finite_pos(m2);
    R q = RealOps<R>::rcp(m2);
    return mk<R>(z.re * q, -(z.im * q));
}

// complex128 memory <-> cx<R>
template <class R> __device__ __forceinline__ cx<R> cload(const double2* p) {
    double2 v = *p;
    return mk<R>(RealOps<R>::from_d(v.x), RealOps<R>::from_d(v.y));
}
template <class R> __device__ __forceinline__ void cstore(double2* p, cx<R> z) {
    *p = make_double2(RealOps<R>::to_d(z.re), RealOps<R>::to_d(z.im));
}

}  // namespace cnb
