// cn_arith.cuh -- real and complex arithmetic of the N-shaped CN kernels.
//
// Two real types share the kernel sources:
//   double : native IEEE binary64.  On B300 the FP64 pipe issues ~1.6 FMA per
//            clock per SM, ~74x below the FP32 pipe.
//   df     : double-float ("double-word") value hi + lo of two binary32 words
//            with |lo| <= ulp(hi)/2, ~48-bit significand, built only from
//            binary32 FMA/add/mul and integer instructions, so it runs on the
//            FP32 pipe.  Its operations are the error-free transformations of
//            Dekker (1971) and Knuth (TAOCP vol. 2: TwoSum) and the double-word
//            algorithms of Joldes, Muller and Popescu, "Tight and rigorous error
//            bounds for basic building blocks of double-word arithmetic", ACM
//            TOMS 44(2), 2017 (JMP17; the algorithm used is named at each
//            function).  Complex products and sums of products are evaluated as
//            one double-word dot product per component (exact binary32 products
//            by FMA, one TwoSum chain, one final renormalisation), a
//            restatement of the compensated dot product of Ogita, Rump and
//            Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26(6),
//            2005, truncated to double-word precision.
//
// Range of df: binary32 exponents.  Conversions from binary64 flush |x| < 2^-70
// to zero (that is below anything that contributes to a normalised state);
// values must stay below ~1e30.  The CN coefficients and normalised states
// satisfy both bounds.
//
// Every binary32 step goes through f_add / f_mul / f_fma, which the compiler
// may neither contract nor reassociate (device: __fadd_rn etc.; host builds of
// the checks use -ffp-contract=off), so the functions are bit-reproducible on
// host and device except for the reciprocal / rsqrt seeds.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "cn_debug.cuh"
#if !defined(__CUDA_ARCH__)
#include <math.h>
#endif

#define CNB_HD __host__ __device__ __forceinline__

namespace cnb {

// ------------------------------------------------------------ binary32 steps
CNB_HD float f_add(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fadd_rn(a, b);
#else
    return a + b;
#endif
}
CNB_HD float f_mul(float a, float b) {
#ifdef __CUDA_ARCH__
    return __fmul_rn(a, b);
#else
    return a * b;
#endif
}
CNB_HD float f_fma(float a, float b, float c) {
#ifdef __CUDA_ARCH__
    return __fmaf_rn(a, b, c);
#else
    return fmaf(a, b, c);
#endif
}
// correctly rounded reciprocal and reciprocal square root (seeds only)
CNB_HD float f_rcp(float a) {
#ifdef __CUDA_ARCH__
    return __frcp_rn(a);
#else
    return 1.0f / a;
#endif
}
CNB_HD float f_rsqrt(float a) {
#ifdef __CUDA_ARCH__
    return __frsqrt_rn(a);
#else
    return (float)(1.0 / sqrt((double)a));
#endif
}
CNB_HD int32_t f_bits(float a) {
#ifdef __CUDA_ARCH__
    return __float_as_int(a);
#else
    int32_t i; memcpy(&i, &a, 4); return i;
#endif
}
CNB_HD float f_from_bits(int32_t i) {
#ifdef __CUDA_ARCH__
    return __int_as_float(i);
#else
    float a; memcpy(&a, &i, 4); return a;
#endif
}
CNB_HD int64_t d_bits(double a) {
#ifdef __CUDA_ARCH__
    return __double_as_longlong(a);
#else
    int64_t i; memcpy(&i, &a, 8); return i;
#endif
}
CNB_HD double d_from_bits(int64_t i) {
#ifdef __CUDA_ARCH__
    return __longlong_as_double(i);
#else
    double a; memcpy(&a, &i, 8); return a;
#endif
}
// high 64 bits of a 64 x 64-bit product; leading zeros of a nonzero word
CNB_HD uint64_t u64_mulhi(uint64_t a, uint64_t b) {
#ifdef __CUDA_ARCH__
    return __umul64hi(a, b);
#else
    return (uint64_t)(((unsigned __int128)a * b) >> 64);
#endif
}
CNB_HD int u64_clz(uint64_t a) {
#ifdef __CUDA_ARCH__
    return __clzll((long long)a);
#else
    return __builtin_clzll(a);
#endif
}

// 1/q for binary64 q, without a division and with one binary64 operation.
// Seed: the top 23 bits of q's significand as a binary32 value f in [1, 2),
// its correctly rounded binary32 reciprocal r, and q's exponent applied with
// integer operations, so y0 = r 2^-e with |1 - q y0| <= 2^-23 + 2^-24 (the
// truncation of f and the rounding of 1/f).  Refinement: with e = 1 - q y0 (one
// binary64 FMA), 1/q = y0 / (1 - e) = y0 (1 + e + e^2 + e^3 + ...), the series
// form of the Newton-Raphson reciprocal iteration (Goldschmidt, MIT thesis 1964;
// Markstein, IBM J. Res. Dev. 34(1), 1990), evaluated here to its cubic term in
// integer fixed point -- T = (e + e^2 + e^3) 2^75 from e's bits (|e| < 2^-22, so
// |e| 2^75 < 2^53), Z = R (2^75 + T) exactly in 128 bits, R = r's 24-bit
// significand -- and rounded once to 53 bits, to nearest even.  On B300 the
// FP64 pipe is the binary64 kernels' limit while the integer pipe idles, so the
// ~60 integer instructions replace two FMAs of the FP64 pipe.  Error: the omitted
// e^4 + ... < 2^-88 relative, the truncations of the three terms and the
// rounding of e below 4 units of 2^-75 relative, and the final rounding, 1/2 ulp:
// |y - 1/q| <= (1/2 + 2^-20) ulp.  Range: positive normal q with biased
// exponent 1..2044 (so that 1/q is normal); anything else (zero, subnormal,
// negative, huge, inf, NaN) clears `ok` and returns NaN.  The checks run on
// integer bits, and every shift count stays in 0..63 for any input.
// Bit-reproducible on host and device (correctly rounded binary32 reciprocal,
// binary64 FMA, integer arithmetic).
CNB_HD double d_rcp(double q, bool& ok) {
    const int64_t b = d_bits(q);
    const uint32_t hi = (uint32_t)((uint64_t)b >> 32);
    const uint32_t E = hi >> 20;  // sign and biased exponent: 1..2044 for the valid range
    const float f = f_from_bits((int32_t)(0x3F800000u | ((hi & 0xFFFFFu) << 3) | ((uint32_t)b >> 29)));
    const int32_t rb = f_bits(f_rcp(f));  // r in (1/2, 1]
    const int64_t ye = (int64_t)(rb >> 23) + 1919 - (int64_t)E;  // biased exponent of r 2^-e
    const double y0 = d_from_bits((int64_t)((uint64_t)ye << 52) | ((int64_t)(rb & 0x7FFFFF) << 29));
    const double e = fma(-q, y0, 1.0);
    // |e| 2^75 = M 2^(x - 1000), x e's biased exponent (<= 1000), truncated to an integer
    const uint64_t eb = (uint64_t)d_bits(e);
    const int x = (int)((eb >> 52) & 0x7FF);
    const int s1 = 1000 - x;
    const uint64_t M = (eb & 0xFFFFFFFFFFFFFull) | 0x10000000000000ull;
    const uint64_t E1 = (x != 0 && s1 >= 0 && s1 < 64) ? (M >> s1) : 0;  // |e| 2^75
    const uint64_t E2 = u64_mulhi(E1, E1) >> 11;                            // e^2 2^75
    const uint64_t E3 = u64_mulhi(E1, E2) >> 11;                            // |e|^3 2^75
    const int64_t T = (eb >> 63) ? (int64_t)E2 - (int64_t)(E1 + E3) : (int64_t)(E1 + E2 + E3);
    // Z = R (2^75 + T) = y in units of 2^(er - 98 - eq), er = r's and eq = q's exponent
    const uint64_t R = (uint64_t)((rb & 0x7FFFFF) | 0x800000);
    const uint64_t Ta = T < 0 ? (uint64_t)0 - (uint64_t)T : (uint64_t)T;
    const uint64_t Pl = R * Ta, Ph = u64_mulhi(R, Ta);
    const uint64_t Zl = T < 0 ? (uint64_t)0 - Pl : Pl;
    const uint64_t Zh = T < 0 ? (R << 11) - Ph - (uint64_t)(Pl != 0) : (R << 11) + Ph;
    // Z's leading bit is bit 52 + sh of the 128 (sh = 45..47 for valid q): 53 bits from
    // there, round to nearest even on the next bit and the sticky bits below it
    const int sh0 = 75 - u64_clz(Zh | 1);
    const int sh = sh0 < 2 ? 2 : (sh0 > 63 ? 63 : sh0);
    uint64_t mant = (Zh << (64 - sh)) | (Zl >> sh);
    const uint64_t rnd = (Zl >> (sh - 1)) & 1u;
    const uint64_t sticky = (Zl << (65 - sh)) != 0;
    mant += rnd & (sticky | (mant & 1u));
    // biased exponent sh + er - E + 2000; the implicit bit in mant carries into it
    const int64_t Ey = (int64_t)sh + (int64_t)(rb >> 23) - 127 - (int64_t)E + 2000;
    const double y = d_from_bits((int64_t)(((uint64_t)(Ey - 1) << 52) + mant));
    const bool in = (E - 1u) < 2044u;
    ok = ok && in;
    return in ? y : d_from_bits(0x7FF8000000000000ll);
}

// binary64 addition and multiplication as FMAs.  On B300 the FP64 pipe retires
// FMAs ~19 % faster than separate additions or multiplications (5.60e11 vs
// 4.72e11 per second over all SMs, independent chains, whatever the operand
// values).  x + y equals fma(x, 1, y) and x y equals fma(x, y, -0) bit for bit,
// signed zeros included; the 1 and the -0 are read from constant memory, whose
// contents the compiler does not assume, so that it keeps the FMAs.
#ifdef __CUDACC__
__constant__ double c_fp64_one = 1.0;
__constant__ double c_fp64_mzero = -0.0;
#endif
CNB_HD double d_add(double a, double b) {
#ifdef __CUDA_ARCH__
    return fma(a, c_fp64_one, b);
#else
    return a + b;
#endif
}
CNB_HD double d_sub(double a, double b) {
#ifdef __CUDA_ARCH__
    return fma(-b, c_fp64_one, a);
#else
    return a - b;
#endif
}
CNB_HD double d_mul(double a, double b) {
#ifdef __CUDA_ARCH__
    return fma(a, b, c_fp64_mzero);
#else
    return a * b;
#endif
}

// The operands' bits move to integer registers through an opaque move: the compiler
// would otherwise fold the sign-bit masks below back into FP64 absolute values.
CNB_HD uint64_t d_bits_opaque(double a) {
#ifdef __CUDA_ARCH__
    uint64_t r;
    asm("mov.b64 %0, %1;" : "=l"(r) : "d"(a));
    return r;
#else
    return (uint64_t)d_bits(a);
#endif
}

// x + y on the integer pipe, the IEEE binary64 sum rounded to nearest even bit for
// bit (signed zeros, subnormals, overflow, infinities; a NaN result is a quiet NaN):
// the operands ordered by magnitude, their significands with three guard bits (the
// lowest a sticky bit) aligned, added or subtracted, normalised by at most one place
// right or any number left (not below the subnormal exponent), and rounded.  For
// additions off the kernels' dependency chains, where the FP64 pipe is the limit and
// the integer pipe idles.
CNB_HD double d_add_int(double x, double y) {
    const uint64_t SIGN = 0x8000000000000000ull, FRAC = 0xFFFFFFFFFFFFFull, HID = 0x10000000000000ull;
    uint64_t a = d_bits_opaque(x), b = d_bits_opaque(y);
    if ((a & ~SIGN) < (b & ~SIGN)) {
        const uint64_t t = a;
        a = b;
        b = t;
    }
    const uint64_t am = a & ~SIGN, bm = b & ~SIGN;
    const int ea = (int)(am >> 52), eb = (int)(bm >> 52);
    if (ea == 2047) {  // an infinity or a NaN, the larger magnitude
        if (am > 0x7FF0000000000000ull) return d_from_bits((int64_t)(a | 0x0008000000000000ull));
        if (bm == 0x7FF0000000000000ull && ((a ^ b) & SIGN)) return d_from_bits(0x7FF8000000000000ll);
        return d_from_bits((int64_t)a);
    }
    if (bm == 0) return d_from_bits((int64_t)(am == 0 ? (a & b) : a));  // (-0) + (-0) = -0, else +0
    const int e0 = ea ? ea : 1;
    const int d = e0 - (eb ? eb : 1);  // >= 0
    const uint64_t ma = ((am & FRAC) | (ea ? HID : 0)) << 3;
    const uint64_t mb0 = ((bm & FRAC) | (eb ? HID : 0)) << 3;
    const uint64_t mb = d == 0 ? mb0 : (d >= 64 ? (uint64_t)1 : ((mb0 >> d) | (uint64_t)((mb0 << (64 - d)) != 0)));
    uint64_t m = ((a ^ b) & SIGN) ? ma - mb : ma + mb;
    if (m == 0) return 0.0;  // exact cancellation: +0
    int e = e0;
    const int lz = u64_clz(m) - 8;  // the leading bit belongs at bit 55
    if (lz < 0) {
        m = (m >> 1) | (m & 1u);
        e += 1;
    } else if (lz > 0) {
        const int sl = lz < e - 1 ? lz : e - 1;
        m <<= sl;
        e -= sl;
    }
    if (e >= 2047) return d_from_bits((int64_t)((a & SIGN) | 0x7FF0000000000000ull));
    const uint64_t g = m & 7u;
    uint64_t q = m >> 3;
    q += (uint64_t)(g > 4u || (g == 4u && (q & 1u)));
    // normal: q holds the hidden bit (a carry into 2^53 bumps the exponent); subnormal: e == 1
    return d_from_bits((int64_t)((a & SIGN) | (((uint64_t)(e - 1) << 52) + q)));
}

// 128-bit unsigned arithmetic for the integer-pipe FMA
struct u128 {
    uint64_t hi, lo;
};
CNB_HD u128 u128_of(uint64_t hi, uint64_t lo) {
    u128 r;
    r.hi = hi;
    r.lo = lo;
    return r;
}
CNB_HD u128 u128_mul(uint64_t a, uint64_t b) { return u128_of(u64_mulhi(a, b), a * b); }
CNB_HD u128 u128_add(u128 a, u128 b) {
    const uint64_t lo = a.lo + b.lo;
    return u128_of(a.hi + b.hi + (uint64_t)(lo < a.lo), lo);
}
CNB_HD u128 u128_sub(u128 a, u128 b) {  // a >= b
    return u128_of(a.hi - b.hi - (uint64_t)(a.lo < b.lo), a.lo - b.lo);
}
CNB_HD bool u128_ge(u128 a, u128 b) { return a.hi != b.hi ? a.hi > b.hi : a.lo >= b.lo; }
// shifts by 0..127 (anything larger gives 0)
CNB_HD u128 u128_shr(u128 a, int s) {
    if (s <= 0) return a;
    if (s >= 128) return u128_of(0, 0);
    if (s >= 64) return u128_of(0, a.hi >> (s - 64));
    return u128_of(a.hi >> s, (a.lo >> s) | (a.hi << (64 - s)));
}
CNB_HD u128 u128_shl(u128 a, int s) {
    if (s <= 0) return a;
    if (s >= 128) return u128_of(0, 0);
    if (s >= 64) return u128_of(a.lo << (s - 64), 0);
    return u128_of((a.hi << s) | (a.lo >> (64 - s)), a.lo << s);
}
// index of the leading bit (a != 0)
CNB_HD int u128_top(u128 a) { return a.hi ? 127 - u64_clz(a.hi) : 63 - u64_clz(a.lo | 1); }
// a 2^s: shifted left, or right with the bits shifted out OR-ed into bit 0 (sticky)
CNB_HD u128 u128_place(u128 a, int s) {
    if (s >= 0) return u128_shl(a, s);
    const int r = -s;
    u128 v = u128_shr(a, r);
    const u128 out = r >= 128 ? a : u128_shl(a, 128 - r);
    if ((out.hi | out.lo) != 0) v.lo |= 1u;
    return v;
}
// the binary64 bits (sign clear) of U 2^X, U != 0, rounded to nearest even;
// subnormal results by the same rounding at the subnormal position, overflow to
// infinity
CNB_HD uint64_t u128_round_pack(u128 U, int X) {
    const int t = u128_top(U);
    int Eo = t + X + 1023;  // biased exponent of a normal result
    int sh = t - 52;        // bits below the 53 kept
    if (Eo < 1) {
        sh += 1 - Eo;
        Eo = 0;
    }
    if (Eo >= 2047) return 0x7FF0000000000000ull;
    uint64_t m;
    if (sh <= 0) {
        m = U.lo << (-sh);  // t <= 52: exact
    } else {
        if (sh - 1 > t) return 0;  // below half the smallest subnormal
        m = u128_shr(U, sh).lo;
        const uint64_t rnd = u128_shr(U, sh - 1).lo & 1u;
        const u128 low = u128_shl(U, 129 - sh);  // the bits below the rounding bit
        const uint64_t sticky = (low.hi | low.lo) != 0;
        m += rnd & (sticky | (m & 1u));
    }
    return Eo >= 1 ? ((uint64_t)(Eo - 1) << 52) + m : m;  // a carry into 2^53 (2^52) bumps the exponent
}
// fma(x, y, z) on the integer pipe, the IEEE binary64 x y + z rounded once to nearest
// even bit for bit (signed zeros, subnormals, overflow, infinities; a NaN result is
// a quiet NaN): the exact 106-bit product and z placed in a 128-bit window whose
// bit 125 holds the larger's leading bit (a smaller operand reaching below bit 0
// folds into a sticky bit there, far below any rounding position: only operands
// within ~20 binades of each other can cancel, and those fit whole), added or
// subtracted, rounded.  For FMAs that feed no recurrence (see d_add_int).
CNB_HD double d_fma_int(double x, double y, double z) {
    const uint64_t SIGN = 0x8000000000000000ull, FRAC = 0xFFFFFFFFFFFFFull, HID = 0x10000000000000ull;
    const uint64_t INF = 0x7FF0000000000000ull, QNAN = 0x7FF8000000000000ull;
    const uint64_t a = d_bits_opaque(x), b = d_bits_opaque(y), c = d_bits_opaque(z);
    const uint64_t sp = (a ^ b) & SIGN, sc = c & SIGN;
    const uint64_t am = a & ~SIGN, bm = b & ~SIGN, cm = c & ~SIGN;
    if (am > INF || bm > INF || cm > INF) return d_from_bits((int64_t)QNAN);
    const bool pzero = am == 0 || bm == 0;
    if (am == INF || bm == INF) {
        if (pzero || (cm == INF && sc != sp)) return d_from_bits((int64_t)QNAN);  // inf 0, inf - inf
        return d_from_bits((int64_t)(sp | INF));
    }
    if (cm == INF) return d_from_bits((int64_t)c);
    if (pzero) return d_from_bits((int64_t)(cm == 0 ? (sp & sc) : c));  // an exact signed zero plus z
    const int ea = (int)(am >> 52), eb = (int)(bm >> 52), ec = (int)(cm >> 52);
    const uint64_t ma = (am & FRAC) | (ea ? HID : 0), mb = (bm & FRAC) | (eb ? HID : 0);
    const int Xp = (ea ? ea : 1) + (eb ? eb : 1) - 2150;  // x y = P 2^Xp exactly
    const u128 P = u128_mul(ma, mb);
    if (cm == 0) return d_from_bits((int64_t)(sp | u128_round_pack(P, Xp)));
    const uint64_t mc = (cm & FRAC) | (ec ? HID : 0);
    const int Xc = (ec ? ec : 1) - 1075;  // z = mc 2^Xc
    const int tP = u128_top(P) + Xp, tC = (63 - u64_clz(mc)) + Xc;
    const int W0 = (tP > tC ? tP : tC) - 125;  // exponent of the window's bit 0
    const u128 Pw = u128_place(P, Xp - W0), Cw = u128_place(u128_of(0, mc), Xc - W0);
    u128 R;
    uint64_t rs;
    if (sp == sc) {
        R = u128_add(Pw, Cw);
        rs = sp;
    } else if (u128_ge(Pw, Cw)) {
        R = u128_sub(Pw, Cw);
        rs = sp;
    } else {
        R = u128_sub(Cw, Pw);
        rs = sc;
    }
    if ((R.hi | R.lo) == 0) return 0.0;  // exact cancellation: +0
    return d_from_bits((int64_t)(rs | u128_round_pack(R, W0)));
}

CNB_HD float i2f(int32_t i) {
#ifdef __CUDA_ARCH__
    return __int2float_rn(i);
#else
    return (float)i;
#endif
}
// 2^k as binary32 for -126 <= k <= 127
CNB_HD float pow2f(int k) { return f_from_bits((k + 127) << 23); }

// ------------------------------------------------------------ double-float
struct df {
    float hi, lo;
};
CNB_HD df df_make(float h, float l) { df r; r.hi = h; r.lo = l; return r; }

// Fast2Sum (Dekker; JMP17 Alg. 1): s + t = a + b exactly when exp(a) >= exp(b).
CNB_HD df fast_two_sum(float a, float b) {
    float s = f_add(a, b);
    float z = f_add(s, -a);
    return df_make(s, f_add(b, -z));
}
// 2Sum (Knuth, Moller; JMP17 Alg. 2): s + t = a + b exactly.
CNB_HD df two_sum(float a, float b) {
    float s = f_add(a, b);
    float ap = f_add(s, -b);
    float bp = f_add(s, -ap);
    return df_make(s, f_add(f_add(a, -ap), f_add(b, -bp)));
}
// Fast2Mult with an FMA: p + e = a b exactly.
CNB_HD df two_prod(float a, float b) {
    float p = f_mul(a, b);
    return df_make(p, f_fma(a, b, -p));
}

CNB_HD df df_neg(df a) { return df_make(-a.hi, -a.lo); }

// SloppyDWPlusDW (JMP17 Alg. 5): absolute error <= 2u^2 (|x| + |y|) -- ample for
// the well-conditioned sums of the elimination (no relative bound is needed).
CNB_HD df df_add(df x, df y) {
    df s = two_sum(x.hi, y.hi);
    float v = f_add(x.lo, y.lo);
    float w = f_add(s.lo, v);
    return fast_two_sum(s.hi, w);
}
CNB_HD df df_sub(df x, df y) { return df_add(x, df_neg(y)); }
// DWPlusFP (JMP17 Alg. 4): double-float plus binary32, relative error <= 2u^2.
CNB_HD df df_add_f(df x, float y) {
    df s = two_sum(x.hi, y);
    float v = f_add(x.lo, s.lo);
    return fast_two_sum(s.hi, v);
}
// DWTimesDW2 (JMP17 Alg. 11): relative error <= 5u^2.
CNB_HD df df_mul(df x, df y) {
    df c = two_prod(x.hi, y.hi);
    float t = f_mul(x.hi, y.lo);
    float cl2 = f_fma(x.lo, y.hi, t);
    return fast_two_sum(c.hi, f_add(c.lo, cl2));
}
// DWTimesFP3 (JMP17 Alg. 9): relative error <= 2u^2.
CNB_HD df df_mul_f(df x, float y) {
    df c = two_prod(x.hi, y);
    return fast_two_sum(c.hi, f_fma(x.lo, y, c.lo));
}
// 1/y: one Newton step t + t (1 - y t) on the correctly rounded binary32
// reciprocal t (relative error <= u), with the residual 1 - y t formed by two
// FMAs (the first is exact); relative error ~ u^2.
CNB_HD df df_rcp(df y) {
    float t = f_rcp(y.hi);
    float e1 = f_fma(-y.hi, t, 1.0f);
    float e2 = f_fma(-y.lo, t, e1);
    return fast_two_sum(t, f_mul(t, e2));
}
// 1/sqrt(q), q > 0: one Newton step y = t + t (1 - q t^2) / 2 on the correctly
// rounded binary32 value t; q t^2 is formed from the exact square t^2 = p + e.
CNB_HD df df_rsqrt(df q) {
    float t = f_rsqrt(q.hi);
    df t2 = two_prod(t, t);
    df qt2 = df_mul(q, t2);                       // ~ 1
    df r = df_add_f(df_neg(qt2), 1.0f);           // 1 - q t^2, tiny
    float corr = f_mul(f_mul(t, 0.5f), f_add(r.hi, r.lo));
    return fast_two_sum(t, corr);
}

// binary64 -> double-float with integer operations only (no FP64 pipe work):
// hi = the 53-bit significand rounded to 24 bits, lo = the remainder rounded
// to 24 bits; |x| < 2^-70 (incl. zero and subnormals) gives 0.
CNB_HD df df_from_double(double x) {
    const int64_t b = d_bits(x);
    const int e = (int)((b >> 52) & 0x7FF) - 1023;
    if (e < -70) return df_make(0.0f, 0.0f);
    if (e > 126) {
        float inf = f_from_bits(0x7F800000 | (b < 0 ? (int32_t)0x80000000 : 0));
        return df_make(inf, 0.0f);
    }
    const uint64_t M = ((uint64_t)b & 0xFFFFFFFFFFFFFull) | (1ull << 52);
    uint32_t hm = (uint32_t)(M >> 29);              // 24 leading bits
    int32_t rem = (int32_t)(M & 0x1FFFFFFFu);       // 29 trailing bits
    if (rem >= (1 << 28)) { hm += 1; rem -= (1 << 29); }
    // hm in [2^23, 2^24]: hm - 2^23 carries into the exponent field when hm = 2^24
    float hi = f_from_bits(((e + 127) << 23) + (int32_t)(hm - (1u << 23)));
    float lo = f_mul(i2f(rem), pow2f(e - 52));
    if (b < 0) { hi = -hi; lo = -lo; }
    return df_make(hi, lo);
}

// double-float -> binary64 with integer operations only: the exact sum
// hi + lo, truncated to 53 bits when lo reaches below the last bit of hi's
// binary64 significand (error < 2^-52 relative).
CNB_HD double df_to_double(df v) {
    const int32_t hb = f_bits(v.hi), lb = f_bits(v.lo);
    const int eh = (hb >> 23) & 0xFF;
    if (eh == 0) return 0.0;                                    // zero (subnormals flushed)
    if (eh == 0xFF) return d_from_bits(((int64_t)(hb < 0) << 63) | (0x7FFll << 52) | ((int64_t)(hb & 0x7FFFFF) << 29));
    int64_t E = eh - 127;                                        // exponent of hi
    int64_t S = (int64_t)((hb & 0x7FFFFF) | 0x800000) << 29;    // 53-bit significand, unit 2^(E-52)
    const int el = (lb >> 23) & 0xFF;
    if (el != 0) {
        int64_t ml = (lb & 0x7FFFFF) | 0x800000;                 // 24-bit significand, unit 2^(El-23)
        int sh = (el - 127) - 23 - ((int)E - 52);                // shift to unit 2^(E-52)
        int64_t L = sh >= 0 ? (sh < 40 ? (ml << sh) : 0) : (sh > -40 ? (ml >> -sh) : 0);
        S += ((lb < 0) == (hb < 0)) ? L : -L;
        if (S >= (1ll << 53)) { S >>= 1; E += 1; }
        else if (S < (1ll << 52)) { S <<= 1; E -= 1; }
    }
    const int64_t bits = ((int64_t)(hb < 0) << 63) | ((E + 1023) << 52) | (S & 0xFFFFFFFFFFFFFll);
    return d_from_bits(bits);
}

// Double-word dot products, one renormalisation each (see header comment).
// sum_k a_k b_k for two terms: a0 b0 + a1 b1.
CNB_HD df df_dot2(df a0, df b0, df a1, df b1) {
    df p0 = two_prod(a0.hi, b0.hi);
    df p1 = two_prod(a1.hi, b1.hi);
    df s = two_sum(p0.hi, p1.hi);
    float e = f_add(f_add(p0.lo, p1.lo), s.lo);
    e = f_fma(a0.hi, b0.lo, e);
    e = f_fma(a0.lo, b0.hi, e);
    e = f_fma(a1.hi, b1.lo, e);
    e = f_fma(a1.lo, b1.hi, e);
    return two_sum(s.hi, e);
}
// c + a0 b0 + a1 b1
CNB_HD df df_dot2_add(df c, df a0, df b0, df a1, df b1) {
    df p0 = two_prod(a0.hi, b0.hi);
    df p1 = two_prod(a1.hi, b1.hi);
    df s = two_sum(p0.hi, p1.hi);
    df t = two_sum(c.hi, s.hi);
    float e = f_add(f_add(p0.lo, p1.lo), f_add(s.lo, t.lo));
    e = f_add(e, c.lo);
    e = f_fma(a0.hi, b0.lo, e);
    e = f_fma(a0.lo, b0.hi, e);
    e = f_fma(a1.hi, b1.lo, e);
    e = f_fma(a1.lo, b1.hi, e);
    return two_sum(t.hi, e);
}

// c + a0 b0 + a1 b1 + a2 b2 + a3 b3: four exact products, the five leading terms
// summed by a TwoSum tree, every error term and cross product collected in one
// binary32 sum, one final renormalisation.
CNB_HD df df_dot4_add(df c, df a0, df b0, df a1, df b1, df a2, df b2, df a3, df b3) {
    df p0 = two_prod(a0.hi, b0.hi);
    df p1 = two_prod(a1.hi, b1.hi);
    df p2 = two_prod(a2.hi, b2.hi);
    df p3 = two_prod(a3.hi, b3.hi);
    df s01 = two_sum(p0.hi, p1.hi);
    df s23 = two_sum(p2.hi, p3.hi);
    df s = two_sum(s01.hi, s23.hi);
    df t = two_sum(c.hi, s.hi);
    float e = f_add(f_add(f_add(p0.lo, p1.lo), f_add(p2.lo, p3.lo)), f_add(f_add(s01.lo, s23.lo), f_add(s.lo, t.lo)));
    e = f_add(e, c.lo);
    e = f_fma(a0.hi, b0.lo, e);
    e = f_fma(a0.lo, b0.hi, e);
    e = f_fma(a1.hi, b1.lo, e);
    e = f_fma(a1.lo, b1.hi, e);
    e = f_fma(a2.hi, b2.lo, e);
    e = f_fma(a2.lo, b2.hi, e);
    e = f_fma(a3.hi, b3.lo, e);
    e = f_fma(a3.lo, b3.hi, e);
    return two_sum(t.hi, e);
}

// ------------------------------------------------------------ complex
template <class R> struct cx {
    R re, im;
};
template <class R> CNB_HD cx<R> mk(R re, R im) { cx<R> z; z.re = re; z.im = im; return z; }

// --- double
CNB_HD cx<double> cadd(cx<double> a, cx<double> b) { return mk(d_add(a.re, b.re), d_add(a.im, b.im)); }
CNB_HD cx<double> csub(cx<double> a, cx<double> b) { return mk(d_sub(a.re, b.re), d_sub(a.im, b.im)); }
CNB_HD cx<double> cneg(cx<double> a) { return mk(-a.re, -a.im); }
CNB_HD cx<double> cmul(cx<double> a, cx<double> b) {
    return mk(fma(a.re, b.re, d_mul(-a.im, b.im)), fma(a.re, b.im, d_mul(a.im, b.re)));
}
// c + a b
CNB_HD cx<double> cfma(cx<double> c, cx<double> a, cx<double> b) {
    return mk(fma(a.re, b.re, fma(-a.im, b.im, c.re)), fma(a.re, b.im, fma(a.im, b.re, c.im)));
}
// c - a b - e f
CNB_HD cx<double> csub2mul(cx<double> c, cx<double> a, cx<double> b, cx<double> e, cx<double> f) {
    return mk(fma(-a.re, b.re, fma(a.im, b.im, fma(-e.re, f.re, fma(e.im, f.im, c.re)))),
              fma(-a.re, b.im, fma(-a.im, b.re, fma(-e.re, f.im, fma(-e.im, f.re, c.im)))));
}
// 1/z = conj(z) / |z|^2, the real reciprocal by d_rcp (ok cleared for |z|^2
// zero, subnormal, above 2^1021 or not finite)
CNB_HD cx<double> crcp(cx<double> z, bool& ok) {
    const double m2 = fma(z.re, z.re, d_mul(z.im, z.im));
    const double q = d_rcp(m2, ok);
    return mk(d_mul(z.re, q), d_mul(-z.im, q));  // (-a) q = -(a q), signed zeros included
}

// --- double-float
CNB_HD cx<df> cadd(cx<df> a, cx<df> b) { return mk(df_add(a.re, b.re), df_add(a.im, b.im)); }
CNB_HD cx<df> csub(cx<df> a, cx<df> b) { return mk(df_sub(a.re, b.re), df_sub(a.im, b.im)); }
CNB_HD cx<df> cneg(cx<df> a) { return mk(df_neg(a.re), df_neg(a.im)); }
CNB_HD cx<df> cmul(cx<df> a, cx<df> b) {
    return mk(df_dot2(a.re, b.re, df_neg(a.im), b.im), df_dot2(a.re, b.im, a.im, b.re));
}
CNB_HD cx<df> cfma(cx<df> c, cx<df> a, cx<df> b) {
    return mk(df_dot2_add(c.re, a.re, b.re, df_neg(a.im), b.im), df_dot2_add(c.im, a.re, b.im, a.im, b.re));
}
// c - a b - e f, one dot product per component
CNB_HD cx<df> csub2mul(cx<df> c, cx<df> a, cx<df> b, cx<df> e, cx<df> f) {
    return mk(df_dot4_add(c.re, df_neg(a.re), b.re, a.im, b.im, df_neg(e.re), f.re, e.im, f.im),
              df_dot4_add(c.im, df_neg(a.re), b.im, df_neg(a.im), b.re, df_neg(e.re), f.im, df_neg(e.im), f.re));
}
// 1/z = conj(z) / |z|^2
CNB_HD cx<df> crcp(cx<df> z, bool& ok) {
    df m2 = df_dot2(z.re, z.re, z.im, z.im);
    ok = ok && (m2.hi > 0.0f && m2.hi < 1.0e37f);
    df q = df_rcp(m2);
    return mk(df_mul(z.re, q), df_neg(df_mul(z.im, q)));
}

// ------------------------------------------------------------ real helpers
template <class R> struct RealOps;
template <> struct RealOps<double> {
    static CNB_HD double from_d(double x) { return x; }
    static CNB_HD double to_d(double x) { return x; }
};
template <> struct RealOps<df> {
    static CNB_HD df from_d(double x) { return df_from_double(x); }
    static CNB_HD double to_d(df x) { return df_to_double(x); }
};
template <class R> CNB_HD cx<R> czero() { return mk<R>(RealOps<R>::from_d(0.0), RealOps<R>::from_d(0.0)); }
template <class R> CNB_HD cx<R> cfrom(double re, double im) {
    return mk<R>(RealOps<R>::from_d(re), RealOps<R>::from_d(im));
}

// ------------------------------------------------------------ storage
// Workspace (reduced systems, their solutions) is stored in the compute type:
// double2 (re, im) for double, float4 (re.hi, re.lo, im.hi, im.lo) for df --
// 16 B per complex either way.  User-facing states are complex128 (double2).
template <class R> struct Store;
template <> struct Store<double> { typedef double2 T; };
template <> struct Store<df> { typedef float4 T; };

CNB_HD cx<double> sload(const double2* p) { double2 v = dbg_ld(p); return mk(v.x, v.y); }
CNB_HD void sstore(double2* p, cx<double> z) { dbg_st(p, make_double2(z.re, z.im)); }
CNB_HD cx<df> sload(const float4* p) {
    float4 v = dbg_ld(p);
    return mk(df_make(v.x, v.y), df_make(v.z, v.w));
}
CNB_HD void sstore(float4* p, cx<df> z) { dbg_st(p, make_float4(z.re.hi, z.re.lo, z.im.hi, z.im.lo)); }

// complex128 in memory <-> cx<R>
template <class R> CNB_HD cx<R> load128(const double2* p) {
    double2 v = dbg_ld(p);
    return mk<R>(RealOps<R>::from_d(v.x), RealOps<R>::from_d(v.y));
}
template <class R> CNB_HD void store128(double2* p, cx<R> z) {
    dbg_st(p, make_double2(RealOps<R>::to_d(z.re), RealOps<R>::to_d(z.im)));
}

}  // namespace cnb
