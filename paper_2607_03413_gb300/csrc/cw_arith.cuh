// cw_arith.cuh -- arithmetic types for the cell-wise operator kernels.
//
// GB300 executes native FP64 FMA at about 1/73 of the FP32 rate (measured 1.0 TFLOP/s FP64 vs
// 73 TFLOP/s FP32), so the FP64 operator path computes in double-float arithmetic: a value is an
// unevaluated sum hi + lo of two floats (Dekker 1971; error-free TwoSum of Knuth and the
// FMA-based TwoProduct, as collected by Muller et al., "Handbook of Floating-Point Arithmetic").
// Storage stays IEEE FP64; a double is split into (hi, lo) with integer bit operations (the
// FP64->FP32 conversion instructions run on the slow FP64 pipe) keeping 24 + 23 significant bits,
// i.e. a relative truncation error below 2^-46.
#pragma once
#include <cuda_bf16.h>
#include <cstdint>

namespace cw {

struct df64 {
    float hi, lo;
};

// storage form of a double-float value (the FP64 metric tensor is kept pre-split, so the operator
// reads each metric entry with one 8-byte load and no conversion work)
struct __align__(8) df64s {
    float hi, lo;
};

// ---------------------------------------------------------------- conversions ----

// Split a double into hi + lo floats using integer operations only. |x| < 2^-126 maps to 0; the
// low part is exact while it is a normal float (|x| above about 2^-102) and rounded to the float
// subnormal grid below that. Infinities, NaNs and finite values
// beyond the float range map to +-inf / NaN in hi (lo = 0), so non-finite data stays non-finite.
__device__ __forceinline__ df64 split_f64(double x)
{
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(x));
    const unsigned h32 = static_cast<unsigned>(b >> 32), l32 = static_cast<unsigned>(b);
    const unsigned sign = h32 & 0x80000000u;
    const int e = static_cast<int>((h32 >> 20) & 0x7FFu);
    const int fe = e - 896;  // float biased exponent
    const unsigned mhi = ((h32 & 0xFFFFFu) << 3) | (l32 >> 29);
    df64 r;
    if (fe <= 0) {
        r.hi = 0.0f;
        r.lo = 0.0f;
        return r;
    }
    if (fe >= 255) {
        const bool nan = (e == 2047) && (((h32 & 0xFFFFFu) | l32) != 0u);
        r.hi = __uint_as_float(sign | 0x7F800000u | (nan ? 0x400000u : 0u));
        r.lo = 0.0f;
        return r;
    }
    r.hi = __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | mhi);
    // remainder: the low 29 mantissa bits, worth rem * 2^(e-1075); keep its top 23 bits
    const unsigned r23 = (l32 & 0x1FFFFFFFu) >> 6;
    const float f = __fsub_rn(__uint_as_float(0x4B000000u | r23), 8388608.0f);  // exact
    // scale by 2^(e-1069): one power-of-two factor (biased exponent se = e - 942) while that is a
    // normal float, else 2^(e-1069+64) and then 2^-64 (f * 2^(e-1005) is exact and normal for every
    // e >= 897; the second product is exact while the low part is normal)
    const int se = e - 942;
    const bool tiny = se < 1;
    const float scale = __uint_as_float(static_cast<unsigned>(tiny ? se + 64 : se) << 23);
    float lo = __fmul_rn(f, scale);
    if (tiny) lo = __fmul_rn(lo, 5.42101086242752217e-20f);  // 2^-64
    r.lo = __uint_as_float(__float_as_uint(lo) | sign);
    return r;
}

// Exact widening float -> double with integer operations (zero and subnormals map to +-0,
// infinities and NaNs stay infinities and NaNs).
__device__ __forceinline__ double widen_f32(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned sign = u & 0x80000000u;
    const unsigned e = (u >> 23) & 0xFFu;
    const unsigned m = u & 0x7FFFFFu;
    unsigned hi = (e == 0u) ? sign : (sign | ((e + 896u) << 20) | (m >> 3));
    unsigned lo = (e == 0u) ? 0u : (m << 29);
    if (e == 255u) {
        hi = sign | 0x7FF00000u | (m ? 0x80000u : 0u);
        lo = 0u;
    }
    return __longlong_as_double(static_cast<long long>((static_cast<unsigned long long>(hi) << 32) | lo));
}

__device__ __forceinline__ double df_to_double(df64 a) { return __dadd_rn(widen_f32(a.hi), widen_f32(a.lo)); }

// ---------------------------------------------------------- double-float ops ----

// s + e = a + b exactly (TwoSum, no ordering requirement)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// renormalise so that |lo| <= ulp(hi)/2 (Fast2Sum; valid because |lo| is small against |hi|)
__device__ __forceinline__ df64 df_norm(df64 a)
{
    df64 r;
    r.hi = __fadd_rn(a.hi, a.lo);
    r.lo = __fsub_rn(a.lo, __fsub_rn(r.hi, a.hi));
    return r;
}

// product of two double-float numbers (low-order term lo*lo dropped), not normalised
__device__ __forceinline__ df64 df_mul(df64 a, df64 b)
{
    df64 r;
    r.hi = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -r.hi);  // exact error of the product
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    r.lo = e;
    return r;
}

// acc += a * b, lazily normalised (acc.lo collects all low-order terms)
__device__ __forceinline__ void df_mad(df64 &acc, df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    two_sum(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(t, e));
}

// a / b in double-float: quotient estimate q1 from the leading floats, the remainder a - q1 b
// in double-float, one correction q2 from it, q1 + q2 renormalised (long division, as in
// Dekker 1971); relative error about 2^-44.
__device__ __forceinline__ df64 df_div(df64 a, df64 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    // r = a - q1 * b with the product exact in two floats
    const float p = __fmul_rn(q1, b.hi);
    const float pe = __fmaf_rn(q1, b.hi, -p);
    float s, t;
    two_sum(a.hi, -p, s, t);
    const float rl = __fadd_rn(__fadd_rn(t, -pe), __fadd_rn(a.lo, -__fmul_rn(q1, b.lo)));
    const float r = __fadd_rn(s, rl);
    const float q2 = __fdiv_rn(r, b.hi);
    df64 q;
    q.hi = __fadd_rn(q1, q2);
    q.lo = __fsub_rn(q2, __fsub_rn(q.hi, q1));
    return q;
}

__device__ __forceinline__ df64 df_add(df64 a, df64 b)
{
    float s, t;
    two_sum(a.hi, b.hi, s, t);
    df64 r;
    r.hi = s;
    r.lo = __fadd_rn(t, __fadd_rn(a.lo, b.lo));
    return r;
}

// ------------------------------------------------- paired double-float operations ----
// Two independent double-float values in one register-pair form: hi = (a.hi, b.hi), lo = (a.lo,
// b.lo). The operations below are the scalar ones above applied to both lanes with the paired FP32
// instructions of sm_100+ (FADD2 / FMUL2 / FFMA2: two FP32 operations per thread instruction, same
// rounding per lane as the scalar forms), so each lane's result is bit-identical to the scalar
// operation and the FP32 pipe gets half the instructions to issue.
struct __align__(16) df64p {
    float2 hi, lo;
};

__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2 &s, float2 &e)
{
    s = __fadd2_rn(a, b);
    const float2 bb = __fadd2_rn(s, neg2(a));
    e = __fadd2_rn(__fadd2_rn(a, neg2(__fadd2_rn(s, neg2(bb)))), __fadd2_rn(b, neg2(bb)));
}

// lane-wise df_mul
__device__ __forceinline__ df64p dfp_mul(df64p a, df64p b)
{
    df64p r;
    r.hi = __fmul2_rn(a.hi, b.hi);
    float2 e = __ffma2_rn(a.hi, b.hi, neg2(r.hi));
    e = __ffma2_rn(a.hi, b.lo, e);
    e = __ffma2_rn(a.lo, b.hi, e);
    r.lo = e;
    return r;
}

// lane-wise df_mad
__device__ __forceinline__ void dfp_mad(df64p &acc, df64p a, df64p b)
{
    const float2 p = __fmul2_rn(a.hi, b.hi);
    float2 e = __ffma2_rn(a.hi, b.hi, neg2(p));
    e = __ffma2_rn(a.hi, b.lo, e);
    e = __ffma2_rn(a.lo, b.hi, e);
    float2 s, t;
    two_sum2(acc.hi, p, s, t);
    acc.hi = s;
    acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(t, e));
}

__device__ __forceinline__ df64p dfp_pack(df64 a, df64 b) { return df64p{make_float2(a.hi, b.hi), make_float2(a.lo, b.lo)}; }
__device__ __forceinline__ df64 dfp_x(df64p a) { return df64{a.hi.x, a.lo.x}; }
__device__ __forceinline__ df64 dfp_y(df64p a) { return df64{a.hi.y, a.lo.y}; }

// ------------------------------------------------------------ arithmetic traits ----
// Each trait defines the register type T, the constant type C used for the 1D tables, and
// mul / mad / add / norm plus conversions from and to each storage type.

struct ArDF {  // double-float arithmetic
    using T = df64;
    using C = df64;
    static __device__ __forceinline__ T zero() { return T{0.0f, 0.0f}; }
    static __device__ __forceinline__ T mul(T a, C b) { return df_mul(a, b); }
    static __device__ __forceinline__ void mad(T &acc, T a, C b) { df_mad(acc, a, b); }
    static __device__ __forceinline__ T add(T a, T b) { return df_add(a, b); }
    static __device__ __forceinline__ T sub(T a, T b) { return df_add(a, T{-b.hi, -b.lo}); }
    static __device__ __forceinline__ T neg(T a) { return T{-a.hi, -a.lo}; }
    static __device__ __forceinline__ T norm(T a) { return df_norm(a); }
    static __device__ __forceinline__ T div(T a, T b) { return df_div(a, b); }
    static __device__ __forceinline__ T from(double v) { return split_f64(v); }
    static __device__ __forceinline__ T from(float v) { return T{v, 0.0f}; }
    static __device__ __forceinline__ T from(df64s v) { return T{v.hi, v.lo}; }
    static __device__ __forceinline__ void to(double &d, T a) { d = df_to_double(a); }
    static __device__ __forceinline__ double to_f64(T a) { return df_to_double(a); }
    static __device__ __forceinline__ df64 to_df(T a) { return a; }
};

struct ArF64 {  // native FP64
    using T = double;
    using C = double;
    static __device__ __forceinline__ T zero() { return 0.0; }
    static __device__ __forceinline__ T mul(T a, C b) { return a * b; }
    static __device__ __forceinline__ void mad(T &acc, T a, C b) { acc = fma(a, b, acc); }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T norm(T a) { return a; }
    static __device__ __forceinline__ T div(T a, T b) { return a / b; }
    static __device__ __forceinline__ T from(double v) { return v; }
    static __device__ __forceinline__ T from(df64s v) { return widen_f32(v.hi) + widen_f32(v.lo); }
    static __device__ __forceinline__ void to(double &d, T a) { d = a; }
    static __device__ __forceinline__ double to_f64(T a) { return a; }
};

struct ArF32 {  // FP32
    using T = float;
    using C = float;
    static __device__ __forceinline__ T zero() { return 0.0f; }
    static __device__ __forceinline__ T mul(T a, C b) { return a * b; }
    static __device__ __forceinline__ void mad(T &acc, T a, C b) { acc = fmaf(a, b, acc); }
    static __device__ __forceinline__ T add(T a, T b) { return a + b; }
    static __device__ __forceinline__ T sub(T a, T b) { return a - b; }
    static __device__ __forceinline__ T neg(T a) { return -a; }
    static __device__ __forceinline__ T norm(T a) { return a; }
    static __device__ __forceinline__ T div(T a, T b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ T from(float v) { return v; }
    static __device__ __forceinline__ T from(__nv_bfloat16 v) { return __bfloat162float(v); }
    static __device__ __forceinline__ void to(float &d, T a) { d = a; }
    static __device__ __forceinline__ void to(__nv_bfloat16 &d, T a) { d = __float2bfloat16_rn(a); }
    static __device__ __forceinline__ double to_f64(T a) { return static_cast<double>(a); }
    static __device__ __forceinline__ df64 to_df(T a) { return df64{a, 0.0f}; }
};

}  // namespace cw
