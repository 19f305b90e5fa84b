// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two float32s,
// about 48 significant bits, computed on the float32 pipe.  Error-free transforms after
// Dekker (1971, "A floating-point technique for extending the available precision") and
// Knuth's two-sum; every step uses the explicitly rounded intrinsics so no compiler
// contraction can change it.
//
// df_exp_neg(t) = exp(-t) for t >= 0: Cody-Waite reduction t = k ln2 + r (|r| <= ln2/2,
// ln2 in three float parts), Taylor series of exp(-r/8) to degree 7 (terms from y^4 on
// summed in float32: |y| <= 0.0434 puts their rounding below 2^-47; coefficients 1/n! as df
// below that), three squarings, scaling by 2^-k.  Relative error ~1e-13; results below
// 2^-126 lose precision gradually and are zero from t = 87 on.
#pragma once

#include <cstdint>

namespace gbxc {
namespace dfl {

struct df {
    float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ df quick_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ df mul(df a, df b) {
    float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ df mul_f(df a, float b) {
    float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ df add(df a, df b) {
    df s = two_sum(a.h, b.h);
    float e = __fadd_rn(s.l, __fadd_rn(a.l, b.l));
    return quick_two_sum(s.h, e);
}

__device__ __forceinline__ df sub(df a, df b) { return add(a, {-b.h, -b.l}); }

__device__ __forceinline__ df add_f(df a, float b) {
    df s = two_sum(a.h, b);
    return quick_two_sum(s.h, __fadd_rn(s.l, a.l));
}

__device__ __forceinline__ df from_double(double d) {
    float h = (float)d;
    return {h, (float)(d - (double)h)};
}

__device__ __forceinline__ double to_double(df a) { return (double)a.h + (double)a.l; }

__device__ __forceinline__ df ldexp_df(df a, int k) { return {ldexpf(a.h, k), ldexpf(a.l, k)}; }

// exp(-t), t >= 0 given as a df.
__device__ __forceinline__ df exp_neg(df t) {
    if (!(t.h < 87.0f)) return {0.f, 0.f};
    // ln 2 = C1 + C2 + C3; C1 has 15 significant bits so k*C1 is exact for k < 2^9
    const float C1 = 0.693145751953125f;
    const float C2 = 1.428606765e-06f;  // ln2 - C1, rounded
    const float C3 = 5.497923148e-14f;  // ln2 - C1 - C2, rounded
    float k = rintf(__fmul_rn(t.h, 1.442695022f));
    // r = t - k ln2 in df
    float a = __fsub_rn(t.h, __fmul_rn(k, C1));   // exact (Sterbenz / small k)
    float p2 = __fmul_rn(k, C2);
    float e2 = __fmaf_rn(k, C2, -p2);
    df r = two_sum(a, -p2);
    r = add_f(r, __fsub_rn(t.l, e2));
    r = add_f(r, -__fmul_rn(k, C3));
    // y = -r / 8, |y| <= 0.0434
    df y = {ldexpf(-r.h, -3), ldexpf(-r.l, -3)};
    // Taylor: 1 + y + y^2/2 + y^3/6 + y^4 (1/24 + y/120 + y^2/720 + y^3/5040) (Horner)
    const df I2 = {0.5f, 0.f};
    const df I3 = {1.666666716e-01f, -4.967053879e-09f};
    float q = 1.984127011e-04f;                    // 1/7!
    q = __fmaf_rn(q, y.h, 1.388888923e-03f);       // 1/6!
    q = __fmaf_rn(q, y.h, 8.333333768e-03f);       // 1/5!
    q = __fmaf_rn(q, y.h, 4.166666791e-02f);       // 1/4!
    df s = add(mul_f(y, q), I3);
    s = add(mul(s, y), I2);
    s = add_f(mul(s, y), 1.0f);
    s = add_f(mul(s, y), 1.0f);
    s = mul(s, s);
    s = mul(s, s);
    s = mul(s, s);
    // 2^-k with 0 <= k <= 126 (t < 87), from the exponent field
    const float sc = __int_as_float((127 - (int)k) << 23);
    return {__fmul_rn(s.h, sc), __fmul_rn(s.l, sc)};
}

}  // namespace dfl
}  // namespace gbxc
