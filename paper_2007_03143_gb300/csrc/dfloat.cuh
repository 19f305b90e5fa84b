// Double-float ("df") arithmetic: a value is the unevaluated sum hi + lo of two float32s,
// about 48 significant bits, computed on the float32 pipe.  Error-free transforms after
// Dekker (1971, "A floating-point technique for extending the available precision") and
// Knuth's two-sum; every step uses the explicitly rounded intrinsics so no compiler
// contraction can change it.
//
// exp_neg(t, tab) = exp(-t) for t >= 0, table-driven after P. T. P. Tang, "Table-driven
// implementation of the exponential function in IEEE floating-point arithmetic" (ACM TOMS
// 15, 1989): t = k ln2/64 + r with |r| <= ln2/128 (ln2/64 in three float parts), exp(-r)
// by its Taylor series to degree 5, times 2^(-(k mod 64)/64) from a 64-entry double-float
// table (make_exp2_table) and 2^-floor(k/64).  Relative error ~1e-14; results below 2^-126
// lose precision gradually and are zero from t = 87 on.
#pragma once

#include <cmath>
#include <cstdint>

#include <cuda_runtime.h>

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

// The table of exp_neg: tab[j] = 2^(-j/64) as (hi, lo), from the host's float64 exp2.
inline void make_exp2_table(float2 *tab) {
    for (int j = 0; j < 64; ++j) {
        const double v = std::exp2(-(double)j / 64.0);
        const float hi = (float)v;
        tab[j] = make_float2(hi, (float)(v - (double)hi));
    }
}

// exp(-t), t >= 0 given as a df; `tab` from make_exp2_table (any memory space).
__device__ __forceinline__ df exp_neg(df t, const float2 *tab) {
    if (!(t.h < 87.0f)) return {0.f, 0.f};
    // ln2/64 = C1 + C2 + C3; C1 has 11 significant bits so k*C1 is exact for k < 2^13
    const float C1 = 0.01082611083984375f;
    const float C2 = 4.3138566070e-06f;
    const float C3 = -2.0164562565e-13f;
    const float k = rintf(__fmul_rn(t.h, 92.33248138f));   // 64 / ln2
    const float a = __fsub_rn(t.h, __fmul_rn(k, C1));       // exact (Sterbenz / k = 0)
    const float p2 = __fmul_rn(k, C2);
    const float e2 = __fmaf_rn(k, C2, -p2);
    df r = two_sum(a, -p2);
    r = add_f(r, __fsub_rn(t.l, e2));
    r = add_f(r, -__fmul_rn(k, C3));
    // exp(-r) = 1 + r (-1 + r (1/2 - r q)), q = 1/6 - r/24 + r^2/120 in float32 (|r| <= 0.0055:
    // its rounding enters below 2^-49); 1/2 - r q by two-sum, the two outer steps in df
    float q = __fmaf_rn(r.h, 8.3333337680e-03f, -4.1666667908e-02f);
    q = __fmaf_rn(q, r.h, 1.6666667163e-01f);
    df w = two_sum(0.5f, -__fmul_rn(r.h, q));
    w = add_f(mul(w, r), -1.0f);
    df s = add_f(mul(w, r), 1.0f);
    const int ki = (int)k;
    const float2 T = tab[ki & 63];
    s = mul(s, {T.x, T.y});
    const float sc = __int_as_float((127 - (ki >> 6)) << 23);   // 2^-floor(k/64), k < 8040
    return {__fmul_rn(s.h, sc), __fmul_rn(s.l, sc)};
}

}  // namespace dfl
}  // namespace gbxc
