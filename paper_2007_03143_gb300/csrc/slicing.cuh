// Ozaki-style slicing of double-float values into bf16-exact integer slices, and the
// power-of-two helpers it uses; float32 arithmetic only (device code).
//
// A value v = (h + l) 2^-e, |v| <= 1, is cut into NSL = 5 slices q_s 2^-(6+7s) with integer
// q_s, so that every slice is exact in bf16 and every product of two slices is exact in the
// fp32 accumulators of the tensor cores (34 bits in total).
#pragma once

#include <cstdint>

namespace gbxc {
namespace slc {

constexpr int NSL = 5;

// 2^k as a float for k in [-126, 127] (built from the exponent field)
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// x 2^k for |k| <= 252 as two exact power-of-two products; the intermediate lies between x
// and the result in magnitude, so nothing is lost that the result could hold
__device__ __forceinline__ float scale2(float x, int k) {
    const int k1 = k >> 1;
    return __fmul_rn(__fmul_rn(x, pow2f(k1)), pow2f(k - k1));
}

// v = (h + l) 2^-e with |v| <= 1 -> five slices q_s 2^-(6+7s), q_s integers, float32 only:
// each q_s is the rounding of the running remainder to the slice grid (the power-of-two
// products are exact) and the subtraction is exact (Sterbenz).  Slices 0-2 come from h
// alone and lie in [-64, 64] (the bound the exact accumulator levels 0-2 rely on).  The
// low word joins the remainder after them, when |remainder| <= 2^-21, so that rounding is
// below 2^-45; slice 3 may then reach +-72, which only feeds the rounded levels 3-4.
__device__ __forceinline__ void slice5(float h, float l, int e, float out[NSL]) {
    float rh = scale2(h, -e);
    const float rl = scale2(l, -e);
#pragma unroll
    for (int s = 0; s < NSL; ++s) {
        if (s == 3) rh = __fadd_rn(rh, rl);
        const float up = (float)(1ull << (6 + 7 * s));
        const float qs = __fmul_rn(rintf(__fmul_rn(rh, up)), 1.0f / up);
        out[s] = qs;
        rh = __fsub_rn(rh, qs);
    }
}

// exponent e with |x| < 2^e for x > 0 (0 for x == 0), from the float's exponent bits
__device__ __forceinline__ int exp_of(float x) {
    if (!(x > 0.f)) return 0;
    int e;
    frexpf(x * 1.0000002f, &e);
    return e;
}

}  // namespace slc
}  // namespace gbxc
