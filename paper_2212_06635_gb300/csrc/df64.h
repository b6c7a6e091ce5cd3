// Double-word ("double-float") arithmetic on the FP32 units: a value is the
// unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h) / 2, a 48-bit
// significand.  On this GPU FP64 runs at about 1/74 of the FP32 FMA rate, so
// the stencil passes of the reliable updates (r = b - A x recomputed at full
// accuracy) run faster in double-word arithmetic than in native FP64.
//
// Building blocks (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2; the double-word
// algorithms and error bounds of Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44 (2017)):
//   two_sum(a, b)      s + e = a + b exactly (6 operations);
//   fast_two_sum(a, b) the same for |a| >= |b| (3 operations);
//   two_prod(a, b)     p + e = a b exactly with one FMA.
// Addition is the "sloppy" double-word sum (error below 2 u^2 (|x| + |y|),
// u = 2^-24), multiplication the FMA-based product (error below 5 u^2 |x y|);
// x y + z is the product followed by the sum.  The absolute error of every
// operation is thus bounded by ~2^-46 times the magnitudes of its operands, as
// in a backward-stable FP64 evaluation with a 48-bit significand.
#pragma once

#include <cuda_runtime.h>

namespace tmk {

using ::fma;   // the FP32 / FP64 overloads stay visible next to the double-word one

struct df {
    float h, l;
    df() = default;
    __host__ __device__ __forceinline__ constexpr df(float a, float b) : h(a), l(b) {}
    __host__ __device__ __forceinline__ explicit df(double x)
        : h((float)x), l((float)(x - (double)(float)x)) {}
    __host__ __device__ __forceinline__ explicit df(int x) : h((float)x), l(0.f) {}
    __host__ __device__ __forceinline__ explicit operator double() const { return (double)h + (double)l; }
};

__device__ __forceinline__ df df_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return df(s, e);
}
__device__ __forceinline__ df df_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return df(s, __fsub_rn(b, __fsub_rn(s, a)));
}
__device__ __forceinline__ df operator+(df x, df y) {
    const df s = df_two_sum(x.h, y.h);
    const float v = __fadd_rn(x.l, y.l);
    return df_fast_two_sum(s.h, __fadd_rn(s.l, v));
}
__device__ __forceinline__ df operator-(df x) { return df(-x.h, -x.l); }
__device__ __forceinline__ df operator-(df x, df y) { return x + (-y); }
__device__ __forceinline__ df operator*(df x, df y) {
    const float p = __fmul_rn(x.h, y.h);
    float e = __fmaf_rn(x.h, y.h, -p);
    e = __fmaf_rn(x.h, y.l, e);
    e = __fmaf_rn(x.l, y.h, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df& operator+=(df& x, df y) { x = x + y; return x; }
// x y + z
__device__ __forceinline__ df fma(df x, df y, df z) { return x * y + z; }

}  // namespace tmk
