// Double-word ("double-float") values on the FP32 units: a value is the
// unevaluated sum h + l of two FP32 numbers with |l| <= ulp(h) / 2, a 48-bit
// significand.  On this GPU FP64 runs at about 1/74 of the FP32 FMA rate, so
// the stencil passes of the reliable updates (r = b - A x recomputed at full
// accuracy, dslash_dw.cu) run faster in double-word arithmetic than in native
// FP64.
//
// Building blocks (Dekker 1971; Knuth, TAOCP vol. 2, 4.2.2; the double-word
// algorithms and error bounds of Joldes, Muller and Popescu, "Tight and rigorous
// error bounds for basic building blocks of double-word arithmetic", ACM TOMS
// 44 (2017)):
//   two_sum(a, b)      s + e = a + b exactly (6 operations);
//   fast_two_sum(a, b) the same for |a| >= |b| (3 operations);
// and the "sloppy" double-word sum built from them (error below
// 2 u^2 (|x| + |y|), u = 2^-24).  Products and sums of products are formed in
// dslash_dw.cu as compensated dot products.
#pragma once

#include <cuda_runtime.h>

namespace tmk {

struct df {
    float h, l;
    df() = default;
    __host__ __device__ __forceinline__ constexpr df(float a, float b) : h(a), l(b) {}
    // nearest double word of a double (FP64 operations: kernel parameters and
    // the conversion kernels only)
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

}  // namespace tmk
