// Unsigned 32-bit division by a loop-invariant divisor as one multiply-high, one
// subtract, one add and two shifts (Granlund and Montgomery, "Division by
// invariant integers using multiplication", PLDI 1994, Sec. 4: the round-up
// multiplier m' = floor(2^32 (2^l - d) / d) + 1 with l = ceil(log2 d)).  The
// result is exact for every dividend n < 2^32 and every divisor 1 <= d < 2^32.
//
// The stencil and site kernels turn a checkerboard index into coordinates with
// three such divisions (by X/2, Y and Z) per thread; as plain 64-bit divisions
// those were a few hundred instructions per site.
//
// Plain C++ when compiled by a host compiler, so the arithmetic can be checked
// exhaustively on the CPU.
#pragma once

#include <stdint.h>

#if defined(__CUDACC__)
#define TM_FD_HD __host__ __device__ __forceinline__
#else
#define TM_FD_HD inline
#endif

namespace tmk {

struct FastDiv {
    uint32_t d;    // divisor
    uint32_t m;    // multiplier m'
    int s1, s2;    // shifts min(l, 1) and max(l - 1, 0)
};

inline FastDiv make_fastdiv(uint32_t d) {
    int l = 0;
    while ((1ull << l) < (uint64_t)d) ++l;   // l = ceil(log2 d); 0 for d = 1
    FastDiv f;
    f.d = d;
    f.m = (uint32_t)(((((1ull << l) - d) << 32) / d) + 1);
    f.s1 = l < 1 ? l : 1;
    f.s2 = l > 1 ? l - 1 : 0;
    return f;
}

TM_FD_HD uint32_t fd_mulhi(uint32_t a, uint32_t b) {
#if defined(__CUDA_ARCH__)
    return __umulhi(a, b);
#else
    return (uint32_t)(((uint64_t)a * b) >> 32);
#endif
}

// floor(n / f.d)
TM_FD_HD uint32_t fdiv(uint32_t n, const FastDiv& f) {
    const uint32_t t = fd_mulhi(f.m, n);
    return (t + ((n - t) >> f.s1)) >> f.s2;
}

}  // namespace tmk
