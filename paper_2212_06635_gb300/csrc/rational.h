// Rational approximation of A^-1/2 (Zolotarev) and the FP64 field combinations
// of its partial-fraction application and correction series (rational.cu).
#pragma once

#include "tm_internal.h"

namespace tmk {

// r(x) = a0 + sum_l a[l] / (x + sigma[l]) ~ x^-1/2 on [lo, hi] (n poles), and the
// maximum relative error delta of sqrt(x) r(x) over [lo, hi].  Host code.
bool zolotarev_inv_sqrt(int n, double lo, double hi, double* a0, double* a, double* sigma, double* delta);

constexpr int LC_MAX = MAX_SHIFTS + 1;

// y = a0 b + sum_k a[k] x[k] over len double2 entries (y may alias b or an x[k])
struct LinComb {
    int n;
    long len;
    double a0;
    const double2* b;
    const double2* x[LC_MAX];
    double a[LC_MAX];
    double2* y;
};
cudaError_t launch_lincomb64(const LinComb& p, cudaStream_t st);

}  // namespace tmk
