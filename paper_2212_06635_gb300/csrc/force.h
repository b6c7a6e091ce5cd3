// Fermion-force outer products of the hopping term on every link (force.cu).
#pragma once

#include "tm_internal.h"

namespace tmk {

constexpr int FORCE_MAXN = 32;   // field pairs per launch (TM_FORCE_MAXN)

struct ForceArgs {
    Geom g;
    float bc_t;                  // phase of the time links crossing t = T-1 -> 0
    int n;                       // field pairs
    const void* gauge[2];        // FP32 native links of parity 0 / 1
    const void* x[FORCE_MAXN][2];   // native fields X_k of parity 0 / 1
    const void* y[FORCE_MAXN][2];   // native fields Y_k of parity 0 / 1
    float c[FORCE_MAXN];         // weights c_k
    int g5y;                     // 1: the Y fields enter as g5 Y_k
    double* force;               // canonical FP64 [lex][mu][3][3] complex, accumulated
};

// force[x][mu] += T_A[U_mu(x) W_mu(x)] on all 4V links; prec is the storage
// precision of the fields (P32, PB16 or PF16), nf 1 or 2
cudaError_t launch_force_outer(int prec, int nf, const ForceArgs& a, cudaStream_t st);

}  // namespace tmk
