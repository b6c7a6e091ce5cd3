// Device helpers shared by the direct and the staged stencil kernels: spin
// projection / colour transport of one hop in the chiral basis, and the 6x6
// chirality-block products of the clover term and its inverses.
#pragma once

#include "tm_internal.h"

namespace tmk {

// ---------------------------------------------------------------------------
// Spin projection / reconstruction of the chiral basis for one hop.
//   S = -1: forward  (1 - g_mu) U_mu(x) psi(x+mu)
//   S = +1: backward (1 + g_mu) U_mu(x-mu)^dagger psi(x-mu)
// With g_mu = [[0, G],[G^+, 0]] (G_x = -i s1, G_y = -i s2, G_z = -i s3, G_t = -1):
//   (1 + S g) psi = (h, S G^+ h),  h = psi_up + S G psi_down,
// so only the two-spin half spinor h is transported by the link.
// ---------------------------------------------------------------------------
// `factor` multiplies the half spinor: the boundary phase of a time hop, times
// the neighbour's scale for 16-bit spinors (SCALED), which are passed unscaled;
// scaling the 6 projected components costs half of scaling the 12 loaded ones.
template <typename R, int MU, int S, bool DAG, bool SCALED = false>
__device__ __forceinline__ void hop_dir(cpx<R> (&acc)[4][3], const cpx<R>* psi,
                                        const cpx<R> (&u)[9], R factor) {
    const R s = (R)S;
    cpx<R> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cpx<R> p0 = psi[c], p1 = psi[3 + c], p2 = psi[6 + c], p3 = psi[9 + c];
        if (MU == 0) {        // h0 = p0 - s i p3, h1 = p1 - s i p2
            h0[c] = p0 - s * mul_i(p3);
            h1[c] = p1 - s * mul_i(p2);
        } else if (MU == 1) { // h0 = p0 - s p3, h1 = p1 + s p2
            h0[c] = p0 - s * p3;
            h1[c] = p1 + s * p2;
        } else if (MU == 2) { // h0 = p0 - s i p2, h1 = p1 + s i p3
            h0[c] = p0 - s * mul_i(p2);
            h1[c] = p1 + s * mul_i(p3);
        } else {              // h0 = p0 - s p2, h1 = p1 - s p3
            h0[c] = p0 - s * p2;
            h1[c] = p1 - s * p3;
        }
        if (MU == 3 || SCALED) { h0[c] = factor * h0[c]; h1[c] = factor * h1[c]; }
    }
    cpx<R> g0[3], g1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        g0[a] = C((R)0, (R)0);
        g1[a] = C((R)0, (R)0);
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            if (DAG) {
                cfma_cj(g0[a], u[3 * b + a], h0[b]);
                cfma_cj(g1[a], u[3 * b + a], h1[b]);
            } else {
                cfma(g0[a], u[3 * a + b], h0[b]);
                cfma(g1[a], u[3 * a + b], h1[b]);
            }
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[0][a] = acc[0][a] + g0[a];
        acc[1][a] = acc[1][a] + g1[a];
        if (MU == 0) {        // lower += s i (g1, g0)
            acc[2][a] = acc[2][a] + s * mul_i(g1[a]);
            acc[3][a] = acc[3][a] + s * mul_i(g0[a]);
        } else if (MU == 1) { // lower += s (g1, -g0)
            acc[2][a] = acc[2][a] + s * g1[a];
            acc[3][a] = acc[3][a] - s * g0[a];
        } else if (MU == 2) { // lower += s i (g0, -g1)
            acc[2][a] = acc[2][a] + s * mul_i(g0[a]);
            acc[3][a] = acc[3][a] - s * mul_i(g1[a]);
        } else {              // lower += -s (g0, g1)
            acc[2][a] = acc[2][a] - s * g0[a];
            acc[3][a] = acc[3][a] - s * g1[a];
        }
    }
}

// w = B v (CONJ: B^dagger v) for a full complex 6x6 block stored row major.
template <typename R, bool CONJ>
__device__ __forceinline__ void full6_mv(cpx<R> (&w)[6], const R* m, const cpx<R> (&v)[6]) {
#pragma unroll
    for (int r = 0; r < 6; ++r) w[r] = C((R)0, (R)0);
#pragma unroll
    for (int r = 0; r < 6; ++r)
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            const cpx<R> e = C(m[2 * (6 * r + j)], m[2 * (6 * r + j) + 1]);
            if (CONJ) cfma_cj(w[j], e, v[r]);   // (B^+)_{j r} = conj(B_{r j})
            else cfma(w[r], e, v[j]);
        }
}

// w += H v for a packed hermitian 6x6 block (36 reals).
template <typename R>
__device__ __forceinline__ void herm6_mv_acc(cpx<R> (&w)[6], const R* m, const cpx<R> (&v)[6]) {
#pragma unroll
    for (int r = 0; r < 6; ++r) w[r] = w[r] + m[r] * v[r];
#pragma unroll
    for (int r = 1; r < 6; ++r)
#pragma unroll
        for (int j = 0; j < r; ++j) {
            const cpx<R> e = C(m[herm_off(r, j)], m[herm_off(r, j) + 1]);
            cfma(w[r], e, v[j]);      // lower:  H_rj v_j
            cfma_cj(w[j], e, v[r]);   // upper:  H_jr = conj(H_rj)
        }
}

}  // namespace tmk
