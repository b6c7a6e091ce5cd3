// Fermion-force outer products of the hopping term on every link.
//
// Sec. 4.3 ("Efficiency") reports that the force of the rational-approximation
// monomials stayed on the CPU, where colour outer products of several
// two-flavour spinors, one pair per shift of the multishift solve, dominated
// its cost.  This kernel computes that step for n field pairs (X_k, Y_k) and
// weights c_k in one pass over the lattice:
//
//   W_mu(x) = ph_mu(x) sum_k c_k sum_flavour [ X_k(x+mu) (x) ((1 - g_mu) Y_k(x))^*
//                                            + ((1 + g_mu) Y_k(x+mu)) (x) X_k(x)^* ]
//   force_mu(x) += T_A[ U_mu(x) W_mu(x) ]    (traceless anti-hermitian part)
//
// so that force_mu(x) is the derivative of S = sum_k c_k Re <Y_k, H[U] X_k>
// along su(3) directions of U_mu(x) (H the hopping term).  Optionally g5 Y_k
// takes the place of Y_k: the Schur operators' hopping force is one such pair
// per shift, X = (M_ee^-1 H_eo b, b) and Y = g5 (M_ee(-s)^-1 H_eo a, a).
//
// Each spin sum reduces to two spin components: in the chiral basis
// g_mu = [[0, G], [G^+, 0]] and (1 + s g_mu) B = (h, s G^+ h) with
// h = B_up + s G B_down, so that
//   sum_spin A (x) ((1 + s g_mu) B)^* = sum_{l=0,1} (A_up + s G A_down)_l (x) h_l^*
// and both terms are sums of two colour outer products of half spinors:
// the forward term pairs the s = -1 halves of X(x+mu) and Y(x), the backward
// term the s = +1 halves of Y(x+mu) and X(x).
//
// Layout and mapping.  Fields are native (structure of arrays over the Vh
// sites of one parity; 32- or 16-bit storage), math is FP32, the force is the
// canonical FP64 link layout and is read, added to and written once.  A block of
// 32 x 4 x 2 threads covers the 64 lexicographic sites [64 b, 64 b + 64): the
// 32 half-site indices 32 b .. 32 b + 31 of both parities (z), one direction mu
// per warp (y), so every warp's load of a field vector is one contiguous
// 512-byte span (16 B per site) and its neighbour loads are the same span
// shifted.  The four warps of one parity reuse X(x), Y(x) through L1.
//
// Bytes per launch (algorithmic): each field read once (2 n V spinors), the FP32
// links once (4 V x 12 reals), the force read and written once (2 x 4 V x 18 x 8).
#include "force.h"

namespace tmk {

// half spinor h = (psi_up + S G_mu psi_down), times f:
//   G_x = -i s1, G_y = -i s2, G_z = -i s3, G_t = -1 (chiral basis)
template <int MU, int S>
__device__ __forceinline__ void force_half(cpx<float> (&h)[2][3], const cpx<float>* p, float f) {
    const float s = (float)S;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cpx<float> p0 = p[c], p1 = p[3 + c], p2 = p[6 + c], p3 = p[9 + c];
        cpx<float> a, b;
        if (MU == 0) {          // G psi_dn = -i (p3, p2)
            a = p0 - s * mul_i(p3);
            b = p1 - s * mul_i(p2);
        } else if (MU == 1) {   // G psi_dn = (-p3, p2)
            a = p0 - s * p3;
            b = p1 + s * p2;
        } else if (MU == 2) {   // G psi_dn = (-i p2, i p3)
            a = p0 - s * mul_i(p2);
            b = p1 + s * mul_i(p3);
        } else {                // G psi_dn = -(p2, p3)
            a = p0 - s * p2;
            b = p1 - s * p3;
        }
        h[0][c] = f * a;
        h[1][c] = f * b;
    }
}

// 12 complex components of flavour f at site i, unscaled; sc = the site's
// scale for 16-bit storage (1 for FP32)
template <int P, int NF>
__device__ __forceinline__ void force_load(const void* base, long vh, long i, int f, cpx<float>* p, float& sc) {
    load_reals<P, 24>(base, vh, i, 24 * f, reinterpret_cast<float*>(p));
    sc = 1.f;
    if constexpr (P == PB16 || P == PF16) {
        const float* nrm = reinterpret_cast<const float*>(reinterpret_cast<const char*>(base) +
                                                          (size_t)vh * NF * 12 * 2 * 2);
        sc = __ldg(nrm + i);
    }
}

// w[3a + b] += sum_l u[l][a] conj(v[l][b])
__device__ __forceinline__ void force_outer2(cpx<float> (&w)[9], const cpx<float> (&u)[2][3],
                                             const cpx<float> (&v)[2][3]) {
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cfma_cj(w[3 * a + b], v[0][b], u[0][a]);
            cfma_cj(w[3 * a + b], v[1][b], u[1][a]);
        }
}

// G5: the Y fields enter as g5 Y.  P_s(g5 B) = B_up - s G B_down = P_-s(B), so
// g5 only flips the projection sign of the Y spinors.
template <int P, int NF, int MU, bool G5>
__device__ __forceinline__ void force_link(const ForceArgs& a, long i, int par, const Coord& c) {
    constexpr int SY1 = G5 ? +1 : -1;   // sign of Y(x) in the forward term
    constexpr int SY2 = G5 ? -1 : +1;   // sign of Y(x+mu) in the backward term
    const Geom& g = a.g;
    int xf = c.x, yf = c.y, zf = c.z, tf = c.t;
    float ph = 1.f;
    if (MU == 0) xf = (c.x + 1 == g.X) ? 0 : c.x + 1;
    if (MU == 1) yf = (c.y + 1 == g.Y) ? 0 : c.y + 1;
    if (MU == 2) zf = (c.z + 1 == g.Z) ? 0 : c.z + 1;
    if (MU == 3) {
        if (c.t + 1 == g.T) { tf = 0; ph = a.bc_t; } else tf = c.t + 1;
    }
    const long j = cb_index(g, xf, yf, zf, tf);
    const long vh = g.vh;
    cpx<float> w[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) w[e] = C(0.f, 0.f);

    for (int k = 0; k < a.n; ++k) {
        const void* xs = a.x[k][par];
        const void* ys = a.y[k][par];
        const void* xn = a.x[k][1 - par];
        const void* yn = a.y[k][1 - par];
        const float ck = a.c[k];
#pragma unroll
        for (int f = 0; f < NF; ++f) {
            cpx<float> p[12], q[12];
            cpx<float> hu[2][3], hv[2][3];
            float s1, s2;
            // forward hop at x: X(x+mu) (x) ((1 - g_mu) Y(x))^*
            force_load<P, NF>(xn, vh, j, f, p, s1);
            force_load<P, NF>(ys, vh, i, f, q, s2);
            force_half<MU, -1>(hu, p, 1.f);
            force_half<MU, SY1>(hv, q, ck * s1 * s2);
            force_outer2(w, hu, hv);
            // backward hop at x+mu (through U_mu(x)^dagger): ((1 + g_mu) Y(x+mu)) (x) X(x)^*
            force_load<P, NF>(yn, vh, j, f, p, s1);
            force_load<P, NF>(xs, vh, i, f, q, s2);
            force_half<MU, SY2>(hu, p, 1.f);
            force_half<MU, +1>(hv, q, ck * s1 * s2);
            force_outer2(w, hu, hv);
        }
    }

    // Z = U W, force += T_A[Z] = (Z - Z^+)/2 - i Im(tr Z)/3
    cpx<float> u[9];
    load_link<P32>(a.gauge[par], vh, MU, i, u);
    cpx<float> z[9];
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            cpx<float> acc = C(0.f, 0.f);
#pragma unroll
            for (int m = 0; m < 3; ++m) cfma(acc, u[3 * r + m], w[3 * m + s]);
            z[3 * r + s] = ph * acc;
        }
    const float itr = (z[0].im + z[4].im + z[8].im) * (1.f / 3.f);
    const long lex = 2 * i + (c.x & 1);
    double2* out = reinterpret_cast<double2*>(a.force) + (lex * 4 + MU) * 9;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int s = 0; s < 3; ++s) {
            const cpx<float> zrs = z[3 * r + s], zsr = z[3 * s + r];
            float re = 0.5f * (zrs.re - zsr.re);
            float im = 0.5f * (zrs.im + zsr.im);
            if (r == s) im -= itr;
            double2 o = out[3 * r + s];
            o.x += (double)re;
            o.y += (double)im;
            out[3 * r + s] = o;
        }
}

// 4 resident blocks per SM (64 registers, a few spilled): 1612 -> 1593 us (FP32
// fields) and 1347 -> 1269 us (FP16) at 24^3x48, 12 two-flavour pairs
template <int P, int NF, bool G5>
__global__ void __launch_bounds__(256, 4) force_outer_kernel(const __grid_constant__ ForceArgs a) {
    const long i = (long)blockIdx.x * 32 + threadIdx.x;
    if (i >= a.g.vh) return;
    const int mu = threadIdx.y;
    const int par = threadIdx.z;
    const Coord c = cb_coords(a.g, i, par);
    switch (mu) {   // warp-uniform
        case 0: force_link<P, NF, 0, G5>(a, i, par, c); break;
        case 1: force_link<P, NF, 1, G5>(a, i, par, c); break;
        case 2: force_link<P, NF, 2, G5>(a, i, par, c); break;
        default: force_link<P, NF, 3, G5>(a, i, par, c); break;
    }
}

template <int P, int NF>
static cudaError_t launch_t(const ForceArgs& a, cudaStream_t st) {
    const long nblk = (a.g.vh + 31) / 32;
    if (a.g5y)
        force_outer_kernel<P, NF, true><<<(unsigned)nblk, dim3(32, 4, 2), 0, st>>>(a);
    else
        force_outer_kernel<P, NF, false><<<(unsigned)nblk, dim3(32, 4, 2), 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_force_outer(int prec, int nf, const ForceArgs& a, cudaStream_t st) {
    if (a.n <= 0 || a.g.vh <= 0) return cudaSuccess;
    switch (prec) {
        case P32: return nf == 1 ? launch_t<P32, 1>(a, st) : launch_t<P32, 2>(a, st);
        case PB16: return nf == 1 ? launch_t<PB16, 1>(a, st) : launch_t<PB16, 2>(a, st);
        case PF16: return nf == 1 ? launch_t<PF16, 1>(a, st) : launch_t<PF16, 2>(a, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tmk
