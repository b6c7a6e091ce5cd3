// Double-word form of the stencil passes of eq:hQpm (light) and eq:hQh (heavy
// doublet), for the true-residual recomputations of the mixed-precision solvers
// (tm_apply_Mhat_dw).
//
//   K1 (even output):  t_e = M_ee^-1 H_eo psi_o
//   K2 (odd output):   out = g5 [ M_oo psi_o - kappa^2 H_oe t_e ] (+ i rho psi_o)
//
// The heavy passes split the flavours over a thread pair (thread 2 i + f: flavour
// f of site i), as the direct FP32 / 16-bit heavy even pass does, so a thread
// holds one flavour's accumulators; the even inverse takes the partner's D v by
// lane shuffles, the odd pass reads the partner flavour of psi_o directly.
//
// Values are double words (df64.h), held as (hi, lo) FP32 pairs in the FP64
// layouts.  Written for the instruction cache rather than for unrolling: the
// fully unrolled double-word passes need ~21,000 instructions per site, overflow
// the instruction cache and stall on instruction fetch (11.8 warps per issue).
// Here the eight hops are one runtime loop over a single hop body whose
// direction-dependent spin projection and reconstruction are selected at run
// time, and every sum of products is a compensated dot product (Ogita, Rump and
// Oishi, "Accurate sum and dot product", SIAM J. Sci. Comput. 26 (2005), Dot2):
// the high parts are summed with two_sum, the product errors (two_prod with one
// FMA), the cross terms and the summation errors go to a second FP32 sum, and
// the pair is renormalised once at the end.
#include "tm_internal.h"
#include "tm_kernels.h"
#include "dslash_common.cuh"

namespace tmk {

// compensated sum: h the running FP32 sum, l the FP32 sum of its errors and of
// the low parts added
struct CSum {
    float h, l;
};
__device__ __forceinline__ void cs_add(CSum& a, float xh, float xl) {
    const float s = __fadd_rn(a.h, xh);
    const float bb = __fsub_rn(s, a.h);
    const float t = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(xh, bb));
    a.h = s;
    a.l = __fadd_rn(a.l, __fadd_rn(t, xl));
}
__device__ __forceinline__ void cs_add(CSum& a, df x) { cs_add(a, x.h, x.l); }
// a += sg x y, sg = +-1 (the low-low product, below 2^-48 |x y|, is dropped)
__device__ __forceinline__ void cs_fma(CSum& a, df x, df y, float sg = 1.f) {
    const float xh = sg * x.h, xl = sg * x.l;
    const float p = __fmul_rn(xh, y.h);
    float e = __fmaf_rn(xh, y.h, -p);
    e = __fmaf_rn(xh, y.l, e);
    e = __fmaf_rn(xl, y.h, e);
    cs_add(a, p, e);
}
__device__ __forceinline__ df cs_get(CSum a) { return df_fast_two_sum(a.h, a.l); }
__device__ __forceinline__ CSum cs_zero() { return CSum{0.f, 0.f}; }

__device__ __forceinline__ df dscale(df x, float s) { return df(s * x.h, s * x.l); }   // s = +-1
// i^k z for k = 0 (z) or 1 (i z), times sg = +-1
__device__ __forceinline__ cpx<df> cmul_unit(cpx<df> z, bool imag, float sg) {
    const df re = imag ? df(-z.im.h, -z.im.l) : z.re;
    const df im = imag ? z.re : z.im;
    return C(dscale(re, sg), dscale(im, sg));
}
__device__ __forceinline__ cpx<df> csel(bool c, cpx<df> a, cpx<df> b) {
    return C(df(c ? a.re.h : b.re.h, c ? a.re.l : b.re.l), df(c ? a.im.h : b.im.h, c ? a.im.l : b.im.l));
}

// One hop into the compensated accumulators acc[spin][colour][re / im]: direction
// mu, forward (fwd: (1 - g_mu) U_mu(x) psi(x+mu)) or backward ((1 + g_mu)
// U_mu(x-mu)^dagger psi(x-mu)), ph the boundary phase (+-1).  The chiral-basis
// projection h = (psi_up + s G psi_dn) and reconstruction (h, s G^+ h) of
// dslash_common.cuh, with s = -1 forward and +1 backward, written with run-time
// selections:
//   h0 = p0 + c0 pA, h1 = p1 + c1 pB, (pA, pB) = (p3, p2) for mu = 0, 1 and (p2, p3) for mu = 2, 3,
//   c0 = -s (i for mu = 0, 2), c1 = s (i, 1, i, 1) (-, +, +, -);
//   lower: acc2 += d2 X2, acc3 += d3 X3, (X2, X3) = (g1, g0) for mu = 0, 1 and (g0, g1) for mu = 2, 3,
//   d2 = s (i, 1, i, -1), d3 = s (i, -1, -i, -1).
__device__ __forceinline__ void hop_dw(CSum (&acc)[4][3][2], const cpx<df> (&psi)[12], const cpx<df> (&u)[9],
                                       int mu, bool fwd, float ph) {
    const float s = fwd ? -1.f : 1.f;
    const bool m01 = mu < 2;
    const bool imag = (mu == 0 || mu == 2);
    const float c0 = -s * ph;
    const float c1 = ((mu == 1 || mu == 2) ? s : -s) * ph;
    cpx<df> h0[3], h1[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const cpx<df> pa = csel(m01, psi[9 + c], psi[6 + c]);
        const cpx<df> pb = csel(m01, psi[6 + c], psi[9 + c]);
        const cpx<df> qa = cmul_unit(pa, imag, c0);
        const cpx<df> qb = cmul_unit(pb, imag, c1);
        const cpx<df> p0 = C(dscale(psi[c].re, ph), dscale(psi[c].im, ph));
        const cpx<df> p1 = C(dscale(psi[3 + c].re, ph), dscale(psi[3 + c].im, ph));
        h0[c] = C(p0.re + qa.re, p0.im + qa.im);
        h1[c] = C(p1.re + qb.re, p1.im + qb.im);
    }
    // g = U h (forward) or U^dagger h (backward)
    cpx<df> g0[3], g1[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        CSum r0 = cs_zero(), i0 = cs_zero(), r1 = cs_zero(), i1 = cs_zero();
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const cpx<df> e = csel(fwd, u[3 * a + b], cj(u[3 * b + a]));
            cs_fma(r0, e.re, h0[b].re);
            cs_fma(r0, e.im, h0[b].im, -1.f);
            cs_fma(i0, e.re, h0[b].im);
            cs_fma(i0, e.im, h0[b].re);
            cs_fma(r1, e.re, h1[b].re);
            cs_fma(r1, e.im, h1[b].im, -1.f);
            cs_fma(i1, e.re, h1[b].im);
            cs_fma(i1, e.im, h1[b].re);
        }
        g0[a] = C(cs_get(r0), cs_get(i0));
        g1[a] = C(cs_get(r1), cs_get(i1));
    }
    const float d2 = (mu == 3) ? -s : s;
    const float d3 = (mu == 0) ? s : -s;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        cs_add(acc[0][a][0], g0[a].re);
        cs_add(acc[0][a][1], g0[a].im);
        cs_add(acc[1][a][0], g1[a].re);
        cs_add(acc[1][a][1], g1[a].im);
        const cpx<df> x2 = cmul_unit(csel(m01, g1[a], g0[a]), imag, d2);
        const cpx<df> x3 = cmul_unit(csel(m01, g0[a], g1[a]), imag, d3);
        cs_add(acc[2][a][0], x2.re);
        cs_add(acc[2][a][1], x2.im);
        cs_add(acc[3][a][0], x3.re);
        cs_add(acc[3][a][1], x3.im);
    }
}

// the eight hops of flavour f (NF flavours stored) of output site i (parity po)
// in one runtime loop
template <int NF>
__device__ __forceinline__ void hops_dw(cpx<df> (&out)[4][3], const OpProb& pr, const Coord& c, long i, int po,
                                        int f) {
    const Geom& g = pr.g;
    CSum acc[4][3][2];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[s][a][0] = acc[s][a][1] = cs_zero();
#pragma unroll 1
    for (int hop = 0; hop < 8; ++hop) {
        const int mu = hop >> 1;
        const bool fwd = (hop & 1) == 0;
        const int xm = mu == 0 ? c.x : mu == 1 ? c.y : mu == 2 ? c.z : c.t;
        const int lm = mu == 0 ? g.X : mu == 1 ? g.Y : mu == 2 ? g.Z : g.T;
        const bool wrap = fwd ? (xm + 1 == lm) : (xm == 0);
        const int xn = fwd ? (wrap ? 0 : xm + 1) : (wrap ? lm - 1 : xm - 1);
        const long n = cb_index(g, mu == 0 ? xn : c.x, mu == 1 ? xn : c.y, mu == 2 ? xn : c.z, mu == 3 ? xn : c.t);
        const float ph = (mu == 3 && wrap) ? pr.bc_t : 1.f;
        cpx<df> psi[12];
        cpx<df> u[9];
        load_reals<PDF, 24>(pr.in, g.vh, n, 24 * f, reinterpret_cast<df*>(psi));
        load_link<PDF>(pr.gauge[fwd ? po : 1 - po], g.vh, mu, fwd ? i : n, u);
        hop_dw(acc, psi, u, mu, fwd, ph);
    }
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) out[s][a] = C(cs_get(acc[s][a][0]), cs_get(acc[s][a][1]));
}

// w += H v for a packed hermitian 6x6 block m (36 reals) as compensated sums
// seeded with w (the double-word form of herm6_mv_acc)
__device__ __forceinline__ void herm6_dw(cpx<df> (&w)[6], const df* m, const cpx<df> (&v)[6]) {
    cpx<df> out[6];
#pragma unroll
    for (int r = 0; r < 6; ++r) {
        CSum wr = cs_zero(), wi = cs_zero();
        cs_add(wr, w[r].re);
        cs_add(wi, w[r].im);
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            if (j == r) {
                cs_fma(wr, m[r], v[j].re);
                cs_fma(wi, m[r], v[j].im);
            } else {
                // H_rj = lower entry (r, j) for r > j, else the conjugate of (j, r)
                const int o = r > j ? herm_off(r, j) : herm_off(j, r);
                const float si = r > j ? 1.f : -1.f;
                cs_fma(wr, m[o], v[j].re);
                cs_fma(wr, m[o + 1], v[j].im, -si);
                cs_fma(wi, m[o], v[j].im);
                cs_fma(wi, m[o + 1], v[j].re, si);
            }
        }
        out[r] = C(cs_get(wr), cs_get(wi));
    }
#pragma unroll
    for (int r = 0; r < 6; ++r) w[r] = out[r];
}

__device__ __forceinline__ df shfl_pair_dw(unsigned mask, df x) {
    return df(__shfl_xor_sync(mask, x.h, 1), __shfl_xor_sync(mask, x.l, 1));
}

// 4 resident blocks per SM (128 registers): the normal operator at 32^3x64 3.94 ->
// 3.68 ms, the heavy one at 24^3x48 3.35 -> 3.01 ms (3 blocks at 136-144 registers)
template <int NF, int KIND>
__global__ void __launch_bounds__(DSLASH_BS, 4) dslash_dw_kernel(const __grid_constant__ OpBatch<1> b) {
    const OpProb& pr = b.p[0];
    if (pr.ctl != nullptr && pr.ctl->flag != CTL_RUN) return;
    const long gt = (long)blockIdx.x * DSLASH_BS + threadIdx.x;
    const long i = NF == 2 ? gt >> 1 : gt;
    const int f = NF == 2 ? (int)(gt & 1) : 0;
    const bool valid = i < pr.g.vh;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);   // both threads of a site agree
    if (!valid) return;
    const int po = (KIND == K1_EO_INV) ? 0 : 1;
    const Coord c = cb_coords(pr.g, i, po);
    cpx<df> acc[4][3];
    hops_dw<NF>(acc, pr, c, i, po, f);
    if constexpr (KIND == K1_EO_INV && NF == 1) {
        // t = B_c v per chirality block c, B_c = (A_c + i s_c mu_t)^-1 stored row
        // major (72 reals); the adjoint sign applies B_c^dagger
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            cpx<df> v[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) v[j] = acc[2 * cb + j / 3][j % 3];
#pragma unroll 1
            for (int r = 0; r < 6; ++r) {
                CSum wr = cs_zero(), wi = cs_zero();
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    // B v: entry (r, j); B^dagger v: conj of entry (j, r)
                    const int off = 72 * cb + 2 * (pr.sign > 0 ? 6 * r + j : 6 * j + r);
                    df m[2];
                    load_reals<PDF, 2>(pr.clov, pr.g.vh, i, off, m);
                    const float si = pr.sign > 0 ? 1.f : -1.f;   // conj for the adjoint
                    cs_fma(wr, m[0], v[j].re);
                    cs_fma(wr, m[1], v[j].im, -si);
                    cs_fma(wi, m[0], v[j].im);
                    cs_fma(wi, m[1], v[j].re, si);
                }
                const cpx<df> w = C(cs_get(wr), cs_get(wi));
                // out[6 cb + r] without a run-time register index: store directly
                store_reals<PDF, 2>(pr.out, pr.g.vh, i, 2 * (6 * cb + r), reinterpret_cast<const df*>(&w));
            }
        }
    } else if constexpr (KIND == K1_EO_INV) {
        // heavy inverse from A_c - 1 and D_c - 1 (dslash_heavy.cu):
        //   dv = D v, w = A dv, out = w + t i dv + epsbar_t (D v of the partner flavour),
        //   t = (f == 0 ? -1 : 1) (c == 0 ? tw : -tw)
        const df tw = df(pr.tw);
        const df eps = df(pr.eps);
        const float tf = f == 0 ? -1.f : 1.f;
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            cpx<df> v[6], dv[6], w[6], dp[6];
#pragma unroll
            for (int j = 0; j < 6; ++j) dv[j] = v[j] = acc[2 * cb + j / 3][j % 3];
            {
                df m[36];
                load_reals<PDF, 36>(pr.clov, pr.g.vh, i, 72 * cb + 36, m);
                herm6_dw(dv, m, v);
            }
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                w[j] = dv[j];
                dp[j] = C(shfl_pair_dw(mask, dv[j].re), shfl_pair_dw(mask, dv[j].im));
            }
            {
                df m[36];
                load_reals<PDF, 36>(pr.clov, pr.g.vh, i, 72 * cb, m);
                herm6_dw(w, m, dv);
            }
            const float ts = tf * (cb == 0 ? 1.f : -1.f);
#pragma unroll
            for (int j = 0; j < 6; ++j) {
                CSum orr = cs_zero(), oi = cs_zero();
                cs_add(orr, w[j].re);
                cs_add(oi, w[j].im);
                cs_fma(orr, tw, dv[j].im, -ts);   // t i dv
                cs_fma(oi, tw, dv[j].re, ts);
                cs_fma(orr, eps, dp[j].re);
                cs_fma(oi, eps, dp[j].im);
                const cpx<df> o = C(cs_get(orr), cs_get(oi));
                store_reals<PDF, 2>(pr.out, pr.g.vh, i, 24 * f + 2 * (6 * cb + j), reinterpret_cast<const df*>(&o));
            }
        }
    } else {
        // out = g5 [ (A + i tw g5 [tau3]) psi - eps tau1 psi - kappa^2 acc ] + i rho psi,
        // A hermitian (36 reals per block)
        cpx<df> psi[12], psp[12];   // this flavour and (heavy) the partner flavour
        load_reals<PDF, 24>(pr.loc, pr.g.vh, i, 24 * f, reinterpret_cast<df*>(psi));
        if constexpr (NF == 2) load_reals<PDF, 24>(pr.loc, pr.g.vh, i, 24 * (1 - f), reinterpret_cast<df*>(psp));
        const df k2 = df(pr.kappa * pr.kappa);
        const df tw = df(pr.tw);
        const df eps = df(pr.eps);
        const df rh = df(pr.rho);
        const float t3 = f == 0 ? 1.f : -1.f;
#pragma unroll
        for (int cb = 0; cb < 2; ++cb) {
            const float sc = cb == 0 ? 1.f : -1.f;   // g5 on the block
            df m[36];
            load_reals<PDF, 36>(pr.clov, pr.g.vh, i, 36 * cb, m);
            cpx<df> v[6], w[6];
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                v[r] = psi[6 * cb + r];
                // i tw sc t3 v_r - eps v'_r - kappa^2 acc_r
                CSum wr = cs_zero(), wi = cs_zero();
                cs_fma(wr, tw, v[r].im, -sc * t3);
                cs_fma(wi, tw, v[r].re, sc * t3);
                if constexpr (NF == 2) {
                    cs_fma(wr, eps, psp[6 * cb + r].re, -1.f);
                    cs_fma(wi, eps, psp[6 * cb + r].im, -1.f);
                }
                cs_fma(wr, k2, acc[2 * cb + r / 3][r % 3].re, -1.f);
                cs_fma(wi, k2, acc[2 * cb + r / 3][r % 3].im, -1.f);
                w[r] = C(cs_get(wr), cs_get(wi));
            }
            herm6_dw(w, m, v);
#pragma unroll
            for (int r = 0; r < 6; ++r) {
                // g5: the lower block changes sign; then + i rho v_r
                CSum orr = cs_zero(), oi = cs_zero();
                cs_add(orr, dscale(w[r].re, sc));
                cs_add(oi, dscale(w[r].im, sc));
                cs_fma(orr, rh, v[r].im, -1.f);
                cs_fma(oi, rh, v[r].re);
                const cpx<df> o = C(cs_get(orr), cs_get(oi));
                store_reals<PDF, 2>(pr.out, pr.g.vh, i, 24 * f + 2 * (6 * cb + r), reinterpret_cast<const df*>(&o));
            }
        }
    }
}

template <int P, int NF, int KIND, int NP>
cudaError_t launch_dslash(const OpBatch<NP>& b, int nblocks, cudaStream_t st);

// the double-word instantiations of launch_dslash (no batch tables, no fused
// norm: the reliable updates use neither); two-flavour passes take 2 vh threads
#define TM_DW_INST(NF, KIND)                                                                       \
    template <>                                                                                    \
    cudaError_t launch_dslash<PDF, NF, KIND, 1>(const OpBatch<1>& b, int nblocks, cudaStream_t st) { \
        if (b.n != 1 || b.p[0].partial != nullptr) return cudaErrorInvalidValue;                    \
        dslash_dw_kernel<NF, KIND><<<nblocks, DSLASH_BS, 0, st>>>(b);                              \
        return cudaGetLastError();                                                                 \
    }
TM_DW_INST(1, K1_EO_INV)
TM_DW_INST(1, K2_OE_LOCAL)
TM_DW_INST(2, K1_EO_INV)
TM_DW_INST(2, K2_OE_LOCAL)

}  // namespace tmk
