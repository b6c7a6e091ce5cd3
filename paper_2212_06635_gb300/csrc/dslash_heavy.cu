// Even pass of the two-flavour (heavy doublet, eq:hQh) Schur operator with the
// flavours split across a thread pair:
//
//   K1 (even output):  t_e = M_h,ee^-1 H_eo psi_o
//
// Thread 2i + f computes flavour f of output site i: its own hop (one transport
// per direction instead of two), its own half of the site epilogue, and its 12
// output components; the two threads of a site share the link and clover loads
// through L1 and exchange the flavour-coupling terms with one lane shuffle.  A
// thread fits in 96 registers at 5 blocks per SM.
// (The odd pass keeps one thread per site: dslash.cu.)
//
// Even-site inverse.  With D_c = (A_c^2 + mubar_t^2 - epsbar_t^2)^-1 (Hermitian,
// commuting with A_c) and sigma = +-1 the sign of the operator (Q_hat_h or its
// adjoint), the inverse of the chirality-c block is
//   [[ (A - i s sigma mubar_t) D,  epsbar_t D ], [ epsbar_t D,  (A + i s sigma mubar_t) D ]]
// (s = +1 for spins 0,1 and -1 for spins 2,3), so the pass stores only A_c - 1
// and D_c - 1 (144 reals per site, the minimum; both are close to the identity,
// and storing the deviation keeps the 16-bit rounding relative to it) and applies
//   w_u = A (D v_u) - i s sigma mubar_t (D v_u) + epsbar_t (D v_d),
//   w_d = A (D v_d) + i s sigma mubar_t (D v_d) + epsbar_t (D v_u):
// each thread multiplies its own flavour by D and then A, and takes the
// partner's D v across the pair.
#include "tm_internal.h"
#include "tm_kernels.h"
#include "dslash_common.cuh"

namespace tmk {

// flavour f half (12 complex, reals 24 f .. 24 f + 23) of a two-flavour spinor,
// 16-bit values left unscaled with the site scale in sc (1 for FP32 / FP64)
template <int P>
__device__ __forceinline__ void load_flavour_unscaled(const void* base, long vh, long i, int f,
                                                      cpx<typename PT<P>::R>* s, float& sc) {
    using R = typename PT<P>::R;
    load_reals<P, 24>(base, vh, i, 24 * f, reinterpret_cast<R*>(s));
    sc = 1.f;
    if constexpr (P == PB16 || P == PF16) {
        const float* nrm = reinterpret_cast<const float*>(reinterpret_cast<const char*>(base) + (size_t)vh * 24 * 2 * 2);
        sc = __ldg(nrm + i);
    }
}

// store flavour f of output site i; 16-bit fields share one scale per site, the
// maximum over both flavours (taken across the pair with `mask`)
template <int P>
__device__ __forceinline__ void store_flavour(void* base, long vh, long i, int f, const cpx<typename PT<P>::R>* s,
                                              unsigned mask) {
    using R = typename PT<P>::R;
    if constexpr (P == PB16 || P == PF16) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(s[k].re), fabsf(s[k].im)));
        m = fmaxf(m, __shfl_xor_sync(mask, m, 1));
        const float inv = m > 0.f ? 1.f / m : 0.f;
        R t[24];
#pragma unroll
        for (int k = 0; k < 12; ++k) { t[2 * k] = s[k].re * inv; t[2 * k + 1] = s[k].im * inv; }
        store_reals<P, 24>(base, vh, i, 24 * f, t);
        if (f == 0) {
            float* nrm = reinterpret_cast<float*>(reinterpret_cast<char*>(base) + (size_t)vh * 24 * 2 * 2);
            nrm[i] = m;
        }
    } else {
        store_reals<P, 24>(base, vh, i, 24 * f, reinterpret_cast<const R*>(s));
    }
}

// hops of direction MU for flavour f into acc
template <int P, int MU>
__device__ __forceinline__ void hop_mu_flavour(cpx<typename PT<P>::R> (&acc)[4][3], const OpProb& pr, const Coord& c,
                                               long i, int po, int f) {
    using R = typename PT<P>::R;
    const Geom& g = pr.g;
    int xf = c.x, yf = c.y, zf = c.z, tf = c.t;
    int xb = c.x, yb = c.y, zb = c.z, tb = c.t;
    R ph_f = (R)1, ph_b = (R)1;
    if (MU == 0) { xf = (c.x + 1 == g.X) ? 0 : c.x + 1; xb = (c.x == 0) ? g.X - 1 : c.x - 1; }
    if (MU == 1) { yf = (c.y + 1 == g.Y) ? 0 : c.y + 1; yb = (c.y == 0) ? g.Y - 1 : c.y - 1; }
    if (MU == 2) { zf = (c.z + 1 == g.Z) ? 0 : c.z + 1; zb = (c.z == 0) ? g.Z - 1 : c.z - 1; }
    if (MU == 3) {
        if (c.t + 1 == g.T) { tf = 0; ph_f = (R)pr.bc_t; } else tf = c.t + 1;
        if (c.t == 0) { tb = g.T - 1; ph_b = (R)pr.bc_t; } else tb = c.t - 1;
    }
    const long nf = cb_index(g, xf, yf, zf, tf);
    const long nb = cb_index(g, xb, yb, zb, tb);
    constexpr bool SC = (P == PF16 || P == PB16);
    cpx<R> u[9];
    cpx<R> psi[12];
    float sc;
    load_flavour_unscaled<P>(pr.in, g.vh, nf, f, psi, sc);
    load_link<P>(pr.gauge[po], g.vh, MU, i, u);
    hop_dir<R, MU, -1, false, SC>(acc, psi, u, SC ? ph_f * (R)sc : ph_f);
    load_flavour_unscaled<P>(pr.in, g.vh, nb, f, psi, sc);
    load_link<P>(pr.gauge[1 - po], g.vh, MU, nb, u);
    hop_dir<R, MU, +1, true, SC>(acc, psi, u, SC ? ph_b * (R)sc : ph_b);
}

// Resident blocks per SM the register allocation must allow (128 threads = 64
// sites).  At 24^3x48: 16-bit 4 / 5 / 6 blocks take 73.9 / 73.5 / 73.9 us (FP16)
// and 72.1 / 69.8 / 72.7 us (BF16); FP32 3 / 4 / 5 blocks 96.4 / 96.4 / 89.7 us.
template <int P, int KIND>
constexpr int heavy_min_blocks() {
    return (P == PF16 || P == PB16) ? 5 : (P == P32 ? 5 : 1);
}

template <int P, int KIND, int NP, int BS>
__global__ void __launch_bounds__(BS, (heavy_min_blocks<P, KIND>())) dslash_heavy_kernel(const __grid_constant__ OpBatch<NP> b) {
    static_assert(KIND == K1_EO_INV, "even pass only");
    using R = typename PT<P>::R;
    const int k = find_problem<NP>(b, blockIdx.x);
    const OpProb& pr = b.p[k];
    if (pr.ctl != nullptr && pr.ctl->flag != CTL_RUN) return;
    const int lb = blockIdx.x - b.blk_start[k];
    const long gt = (long)lb * BS + threadIdx.x;
    const long i = gt >> 1;
    const int f = (int)(gt & 1);
    const bool valid = i < pr.g.vh;
    const unsigned mask = __ballot_sync(0xffffffffu, valid);   // both threads of a site agree
    const int po = 0;
    if (valid) {
        const Coord c = cb_coords(pr.g, i, po);
        cpx<R> acc[4][3];
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) acc[s][a] = C((R)0, (R)0);
        hop_mu_flavour<P, 0>(acc, pr, c, i, po, f);
        hop_mu_flavour<P, 1>(acc, pr, c, i, po, f);
        hop_mu_flavour<P, 2>(acc, pr, c, i, po, f);
        hop_mu_flavour<P, 3>(acc, pr, c, i, po, f);
        cpx<R> out[12];
        const R tw = (R)pr.tw;       // sign * mubar_t
        const R eps = (R)pr.eps;     // epsbar_t
        const R tf = f == 0 ? (R)-1 : (R)1;
        {
#pragma unroll
            for (int cb = 0; cb < 2; ++cb) {
                cpx<R> v[6], dv[6], w[6];
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    v[j] = acc[2 * cb + j / 3][j % 3];
                    dv[j] = v[j];
                }
                {   // D_c - 1: 40 reals from 72 cb + 32 (aligned for every storage width), at offset 4
                    R m[40];
                    load_reals<P, 40>(pr.clov, pr.g.vh, i, 72 * cb + 32, m);
                    herm6_mv_acc<R>(dv, m + 4, v);
                }
#pragma unroll
                for (int j = 0; j < 6; ++j) w[j] = dv[j];
                cpx<R> dp[6];   // the partner flavour's D v
#pragma unroll
                for (int j = 0; j < 6; ++j) {
                    dp[j].re = __shfl_xor_sync(mask, dv[j].re, 1);
                    dp[j].im = __shfl_xor_sync(mask, dv[j].im, 1);
                }
                {   // A_c - 1: 40 reals from 72 cb, at offset 0
                    R m[40];
                    load_reals<P, 40>(pr.clov, pr.g.vh, i, 72 * cb, m);
                    herm6_mv_acc<R>(w, m, dv);
                }
                const R t = tf * (cb == 0 ? tw : -tw);
#pragma unroll
                for (int j = 0; j < 6; ++j) out[6 * cb + j] = w[j] + t * mul_i(dv[j]) + eps * dp[j];
            }
        }
        store_flavour<P>(pr.out, pr.g.vh, i, f, out, mask);
    }
}

template <int P, int NF, int KIND, int NP>
cudaError_t launch_dslash(const OpBatch<NP>& b, int nblocks, cudaStream_t st);

// the two-flavour even-pass instantiations of launch_dslash: nblocks covers 2 vh threads
#define TM_HEAVY_INST(P, KIND)                                                                        \
    template <>                                                                                       \
    cudaError_t launch_dslash<P, 2, KIND, 1>(const OpBatch<1>& b, int nblocks, cudaStream_t st) {     \
        dslash_heavy_kernel<P, KIND, 1, DSLASH_BS><<<nblocks, DSLASH_BS, 0, st>>>(b);                \
        return cudaGetLastError();                                                                    \
    }
TM_HEAVY_INST(P64, K1_EO_INV)
TM_HEAVY_INST(P32, K1_EO_INV)
TM_HEAVY_INST(PB16, K1_EO_INV)
TM_HEAVY_INST(PF16, K1_EO_INV)

}  // namespace tmk
