// Even-odd Schur operator kernels of eq:hQpm (light doublet) and the odd pass of
// eq:hQh (heavy doublet; its even pass is in dslash_heavy.cu).
//
//   Q_hat psi_o = g5 [ (M_oo) psi_o - M_oe M_ee^-1 M_eo psi_o ],  M_eo = -kappa H_eo
//
// is applied in two passes, one thread per output site:
//   K1 (even output):  t_e = (M_ee)^-1 H_eo psi_o            hop + site-local 6x6 inverse blocks
//   K2 (odd output):   out = g5 [ M_oo psi_o - kappa^2 H_oe t_e ]   hop + clover/twist + g5
// K2 can fuse ||out||^2 into a deterministic two-level FP64 reduction whose last
// block finalises a solver scalar (CG alpha), so a CG iteration needs no separate
// reduction launch.  Every kernel takes a table of problems (one or a batch of
// lattices of different volumes); a block belongs to exactly one problem.
#include "tm_internal.h"
#include "tm_kernels.h"
#include "dslash_common.cuh"

namespace tmk {

// All 8 hops for NF flavours into acc[NF][4][3]; output site (c, i) of parity po.
template <int P, int NF, int MU>
__device__ __forceinline__ void hop_mu(cpx<typename PT<P>::R> (&acc)[NF][4][3], const OpProb& pr,
                                       const Coord& c, long i, int po) {
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
    constexpr bool SC = (P == PF16 || P == PB16);   // 16-bit: the scale joins the phase
    cpx<R> u[9];
    cpx<R> psi[NF * 12];
    float sc;
    // forward
    load_spinor_unscaled<P, NF * 12>(pr.in, g.vh, nf, psi, sc);
    load_link<P>(pr.gauge[po], g.vh, MU, i, u);
#pragma unroll
    for (int f = 0; f < NF; ++f) hop_dir<R, MU, -1, false, SC>(acc[f], psi + 12 * f, u, SC ? ph_f * (R)sc : ph_f);
    // backward
    load_spinor_unscaled<P, NF * 12>(pr.in, g.vh, nb, psi, sc);
    load_link<P>(pr.gauge[1 - po], g.vh, MU, nb, u);
#pragma unroll
    for (int f = 0; f < NF; ++f) hop_dir<R, MU, +1, true, SC>(acc[f], psi + 12 * f, u, SC ? ph_b * (R)sc : ph_b);
}

// Resident blocks the compiler must fit per SM (128-thread blocks; the register
// cap follows).  Sweeps at 32^3x64 (light) and 24^3x48 (heavy) put the optimum at:
//   light 16-bit even pass: 5 blocks (96 registers; the inverse blocks stream two
//     rows at a time for this).  6 blocks: 112.8 -> 133.4 us FP16, 116.6 -> 174.2 us BF16;
//   light odd pass: 7 blocks FP16 (72 registers, 16 B spilled) and 6 BF16 (80
//     registers): 5 / 6 / 7 blocks take 112.2 / 104.9 / 103.0 us FP16 and
//     126.9 / 113.2 / 119.0 us BF16 (4 blocks: 108.3 / 113.1 us);
//   light FP32 odd pass: 4 blocks (128 registers, 16 B spilled): 156.5 -> 150.0 us
//     (3 blocks 152.0 us); the FP32 even pass keeps the default (3 blocks at 156
//     registers; 4 blocks: 187 -> 227 us);
//   two-flavour odd pass: 4 blocks in 16-bit storage (128 registers; 3 / 5
//     blocks: 63.8 -> 67.7 / 75.0 us FP16) and 3 in FP32 (168 registers, 8 B
//     spilled: 94.8 -> 78.1 us at 24^3x48; 2 / 4 blocks: 94.5 / 84.4 us).
// The FP64 passes keep the default.  (The two-flavour even pass splits the
// flavours over a thread pair: dslash_heavy.cu.)
template <int P, int NF, int KIND>
constexpr int dslash_min_blocks() {
    if (P == PF16 || P == PB16) {
        if (NF == 2) return 4;
        if (KIND == K1_EO_INV) return 5;
        return P == PF16 ? 7 : 6;
    }
    if (P == P32 && KIND == K2_OE_LOCAL) return NF == 2 ? 3 : 4;
    return 1;
}

template <int P, int NF, int KIND, int NP, int BS>
__global__ void __launch_bounds__(BS, (dslash_min_blocks<P, NF, KIND>())) dslash_kernel(const __grid_constant__ OpBatch<NP> b) {
    static_assert(NF == 1 || KIND == K2_OE_LOCAL, "the two-flavour even pass lives in dslash_heavy.cu");
    using R = typename PT<P>::R;
    __shared__ double sh[BS / 32];
    const int k = find_problem<NP>(b, blockIdx.x);
    const OpProb& pr = b.p[k];
    if (pr.ctl != nullptr && pr.ctl->flag != CTL_RUN) return;
    const int lb = blockIdx.x - b.blk_start[k];
    const long i = (long)lb * BS + threadIdx.x;
    const bool valid = i < pr.g.vh;
    const int po = (KIND == K1_EO_INV) ? 0 : 1;   // output parity
    double nrm = 0.0;
    if (valid) {
        const Coord c = cb_coords(pr.g, i, po);
        cpx<R> acc[NF][4][3];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int a = 0; a < 3; ++a) acc[f][s][a] = C((R)0, (R)0);
        hop_mu<P, NF, 0>(acc, pr, c, i, po);
        hop_mu<P, NF, 1>(acc, pr, c, i, po);
        hop_mu<P, NF, 2>(acc, pr, c, i, po);
        hop_mu<P, NF, 3>(acc, pr, c, i, po);

        cpx<R> out[NF * 12];
        if constexpr (KIND == K1_EO_INV) {
            if constexpr (NF == 1) {
                // t_e = (A_c + i sign s_c mu_t)^-1 (H psi) per chirality block c
#pragma unroll
                for (int cb = 0; cb < 2; ++cb) {
                    cpx<R> v[6], w[6];
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        v[j] = acc[0][2 * cb + j / 3][j % 3];
                        w[j] = C((R)0, (R)0);
                    }
                    // stream the block two rows (24 reals) at a time to bound registers
#pragma unroll
                    for (int rr = 0; rr < 3; ++rr) {
                        R m[24];
                        load_reals<P, 24>(pr.clov, pr.g.vh, i, 72 * cb + 24 * rr, m);
#pragma unroll
                        for (int r2 = 0; r2 < 2; ++r2) {
                            const int r = 2 * rr + r2;
#pragma unroll
                            for (int j = 0; j < 6; ++j) {
                                const cpx<R> e = C(m[2 * (6 * r2 + j)], m[2 * (6 * r2 + j) + 1]);
                                if (pr.sign > 0) cfma(w[r], e, v[j]);       // B v
                                else cfma_cj(w[j], e, v[r]);                // B^dagger v
                            }
                        }
                    }
#pragma unroll
                    for (int j = 0; j < 6; ++j) out[6 * cb + j] = w[j];
                }
            }
        } else {
            // out = g5 [ (A + i tw g5 [tau3]) psi - eps tau1 psi - kappa^2 acc ]
            cpx<R> psi[NF * 12];
            load_spinor<P, NF * 12>(pr.loc, pr.g.vh, i, psi);
            R m[72];
            load_reals<P, 72>(pr.clov, pr.g.vh, i, 0, m);
            const R k2 = (R)(pr.kappa * pr.kappa);
            const R tw = (R)pr.tw;
            const R eps = (R)pr.eps;
#pragma unroll
            for (int f = 0; f < NF; ++f) {
                const R t3 = (f == 0) ? (R)1 : (R)-1;
#pragma unroll
                for (int cb = 0; cb < 2; ++cb) {
                    const R sc = (cb == 0) ? (R)1 : (R)-1;
                    cpx<R> v[6], w[6];
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        v[j] = psi[12 * f + 6 * cb + j];
                        w[j] = (tw * sc * t3) * mul_i(v[j]);
                        if constexpr (NF == 2) w[j] = w[j] - eps * psi[12 * (1 - f) + 6 * cb + j];
                        w[j] = w[j] - k2 * acc[f][2 * cb + j / 3][j % 3];
                    }
                    herm6_mv_acc<R>(w, m + 36 * cb, v);
                    const R rh = (R)pr.rho;   // W_hat = Q_hat + i rho (eq:hWpm), added after g5
#pragma unroll
                    for (int j = 0; j < 6; ++j)
                        out[12 * f + 6 * cb + j] = ((cb == 0) ? w[j] : -w[j]) + rh * mul_i(v[j]);
                }
            }
            if (pr.partial != nullptr) {
                R s = (R)0;
#pragma unroll
                for (int q = 0; q < NF * 12; ++q) s += norm2(out[q]);
                nrm = (double)s;
            }
        }
        store_spinor<P, NF * 12>(pr.out, pr.g.vh, i, out);
    }
    if constexpr (KIND == K2_OE_LOCAL) {
      if (pr.partial != nullptr) {
        const double bs = block_sum<BS>(nrm, sh);
        reduce_finalize<BS>(pr.partial, pr.counter, pr.nblk, lb, bs, b.fin, pr.ctl, pr.ms,
                            nullptr, sh);
      }
    }
}

template <int P, int NF, int KIND, int NP>
cudaError_t launch_dslash(const OpBatch<NP>& b, int nblocks, cudaStream_t st) {
    dslash_kernel<P, NF, KIND, NP, DSLASH_BS><<<nblocks, DSLASH_BS, 0, st>>>(b);
    return cudaGetLastError();
}

#define TM_INST(P, NF, KIND, NP) \
    template cudaError_t launch_dslash<P, NF, KIND, NP>(const OpBatch<NP>&, int, cudaStream_t);
#define TM_INST_P(P)                                                                      \
    TM_INST(P, 1, K1_EO_INV, 1) TM_INST(P, 1, K2_OE_LOCAL, 1) TM_INST(P, 2, K2_OE_LOCAL, 1) \
    TM_INST(P, 1, K1_EO_INV, MAXP) TM_INST(P, 1, K2_OE_LOCAL, MAXP)
TM_INST_P(P64)
// (the double-word passes: dslash_dw.cu)
TM_INST_P(P32)
TM_INST_P(PB16)
TM_INST_P(PF16)

}  // namespace tmk
