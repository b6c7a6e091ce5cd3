// Shared-memory staged variant of the two stencil passes of eq:hQpm / eq:hQh.
//
// The direct kernel (dslash.cu) loads neighbour spinors and links into registers
// just before it uses them, so at the occupancy its ~110-130 registers allow the
// warps wait on DRAM (long-scoreboard stalls) and 16-bit passes reach only 40-80 %
// of HBM bandwidth.  Here every thread first issues asynchronous global->shared
// copies (cp.async) of everything it will need: the site-local epilogue data
// (clover or inverse blocks, and in the odd pass the local spinor), then the
// forward/backward neighbour spinors and links of direction 0 and 1.  It then
// consumes direction mu from one buffer while the copies of direction mu+1 and
// mu+2 are in flight, refilling the freed buffer.  Bytes in flight per SM no
// longer depend on registers.  Each thread only ever reads the shared memory
// it filled itself, so the pipeline needs no block barrier (cp.async.wait_group
// makes a thread's own copies visible to it).
//
// Shared memory per thread (16-bit, light, 12-real links): odd pass 500 B, even pass 592 B.
#include "tm_internal.h"
#include "tm_kernels.h"
#include "dslash_common.cuh"

#include <type_traits>

namespace tmk {

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void cp_async16(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async8(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_async4(void* s, const void* g) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(smem_addr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// staging geometry of storage precision P, NC complex per spinor, pass KIND
template <int P, int NC, int KIND, int NF>
struct Stg {
    static constexpr int ESZ = PT<P>::ESZ;
    static constexpr int SP16 = NC * 2 * ESZ / 16;                     // 16-B vectors per spinor
    static constexpr bool NORM = (P == PB16 || P == PF16);
    static constexpr int LB = (P == P64) ? 16 : (P == P32 ? 8 : 4);    // bytes per link element
    static constexpr int CLVR = KIND == K1_EO_INV ? (NF == 1 ? CLOV_EVEN_LIGHT_REALS : CLOV_EVEN_HEAVY_REALS)
                                                  : CLOV_ODD_REALS;
    static constexpr int CLV16 = CLVR * ESZ / 16;
    static constexpr int LOC = (KIND == K2_OE_LOCAL) ? 1 : 0;
    static constexpr int U16 = 4 * SP16 + CLV16 + LOC * SP16;           // 16-B units per thread
    static constexpr int NN = NORM ? (4 + LOC) : 0;                     // FP32 scales per thread
    static constexpr int NL = LinkStore<P>::N;                          // stored complex per link
    static constexpr int BYTES = U16 * 16 + 4 * NL * LB + NN * 4;       // shared bytes per thread
};

template <int P, int NC>
__device__ __forceinline__ void sp_from_smem(const uint4* s16, int unit0, const float* sN, int nidx, int BS,
                                             int t, cpx<typename PT<P>::R>* s) {
    using R = typename PT<P>::R;
    R* r = reinterpret_cast<R*>(s);
    constexpr int W = PT<P>::W;
#pragma unroll
    for (int u = 0; u < NC * 2 / W; ++u) {
        const uint4 q = s16[(unit0 + u) * BS + t];
        if constexpr (P == P64) {
            r[2 * u] = __longlong_as_double(((long long)q.y << 32) | q.x);
            r[2 * u + 1] = __longlong_as_double(((long long)q.w << 32) | q.z);
        } else if constexpr (P == P32) {
            r[4 * u] = __uint_as_float(q.x); r[4 * u + 1] = __uint_as_float(q.y);
            r[4 * u + 2] = __uint_as_float(q.z); r[4 * u + 3] = __uint_as_float(q.w);
        } else {
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = h2f2<P>(w[k]);
                r[8 * u + 2 * k] = f.x;
                r[8 * u + 2 * k + 1] = f.y;
            }
        }
    }
    // 16-bit spinors stay unscaled here: hop_dir applies the scale (sN) to the
    // projected half spinor
}

template <int P, int NR>
__device__ __forceinline__ void reals_from_smem(const uint4* s16, int unit0, int BS, int t,
                                                typename PT<P>::R* r) {
    constexpr int W = PT<P>::W;
#pragma unroll
    for (int u = 0; u < NR / W; ++u) {
        const uint4 q = s16[(unit0 + u) * BS + t];
        if constexpr (P == P64) {
            r[2 * u] = __longlong_as_double(((long long)q.y << 32) | q.x);
            r[2 * u + 1] = __longlong_as_double(((long long)q.w << 32) | q.z);
        } else if constexpr (P == P32) {
            r[4 * u] = __uint_as_float(q.x); r[4 * u + 1] = __uint_as_float(q.y);
            r[4 * u + 2] = __uint_as_float(q.z); r[4 * u + 3] = __uint_as_float(q.w);
        } else {
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = h2f2<P>(w[k]);
                r[8 * u + 2 * k] = f.x;
                r[8 * u + 2 * k + 1] = f.y;
            }
        }
    }
}

template <int P>
__device__ __forceinline__ void link_from_smem(const unsigned char* sL, int unit0, int BS, int t,
                                               cpx<typename PT<P>::R>* u) {
    constexpr int N = LinkStore<P>::N;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const int e = (unit0 + k) * BS + t;
        if constexpr (P == P64) {
            const double2 q = reinterpret_cast<const double2*>(sL)[e];
            u[k] = C(q.x, q.y);
        } else if constexpr (P == P32) {
            const float2 q = reinterpret_cast<const float2*>(sL)[e];
            u[k] = C(q.x, q.y);
        } else {
            const uint32_t q = reinterpret_cast<const uint32_t*>(sL)[e];
            const float2 f = h2f2<P>(q);
            u[k] = C(f.x, f.y);
        }
    }
    if constexpr (N == 6) su3_third_row(u);
}

template <int P, int NF, int KIND, int NP, int BS>
__global__ void __launch_bounds__(BS) dslash_staged_kernel(const __grid_constant__ OpBatch<NP> b) {
    using R = typename PT<P>::R;
    constexpr int NC = 12 * NF;
    using G = Stg<P, NC, KIND, NF>;
    extern __shared__ __align__(16) unsigned char smem[];
    uint4* s16 = reinterpret_cast<uint4*>(smem);
    unsigned char* sL = smem + (size_t)G::U16 * BS * 16;
    float* sN = reinterpret_cast<float*>(sL + (size_t)4 * G::NL * BS * G::LB);
    __shared__ double shred[BS / 32];

    const int k = find_problem<NP>(b, blockIdx.x);
    const OpProb& pr = b.p[k];
    if (pr.ctl != nullptr && pr.ctl->flag != CTL_RUN) return;
    const int lb = blockIdx.x - b.blk_start[k];
    const int t = threadIdx.x;
    const long i = (long)lb * BS + t;
    const bool valid = i < pr.g.vh;
    constexpr int po = (KIND == K1_EO_INV) ? 0 : 1;
    const Geom& g = pr.g;
    double nrm = 0.0;

    if (valid) {
        const Coord c = cb_coords(g, i, po);
        auto nbr = [&](int mu, long& nf, long& nb) {
            int xf = c.x, yf = c.y, zf = c.z, tf = c.t, xb = c.x, yb = c.y, zb = c.z, tb = c.t;
            if (mu == 0) { xf = (c.x + 1 == g.X) ? 0 : c.x + 1; xb = (c.x == 0) ? g.X - 1 : c.x - 1; }
            if (mu == 1) { yf = (c.y + 1 == g.Y) ? 0 : c.y + 1; yb = (c.y == 0) ? g.Y - 1 : c.y - 1; }
            if (mu == 2) { zf = (c.z + 1 == g.Z) ? 0 : c.z + 1; zb = (c.z == 0) ? g.Z - 1 : c.z - 1; }
            if (mu == 3) { tf = (c.t + 1 == g.T) ? 0 : c.t + 1; tb = (c.t == 0) ? g.T - 1 : c.t - 1; }
            nf = cb_index(g, xf, yf, zf, tf);
            nb = cb_index(g, xb, yb, zb, tb);
        };
        auto issue_spinor = [&](const void* base, long idx, int unit0, int nidx) {
            const uint4* gp = reinterpret_cast<const uint4*>(base);
#pragma unroll
            for (int u = 0; u < G::SP16; ++u) cp_async16(&s16[(unit0 + u) * BS + t], gp + (long)u * g.vh + idx);
            if constexpr (G::NORM)
                cp_async4(&sN[nidx * BS + t], reinterpret_cast<const char*>(base) + (size_t)g.vh * NC * 4 + idx * 4);
        };
        auto issue_link = [&](const void* base, int mu, long idx, int unit0) {
            const unsigned char* gp = reinterpret_cast<const unsigned char*>(base);
#pragma unroll
            for (int kk = 0; kk < G::NL; ++kk) {
                const unsigned char* src = gp + ((long)(mu * G::NL + kk) * g.vh + idx) * G::LB;
                unsigned char* dst = sL + (size_t)((unit0 + kk) * BS + t) * G::LB;
                if constexpr (G::LB == 16) cp_async16(dst, src);
                else if constexpr (G::LB == 8) cp_async8(dst, src);
                else cp_async4(dst, src);
            }
        };
        auto issue_stage = [&](int mu, int buf) {
            long nf, nb;
            nbr(mu, nf, nb);
            issue_spinor(pr.in, nf, (buf * 2 + 0) * G::SP16, buf * 2 + 0);
            issue_link(pr.gauge[po], mu, i, (buf * 2 + 0) * G::NL);
            issue_spinor(pr.in, nb, (buf * 2 + 1) * G::SP16, buf * 2 + 1);
            issue_link(pr.gauge[1 - po], mu, nb, (buf * 2 + 1) * G::NL);
        };
        // group 0: site-local epilogue data; groups 1, 2: directions 0, 1
        {
            const uint4* gc = reinterpret_cast<const uint4*>(pr.clov);
#pragma unroll
            for (int u = 0; u < G::CLV16; ++u) cp_async16(&s16[(4 * G::SP16 + u) * BS + t], gc + (long)u * g.vh + i);
            if constexpr (G::LOC) issue_spinor(pr.loc, i, 4 * G::SP16 + G::CLV16, 4);
            cp_commit();
        }
        issue_stage(0, 0);
        cp_commit();
        issue_stage(1, 1);
        cp_commit();

        cpx<R> acc[NF][4][3];
#pragma unroll
        for (int f = 0; f < NF; ++f)
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int a = 0; a < 3; ++a) acc[f][s][a] = C((R)0, (R)0);

        const R phf = (c.t + 1 == g.T) ? (R)pr.bc_t : (R)1;
        const R phb = (c.t == 0) ? (R)pr.bc_t : (R)1;
        auto consume = [&](auto MUc, int buf) {
            constexpr int MU = decltype(MUc)::value;
            cpx<R> u[9];
            cpx<R> psi[NC];
            constexpr bool SC = (P == PF16 || P == PB16);
            sp_from_smem<P, NC>(s16, (buf * 2 + 0) * G::SP16, sN, buf * 2 + 0, BS, t, psi);
            link_from_smem<P>(sL, (buf * 2 + 0) * G::NL, BS, t, u);
            R fac = MU == 3 ? phf : (R)1;
            if constexpr (SC) fac *= (R)sN[(buf * 2 + 0) * BS + t];
#pragma unroll
            for (int f = 0; f < NF; ++f) hop_dir<R, MU, -1, false, SC>(acc[f], psi + 12 * f, u, fac);
            sp_from_smem<P, NC>(s16, (buf * 2 + 1) * G::SP16, sN, buf * 2 + 1, BS, t, psi);
            link_from_smem<P>(sL, (buf * 2 + 1) * G::NL, BS, t, u);
            fac = MU == 3 ? phb : (R)1;
            if constexpr (SC) fac *= (R)sN[(buf * 2 + 1) * BS + t];
#pragma unroll
            for (int f = 0; f < NF; ++f) hop_dir<R, MU, +1, true, SC>(acc[f], psi + 12 * f, u, fac);
        };
        cp_wait<1>();
        consume(std::integral_constant<int, 0>{}, 0);
        issue_stage(2, 0);
        cp_commit();
        cp_wait<1>();
        consume(std::integral_constant<int, 1>{}, 1);
        issue_stage(3, 1);
        cp_commit();
        cp_wait<1>();
        consume(std::integral_constant<int, 2>{}, 0);
        cp_wait<0>();
        consume(std::integral_constant<int, 3>{}, 1);

        const int ue = 4 * G::SP16;   // first epilogue unit
        cpx<R> out[NC];
        if constexpr (KIND == K1_EO_INV) {
            if constexpr (NF == 1) {
#pragma unroll
                for (int cb = 0; cb < 2; ++cb) {
                    cpx<R> v[6], w[6];
#pragma unroll
                    for (int j = 0; j < 6; ++j) v[j] = acc[0][2 * cb + j / 3][j % 3];
                    R m[72];
                    reals_from_smem<P, 72>(s16, ue + 72 * cb * G::ESZ / 16, BS, t, m);
                    if (pr.sign > 0) full6_mv<R, false>(w, m, v);
                    else full6_mv<R, true>(w, m, v);
#pragma unroll
                    for (int j = 0; j < 6; ++j) out[6 * cb + j] = w[j];
                }
            } else {
                // heavy: per chirality [A_c - 1 36][D_c - 1 36] (the layout and the
                // block inverse are described in dslash_heavy.cu):
                //   w_u = A D v_u - i s sigma mubar_t D v_u + epsbar_t D v_d, and u <-> d with +i
                const R tw = (R)pr.tw, eps = (R)pr.eps;
#pragma unroll
                for (int cb = 0; cb < 2; ++cb) {
                    cpx<R> vu[6], vd[6], du[6], dd[6], wu[6], wd[6];
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        vu[j] = acc[0][2 * cb + j / 3][j % 3];
                        vd[j] = acc[NF - 1][2 * cb + j / 3][j % 3];
                        du[j] = vu[j];
                        dd[j] = vd[j];
                    }
                    R m[40];
                    reals_from_smem<P, 40>(s16, ue + (72 * cb + 32) * G::ESZ / 16, BS, t, m);   // D_c - 1 at m + 4
                    herm6_mv_acc<R>(du, m + 4, vu);
                    herm6_mv_acc<R>(dd, m + 4, vd);
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        wu[j] = du[j];
                        wd[j] = dd[j];
                    }
                    reals_from_smem<P, 40>(s16, ue + 72 * cb * G::ESZ / 16, BS, t, m);          // A_c - 1 at m
                    herm6_mv_acc<R>(wu, m, du);
                    herm6_mv_acc<R>(wd, m, dd);
                    const R ts = cb == 0 ? tw : -tw;
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        out[6 * cb + j] = wu[j] - ts * mul_i(du[j]) + eps * dd[j];
                        out[12 + 6 * cb + j] = wd[j] + ts * mul_i(dd[j]) + eps * du[j];
                    }
                }
            }
        } else {
            cpx<R> psi[NC];
            sp_from_smem<P, NC>(s16, ue + G::CLV16, sN, 4, BS, t, psi);
            if constexpr (P == PB16 || P == PF16) {
                const R sc = (R)sN[4 * BS + t];
#pragma unroll
                for (int k = 0; k < NC; ++k) psi[k] = sc * psi[k];
            }
            R m[72];
            reals_from_smem<P, 72>(s16, ue, BS, t, m);
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
                for (int q = 0; q < NC; ++q) s += norm2(out[q]);
                nrm = (double)s;
            }
        }
        store_spinor<P, NC>(pr.out, g.vh, i, out);
    }
    if constexpr (KIND == K2_OE_LOCAL) {
        if (pr.partial != nullptr) {
            const double bs = block_sum<BS>(nrm, shred);
            reduce_finalize<BS>(pr.partial, pr.counter, pr.nblk, lb, bs, b.fin, pr.ctl, pr.ms, nullptr, shred);
        }
    }
}

template <int P, int NF, int KIND, int NP>
cudaError_t launch_dslash_staged(const OpBatch<NP>& b, int nblocks, cudaStream_t st) {
    constexpr int BS = STAGED_BS;
    constexpr size_t bytes = (size_t)Stg<P, 12 * NF, KIND, NF>::BYTES * BS;
    static bool configured = false;
    if (!configured) {
        cudaError_t e = cudaFuncSetAttribute(dslash_staged_kernel<P, NF, KIND, NP, BS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
        if (e != cudaSuccess) return e;
        configured = true;
    }
    dslash_staged_kernel<P, NF, KIND, NP, BS><<<nblocks, BS, bytes, st>>>(b);
    return cudaGetLastError();
}

#define TM_SINST(P, NF, KIND, NP) \
    template cudaError_t launch_dslash_staged<P, NF, KIND, NP>(const OpBatch<NP>&, int, cudaStream_t);
#define TM_SINST_P(P)                                                                         \
    TM_SINST(P, 1, K1_EO_INV, 1) TM_SINST(P, 1, K2_OE_LOCAL, 1) TM_SINST(P, 2, K1_EO_INV, 1)   \
    TM_SINST(P, 2, K2_OE_LOCAL, 1) TM_SINST(P, 1, K1_EO_INV, MAXP) TM_SINST(P, 1, K2_OE_LOCAL, MAXP)
TM_SINST_P(P32)
TM_SINST_P(PB16)
TM_SINST_P(PF16)

}  // namespace tmk
