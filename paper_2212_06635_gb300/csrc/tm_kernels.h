// Kernel-side helpers shared by the translation units (deterministic block/grid
// reductions, solver-scalar finalisers) and the host-visible launcher
// declarations.
#pragma once

#include "tm_internal.h"

namespace tmk {

constexpr int DSLASH_BS = 128;   // direct stencil kernel
constexpr int STAGED_BS = 64;    // shared-memory staged stencil kernel
constexpr int BLAS_BS = 256;
constexpr int MIN_BS = 64;       // smallest block size of any reducing kernel (sizes the partials)

enum DslashKind { K1_EO_INV = 0, K2_OE_LOCAL = 1 };

// FinOp codes beyond those in tm_internal.h
enum { FIN_PP = 4, FIN_CG_UPDATE = 5, FIN_MS_UPDATE = 6 };

// ---------------------------------------------------------------------------
// solver scalar finalisers (run by one thread of the last block of a reduction)
// ---------------------------------------------------------------------------
__device__ inline void ms_alpha(MsCtl* ms, double alpha) {
    // zeta recurrences of multishift CG for the shifts still active
    for (int k = 0; k < ms->nshift; ++k) {
        if (ms->active[k] != 1) { ms->active[k] = 0; ms->alpha_s[k] = 0.0; continue; }
        const double z = ms->zeta[k], zo = ms->zeta_old[k];
        const double den = alpha * ms->beta_old * (zo - z) + zo * ms->alpha_old * (1.0 + ms->dshift[k] * alpha);
        const double zn = z * zo * ms->alpha_old / den;
        ms->alpha_s[k] = alpha * zn / z;
        ms->beta_s[k] = zn / z;            // ratio kept until beta is known
        ms->zeta_old[k] = z;
        ms->zeta[k] = zn;
    }
    ms->alpha_old = alpha;
}

__device__ inline void finalize_scalar(int fin, double t, SolverCtl* ctl, MsCtl* ms, double* dst) {
    switch (fin) {
        case FIN_STORE:
            if (dst) *dst = t; else ctl->result = t;
            break;
        case FIN_PP:
            ctl->result = t;   // ||p||^2 for shifted systems
            break;
        case FIN_CG_ALPHA:
        case FIN_MS_ALPHA: {
            const double pAp = t + ctl->shift * ctl->result;
            ctl->pAp = pAp;
            if (!(pAp > 0.0) || !isfinite(pAp)) {
                ctl->flag = CTL_BREAKDOWN;
            } else {
                ctl->alpha = ctl->rr / pAp;
                if (fin == FIN_MS_ALPHA) ms_alpha(ms, ctl->alpha);
            }
            break;
        }
        case FIN_CG_UPDATE:
        case FIN_MS_UPDATE: {
            ctl->rr_old = ctl->rr;
            ctl->rr = t;
            ctl->beta = t / ctl->rr_old;
            ctl->iter += 1;
            if (!isfinite(t)) ctl->flag = CTL_BREAKDOWN;
            else if (t < ctl->stop_rr) ctl->flag = CTL_STOP;
            else if (ctl->iter >= ctl->maxiter) ctl->flag = CTL_MAXITER;
            if (fin == FIN_MS_UPDATE) {
                int na = 0;
                for (int k = 0; k < ms->nshift; ++k) {
                    if (!ms->active[k]) continue;
                    const double ratio = ms->beta_s[k];
                    ms->beta_s[k] = ctl->beta * ratio * ratio;
                    // shifted residual r_k = zeta_k r
                    if (ms->zeta[k] * ms->zeta[k] * t < ms->stop_rr) ms->active[k] = 2;  // converged, last update pending
                    else ++na;
                }
                ms->beta_old = ctl->beta;
                ms->n_active = na;
                if (na == 0 && ctl->flag == CTL_RUN) ctl->flag = CTL_STOP;
            }
            break;
        }
        default:
            break;
    }
}

template <int BS>
__device__ __forceinline__ double block_sum(double v, double* sh) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) sh[w] = v;
    __syncthreads();
    double t = 0.0;
    if (threadIdx.x < 32) {
        t = (threadIdx.x < BS / 32) ? sh[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
}

// Each block stores its partial; the last block to arrive sums all partials in
// index order (deterministic for a fixed grid) and runs the finaliser.
template <int BS>
__device__ __forceinline__ void reduce_finalize(double* partial, unsigned int* counter, int nblk,
                                                int lb, double bsum, int fin, SolverCtl* ctl,
                                                MsCtl* ms, double* dst, double* sh) {
    __shared__ int am_last;
    if (threadIdx.x == 0) {
        partial[lb] = bsum;
        __threadfence();
        const unsigned prev = atomicAdd(counter, 1u);
        am_last = (prev == (unsigned)(nblk - 1));
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double t = 0.0;
    for (int k = threadIdx.x; k < nblk; k += BS) t += ((volatile double*)partial)[k];
    t = block_sum<BS>(t, sh);
    if (threadIdx.x == 0) {
        *counter = 0u;
        finalize_scalar(fin, t, ctl, ms, dst);
    }
}

// ---------------------------------------------------------------------------
// vector (BLAS-1) problem tables
// ---------------------------------------------------------------------------
struct VecProb {
    long vh;
    int nblk;
    void* v[6];
    SolverCtl* ctl;
    MsCtl* ms;
    double* partial;
    unsigned int* counter;
    double* dst;
};

template <int NP>
struct VecBatch {
    int n;
    int fin;
    int blk_start[NP + 1];
    VecProb p[NP];
};

template <int NP>
__device__ __forceinline__ int find_vproblem(const VecBatch<NP>& b, int blk) {
    int k = 0;
#pragma unroll 1
    while (k + 1 < b.n && blk >= b.blk_start[k + 1]) ++k;
    return k;
}

// multishift vectors (single problem)
struct MsVecs {
    void* x[MAX_SHIFTS];
    void* p[MAX_SHIFTS];
};

// ---------------------------------------------------------------------------
// launchers (host)
// ---------------------------------------------------------------------------
template <int P, int NF, int KIND, int NP>
cudaError_t launch_dslash(const OpBatch<NP>& b, int nblocks, cudaStream_t st);
// shared-memory staged variant (FP32 / 16-bit storage), STAGED_BS threads per block
template <int P, int NF, int KIND, int NP>
cudaError_t launch_dslash_staged(const OpBatch<NP>& b, int nblocks, cudaStream_t st);

// p = r + beta p (+ ||p||^2 when the problem has a shift)       v = {p, r}
template <int P, int NC, int NP>
cudaError_t launch_cg_pupdate(const VecBatch<NP>& b, int nblocks, cudaStream_t st);
// x += alpha p; r -= alpha (Ap + shift p); ||r||^2 -> FIN_CG_UPDATE   v = {x, p, r, Ap}
template <int P, int PX, int NC, int NP>
cudaError_t launch_cg_update(const VecBatch<NP>& b, int nblocks, cudaStream_t st);
// dst (precision PD) = src (precision PS)                        v = {dst, src}
template <int PD, int PS, int NC, int NP>
cudaError_t launch_convert(const VecBatch<NP>& b, int nblocks, cudaStream_t st);
// y(F64) += x(PS)                                                v = {y, x}
template <int PS, int NC, int NP>
cudaError_t launch_add_to64(const VecBatch<NP>& b, int nblocks, cudaStream_t st);
// r(F64) = b - Ax - shift x, ||r||^2 -> FIN_STORE(dst)           v = {r, b, Ax, x}
template <int NC, int NP>
cudaError_t launch_residual64(const VecBatch<NP>& b, int nblocks, cudaStream_t st);
// ||v0||^2 -> FIN_STORE(dst)
template <int P, int NC, int NP>
cudaError_t launch_norm2(const VecBatch<NP>& b, int nblocks, cudaStream_t st);
// v0 = v0 * scale (F64 native) where scale = 1/sqrt(*dst)  (power iteration)
template <int NC>
cudaError_t launch_normalize64(const VecBatch<1>& b, int nblocks, cudaStream_t st);

// multishift: r_new = r - alpha (Ap + s0 p), ||r||^2 -> FIN_MS_UPDATE    v = {r, p, Ap}
template <int P, int NC>
cudaError_t launch_ms_update(const VecBatch<1>& b, int nblocks, cudaStream_t st);
// multishift: x_k += alpha_k p_k (pending); p_k = zeta_k r + beta_k p_k; p = r + beta p
template <int P, int PX, int NC>
cudaError_t launch_ms_pupdate(const VecBatch<1>& b, const MsVecs& mv, int first, int nblocks,
                              cudaStream_t st);
// multishift tail: x_k += alpha_k p_k for shifts with a pending update
template <int P, int PX, int NC>
cudaError_t launch_ms_finish(const VecBatch<1>& b, const MsVecs& mv, int nblocks, cudaStream_t st);

// layout
template <int P, int NC>
cudaError_t launch_import(void* dst, const double* src, long vh, cudaStream_t st);
template <int P, int NC>
cudaError_t launch_export(double* dst, const void* src, long vh, cudaStream_t st);
template <int P>
cudaError_t launch_links_from64(void* dst, const void* src64, long vh, cudaStream_t st);
template <int P>
cudaError_t launch_clover_from64(void* dst, const double* src, long vh, int nreal, cudaStream_t st);
cudaError_t launch_f64_to_df(void* dst, const void* src, long n, cudaStream_t st);
cudaError_t launch_df_to_f64(void* dst, const void* src, long n, cudaStream_t st);

}  // namespace tmk
