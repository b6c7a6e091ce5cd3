// BLAS-1 steps of CG / multishift CG (Sec. 4) with fused FP64 reductions, and
// precision conversions between native fields.  One thread per site; each
// thread moves a whole spinor with 16-byte vector accesses.  Reductions: per
// thread in the arithmetic precision, then FP64 warp shuffles, one partial per
// block, and a fixed-order sum by the last block (deterministic).
#include "tm_internal.h"
#include "tm_kernels.h"

namespace tmk {

#define TM_VEC_PROLOGUE(NP)                                 \
    __shared__ double sh[BLAS_BS / 32];                     \
    const int k = find_vproblem<NP>(b, blockIdx.x);         \
    const VecProb& pr = b.p[k];                             \
    const int lb = blockIdx.x - b.blk_start[k];             \
    const long i = (long)lb * BLAS_BS + threadIdx.x;        \
    const bool valid = i < pr.vh;                           \
    (void)sh; (void)valid;

// p = r + beta p
template <int P, int NC, int NP>
__global__ void __launch_bounds__(BLAS_BS) k_cg_pupdate(const __grid_constant__ VecBatch<NP> b) {
    using R = typename PT<P>::R;
    TM_VEC_PROLOGUE(NP)
    if (pr.ctl->flag != CTL_RUN) return;
    const R beta = (R)pr.ctl->beta;
    const bool want = pr.ctl->shift != 0.0;
    double s = 0.0;
    if (valid) {
        cpx<R> p[NC], r[NC];
        load_spinor<P, NC>(pr.v[1], pr.vh, i, r);
        if (beta != (R)0) {
            load_spinor<P, NC>(pr.v[0], pr.vh, i, p);
#pragma unroll
            for (int q = 0; q < NC; ++q) p[q] = r[q] + beta * p[q];
        } else {
#pragma unroll
            for (int q = 0; q < NC; ++q) p[q] = r[q];
        }
        store_spinor<P, NC>(pr.v[0], pr.vh, i, p);
        if (want) {
            R t = (R)0;
#pragma unroll
            for (int q = 0; q < NC; ++q) t += norm2(p[q]);
            s = (double)t;
        }
    }
    if (want) {
        const double bs = block_sum<BLAS_BS>(s, sh);
        reduce_finalize<BLAS_BS>(pr.partial, pr.counter, pr.nblk, lb, bs, FIN_PP, pr.ctl, pr.ms,
                                 nullptr, sh);
    }
}

// x += alpha p;  r -= alpha (Ap + shift p);  ||r||^2
template <int P, int PX, int NC, int NP>
__global__ void __launch_bounds__(BLAS_BS) k_cg_update(const __grid_constant__ VecBatch<NP> b) {
    using R = typename PT<P>::R;
    using RX = typename PT<PX>::R;
    TM_VEC_PROLOGUE(NP)
    if (pr.ctl->flag != CTL_RUN) return;
    const R alpha = (R)pr.ctl->alpha;
    const R sh_ = (R)pr.ctl->shift;
    double s = 0.0;
    if (valid) {
        cpx<R> p[NC], r[NC], ap[NC];
        cpx<RX> x[NC];
        load_spinor<P, NC>(pr.v[1], pr.vh, i, p);
        load_spinor<P, NC>(pr.v[2], pr.vh, i, r);
        load_spinor<P, NC>(pr.v[3], pr.vh, i, ap);
        load_spinor<PX, NC>(pr.v[0], pr.vh, i, x);
        R t = (R)0;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            x[q].re += (RX)(alpha * p[q].re);
            x[q].im += (RX)(alpha * p[q].im);
            cpx<R> a = ap[q];
            if (sh_ != (R)0) a = a + sh_ * p[q];
            r[q] = r[q] - alpha * a;
            t += norm2(r[q]);
        }
        store_spinor<PX, NC>(pr.v[0], pr.vh, i, x);
        store_spinor<P, NC>(pr.v[2], pr.vh, i, r);
        s = (double)t;
    }
    const double bs = block_sum<BLAS_BS>(s, sh);
    reduce_finalize<BLAS_BS>(pr.partial, pr.counter, pr.nblk, lb, bs, FIN_CG_UPDATE, pr.ctl, pr.ms,
                             nullptr, sh);
}

template <int PD, int PS, int NC, int NP>
__global__ void __launch_bounds__(BLAS_BS) k_convert(const __grid_constant__ VecBatch<NP> b) {
    using RD = typename PT<PD>::R;
    using RS = typename PT<PS>::R;
    TM_VEC_PROLOGUE(NP)
    if (!valid) return;
    cpx<RS> s[NC];
    cpx<RD> d[NC];
    load_spinor<PS, NC>(pr.v[1], pr.vh, i, s);
#pragma unroll
    for (int q = 0; q < NC; ++q) d[q] = C((RD)s[q].re, (RD)s[q].im);
    store_spinor<PD, NC>(pr.v[0], pr.vh, i, d);
}

template <int PS, int NC, int NP>
__global__ void __launch_bounds__(BLAS_BS) k_add_to64(const __grid_constant__ VecBatch<NP> b) {
    using RS = typename PT<PS>::R;
    TM_VEC_PROLOGUE(NP)
    if (!valid) return;
    cpx<RS> x[NC];
    cpx<double> y[NC];
    load_spinor<PS, NC>(pr.v[1], pr.vh, i, x);
    load_spinor<P64, NC>(pr.v[0], pr.vh, i, y);
#pragma unroll
    for (int q = 0; q < NC; ++q) y[q] = y[q] + C((double)x[q].re, (double)x[q].im);
    store_spinor<P64, NC>(pr.v[0], pr.vh, i, y);
}

// r = b - Ax - shift x (FP64), ||r||^2 -> *dst
template <int NC, int NP>
__global__ void __launch_bounds__(BLAS_BS) k_residual64(const __grid_constant__ VecBatch<NP> b) {
    TM_VEC_PROLOGUE(NP)
    const double shv = pr.ctl ? pr.ctl->shift : 0.0;
    double s = 0.0;
    if (valid) {
        cpx<double> r[NC], bb[NC], ax[NC], x[NC];
        load_spinor<P64, NC>(pr.v[1], pr.vh, i, bb);
        load_spinor<P64, NC>(pr.v[2], pr.vh, i, ax);
        if (shv != 0.0) load_spinor<P64, NC>(pr.v[3], pr.vh, i, x);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            r[q] = bb[q] - ax[q];
            if (shv != 0.0) r[q] = r[q] - shv * x[q];
            s += norm2(r[q]);
        }
        store_spinor<P64, NC>(pr.v[0], pr.vh, i, r);
    }
    const double bs = block_sum<BLAS_BS>(s, sh);
    reduce_finalize<BLAS_BS>(pr.partial, pr.counter, pr.nblk, lb, bs, FIN_STORE, pr.ctl, pr.ms,
                             pr.dst, sh);
}

template <int P, int NC, int NP>
__global__ void __launch_bounds__(BLAS_BS) k_norm2(const __grid_constant__ VecBatch<NP> b) {
    using R = typename PT<P>::R;
    TM_VEC_PROLOGUE(NP)
    double s = 0.0;
    if (valid) {
        cpx<R> v[NC];
        load_spinor<P, NC>(pr.v[0], pr.vh, i, v);
        if constexpr (P == P64) {
#pragma unroll
            for (int q = 0; q < NC; ++q) s += norm2(v[q]);
        } else {
            R t = (R)0;
#pragma unroll
            for (int q = 0; q < NC; ++q) t += norm2(v[q]);
            s = (double)t;
        }
    }
    const double bs = block_sum<BLAS_BS>(s, sh);
    reduce_finalize<BLAS_BS>(pr.partial, pr.counter, pr.nblk, lb, bs, FIN_STORE, pr.ctl, pr.ms,
                             pr.dst, sh);
}

template <int NC>
__global__ void __launch_bounds__(BLAS_BS) k_normalize64(const __grid_constant__ VecBatch<1> b) {
    TM_VEC_PROLOGUE(1)
    if (!valid) return;
    const double sc = 1.0 / sqrt(*pr.dst);
    cpx<double> v[NC];
    load_spinor<P64, NC>(pr.v[0], pr.vh, i, v);
#pragma unroll
    for (int q = 0; q < NC; ++q) v[q] = sc * v[q];
    store_spinor<P64, NC>(pr.v[0], pr.vh, i, v);
}

// ---------------------------------------------------------------------------
// multishift CG vector updates (Sec. 4.2)
// ---------------------------------------------------------------------------
// r_new = r - alpha (Ap + s0 p);  ||r_new||^2 -> FIN_MS_UPDATE
template <int P, int NC>
__global__ void __launch_bounds__(BLAS_BS) k_ms_update(const __grid_constant__ VecBatch<1> b) {
    using R = typename PT<P>::R;
    TM_VEC_PROLOGUE(1)
    if (pr.ctl->flag != CTL_RUN) return;
    const R alpha = (R)pr.ctl->alpha;
    const R s0 = (R)pr.ctl->shift;
    double s = 0.0;
    if (valid) {
        cpx<R> r[NC], p[NC], ap[NC];
        load_spinor<P, NC>(pr.v[0], pr.vh, i, r);
        load_spinor<P, NC>(pr.v[1], pr.vh, i, p);
        load_spinor<P, NC>(pr.v[2], pr.vh, i, ap);
        R t = (R)0;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            r[q] = r[q] - alpha * (ap[q] + s0 * p[q]);
            t += norm2(r[q]);
        }
        store_spinor<P, NC>(pr.v[0], pr.vh, i, r);
        s = (double)t;
    }
    const double bs = block_sum<BLAS_BS>(s, sh);
    reduce_finalize<BLAS_BS>(pr.partial, pr.counter, pr.nblk, lb, bs, FIN_MS_UPDATE, pr.ctl, pr.ms,
                             nullptr, sh);
}

// Start of a multishift iteration: the x_k update of the previous iteration
// (x_k += alpha_k p_k, deferred so that p_k is read once) fused with the new
// directions p_k = zeta_k r + beta_k p_k and p = r + beta p, plus ||p||^2.
template <int P, int PX, int NC>
__global__ void __launch_bounds__(BLAS_BS) k_ms_pupdate(const __grid_constant__ VecBatch<1> b,
                                                        const __grid_constant__ MsVecs mv, int first) {
    using R = typename PT<P>::R;
    using RX = typename PT<PX>::R;
    TM_VEC_PROLOGUE(1)
    if (pr.ctl->flag != CTL_RUN) return;
    const MsCtl* ms = pr.ms;
    const R beta = first ? (R)0 : (R)pr.ctl->beta;
    double s = 0.0;
    if (valid) {
        cpx<R> r[NC];
        load_spinor<P, NC>(pr.v[0], pr.vh, i, r);
        {
            cpx<R> p[NC];
            if (!first) load_spinor<P, NC>(pr.v[1], pr.vh, i, p);
            R t = (R)0;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                p[q] = first ? r[q] : r[q] + beta * p[q];
                t += norm2(p[q]);
            }
            store_spinor<P, NC>(pr.v[1], pr.vh, i, p);
            s = (double)t;
        }
#pragma unroll 1
        for (int kk = 0; kk < ms->nshift; ++kk) {
            const int act = ms->active[kk];
            if (act == 0) continue;
            cpx<R> pk[NC];
            const R zk = (R)ms->zeta[kk];
            if (!first) {
                load_spinor<P, NC>(mv.p[kk], pr.vh, i, pk);
                const R ak = (R)ms->alpha_s[kk];
                cpx<RX> xk[NC];
                load_spinor<PX, NC>(mv.x[kk], pr.vh, i, xk);
#pragma unroll
                for (int q = 0; q < NC; ++q) {
                    xk[q].re += (RX)(ak * pk[q].re);
                    xk[q].im += (RX)(ak * pk[q].im);
                }
                store_spinor<PX, NC>(mv.x[kk], pr.vh, i, xk);
            }
            if (act == 1) {
                const R bk = first ? (R)0 : (R)ms->beta_s[kk];
#pragma unroll
                for (int q = 0; q < NC; ++q) pk[q] = first ? zk * r[q] : zk * r[q] + bk * pk[q];
                store_spinor<P, NC>(mv.p[kk], pr.vh, i, pk);
            }
        }
    }
    const double bs = block_sum<BLAS_BS>(s, sh);
    reduce_finalize<BLAS_BS>(pr.partial, pr.counter, pr.nblk, lb, bs, FIN_PP, pr.ctl, pr.ms,
                             nullptr, sh);
}

// End of a multishift solve: apply the pending x_k += alpha_k p_k.
template <int P, int PX, int NC>
__global__ void __launch_bounds__(BLAS_BS) k_ms_finish(const __grid_constant__ VecBatch<1> b,
                                                       const __grid_constant__ MsVecs mv) {
    using R = typename PT<P>::R;
    using RX = typename PT<PX>::R;
    TM_VEC_PROLOGUE(1)
    if (!valid) return;
    const MsCtl* ms = pr.ms;
#pragma unroll 1
    for (int kk = 0; kk < ms->nshift; ++kk) {
        if (ms->active[kk] == 0) continue;
        const R ak = (R)ms->alpha_s[kk];
        cpx<R> pk[NC];
        cpx<RX> xk[NC];
        load_spinor<P, NC>(mv.p[kk], pr.vh, i, pk);
        load_spinor<PX, NC>(mv.x[kk], pr.vh, i, xk);
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            xk[q].re += (RX)(ak * pk[q].re);
            xk[q].im += (RX)(ak * pk[q].im);
        }
        store_spinor<PX, NC>(mv.x[kk], pr.vh, i, xk);
    }
}

// ---------------------------------------------------------------------------
// canonical FP64 AoS <-> native
// ---------------------------------------------------------------------------
template <int P, int NC>
__global__ void __launch_bounds__(BLAS_BS) k_import(void* dst, const double* __restrict__ src, long vh) {
    using R = typename PT<P>::R;
    const long i = (long)blockIdx.x * BLAS_BS + threadIdx.x;
    if (i >= vh) return;
    cpx<R> s[NC];
    const double2* p = reinterpret_cast<const double2*>(src) + i * NC;
#pragma unroll
    for (int q = 0; q < NC; ++q) {
        const double2 v = p[q];
        s[q] = C((R)v.x, (R)v.y);
    }
    store_spinor<P, NC>(dst, vh, i, s);
}

template <int P, int NC>
__global__ void __launch_bounds__(BLAS_BS) k_export(double* dst, const void* src, long vh) {
    using R = typename PT<P>::R;
    const long i = (long)blockIdx.x * BLAS_BS + threadIdx.x;
    if (i >= vh) return;
    cpx<R> s[NC];
    load_spinor<P, NC>(src, vh, i, s);
    double2* p = reinterpret_cast<double2*>(dst) + i * NC;
#pragma unroll
    for (int q = 0; q < NC; ++q) p[q] = make_double2((double)s[q].re, (double)s[q].im);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <int P, int NC, int NP>
cudaError_t launch_cg_pupdate(const VecBatch<NP>& b, int nb, cudaStream_t st) {
    k_cg_pupdate<P, NC, NP><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int P, int PX, int NC, int NP>
cudaError_t launch_cg_update(const VecBatch<NP>& b, int nb, cudaStream_t st) {
    k_cg_update<P, PX, NC, NP><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int PD, int PS, int NC, int NP>
cudaError_t launch_convert(const VecBatch<NP>& b, int nb, cudaStream_t st) {
    k_convert<PD, PS, NC, NP><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int PS, int NC, int NP>
cudaError_t launch_add_to64(const VecBatch<NP>& b, int nb, cudaStream_t st) {
    k_add_to64<PS, NC, NP><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int NC, int NP>
cudaError_t launch_residual64(const VecBatch<NP>& b, int nb, cudaStream_t st) {
    k_residual64<NC, NP><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int P, int NC, int NP>
cudaError_t launch_norm2(const VecBatch<NP>& b, int nb, cudaStream_t st) {
    k_norm2<P, NC, NP><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int NC>
cudaError_t launch_normalize64(const VecBatch<1>& b, int nb, cudaStream_t st) {
    k_normalize64<NC><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int P, int NC>
cudaError_t launch_ms_update(const VecBatch<1>& b, int nb, cudaStream_t st) {
    k_ms_update<P, NC><<<nb, BLAS_BS, 0, st>>>(b);
    return cudaGetLastError();
}
template <int P, int PX, int NC>
cudaError_t launch_ms_pupdate(const VecBatch<1>& b, const MsVecs& mv, int first, int nb, cudaStream_t st) {
    k_ms_pupdate<P, PX, NC><<<nb, BLAS_BS, 0, st>>>(b, mv, first);
    return cudaGetLastError();
}
template <int P, int PX, int NC>
cudaError_t launch_ms_finish(const VecBatch<1>& b, const MsVecs& mv, int nb, cudaStream_t st) {
    k_ms_finish<P, PX, NC><<<nb, BLAS_BS, 0, st>>>(b, mv);
    return cudaGetLastError();
}
template <int P, int NC>
cudaError_t launch_import(void* dst, const double* src, long vh, cudaStream_t st) {
    k_import<P, NC><<<(unsigned)((vh + BLAS_BS - 1) / BLAS_BS), BLAS_BS, 0, st>>>(dst, src, vh);
    return cudaGetLastError();
}
template <int P, int NC>
cudaError_t launch_export(double* dst, const void* src, long vh, cudaStream_t st) {
    k_export<P, NC><<<(unsigned)((vh + BLAS_BS - 1) / BLAS_BS), BLAS_BS, 0, st>>>(dst, src, vh);
    return cudaGetLastError();
}

// explicit instantiations
#define TM_PX(P) ((P) == P64 ? P64 : P32)
#define TM_BLAS_P_NC_NP(P, NC, NP)                                                           \
    template cudaError_t launch_cg_pupdate<P, NC, NP>(const VecBatch<NP>&, int, cudaStream_t); \
    template cudaError_t launch_cg_update<P, TM_PX(P), NC, NP>(const VecBatch<NP>&, int, cudaStream_t); \
    template cudaError_t launch_add_to64<P, NC, NP>(const VecBatch<NP>&, int, cudaStream_t);   \
    template cudaError_t launch_norm2<P, NC, NP>(const VecBatch<NP>&, int, cudaStream_t);
#define TM_BLAS_P_NC(P, NC)                                                                  \
    TM_BLAS_P_NC_NP(P, NC, 1)                                                                \
    template cudaError_t launch_ms_update<P, NC>(const VecBatch<1>&, int, cudaStream_t);      \
    template cudaError_t launch_ms_pupdate<P, TM_PX(P), NC>(const VecBatch<1>&, const MsVecs&, int, int, cudaStream_t); \
    template cudaError_t launch_ms_finish<P, TM_PX(P), NC>(const VecBatch<1>&, const MsVecs&, int, cudaStream_t); \
    template cudaError_t launch_import<P, NC>(void*, const double*, long, cudaStream_t);      \
    template cudaError_t launch_export<P, NC>(double*, const void*, long, cudaStream_t);
#define TM_BLAS_P(P) TM_BLAS_P_NC(P, 12) TM_BLAS_P_NC(P, 24) TM_BLAS_P_NC_NP(P, 12, MAXP)

TM_BLAS_P(P64)
TM_BLAS_P(P32)
TM_BLAS_P(PB16)
TM_BLAS_P(PF16)
#define TM_CONV2(P, NC, NP)                                                                 \
    template cudaError_t launch_convert<P, P64, NC, NP>(const VecBatch<NP>&, int, cudaStream_t); \
    template cudaError_t launch_convert<P64, P, NC, NP>(const VecBatch<NP>&, int, cudaStream_t);
#define TM_CONV_P(P) TM_CONV2(P, 12, 1) TM_CONV2(P, 24, 1) TM_CONV2(P, 12, MAXP)
TM_CONV_P(P32)
TM_CONV_P(PB16)
TM_CONV_P(PF16)
template cudaError_t launch_convert<P64, P64, 12, 1>(const VecBatch<1>&, int, cudaStream_t);
template cudaError_t launch_convert<P64, P64, 24, 1>(const VecBatch<1>&, int, cudaStream_t);
template cudaError_t launch_convert<P64, P64, 12, MAXP>(const VecBatch<MAXP>&, int, cudaStream_t);
template cudaError_t launch_residual64<12, 1>(const VecBatch<1>&, int, cudaStream_t);
template cudaError_t launch_residual64<24, 1>(const VecBatch<1>&, int, cudaStream_t);
template cudaError_t launch_residual64<12, MAXP>(const VecBatch<MAXP>&, int, cudaStream_t);
template cudaError_t launch_normalize64<12>(const VecBatch<1>&, int, cudaStream_t);
template cudaError_t launch_normalize64<24>(const VecBatch<1>&, int, cudaStream_t);

}  // namespace tmk

// ---------------------------------------------------------------------------
// complex BLAS-1 for flexible CG (FP32 native light fields)
// ---------------------------------------------------------------------------
namespace tmk {

// <a, b> = sum conj(a) b -> dst2[0] (re), dst2[1] (im); deterministic two-level sum
__global__ void __launch_bounds__(BLAS_BS) k_cdot32(const void* a, const void* b, long vh, double* partial,
                                                    unsigned int* counter, double* dst2) {
    __shared__ double sh[BLAS_BS / 32];
    __shared__ int am_last;
    const long i = (long)blockIdx.x * BLAS_BS + threadIdx.x;
    double re = 0.0, im = 0.0;
    if (i < vh) {
        cpx<float> x[12], y[12];
        load_spinor<P32, 12>(a, vh, i, x);
        load_spinor<P32, 12>(b, vh, i, y);
        float r = 0.f, m = 0.f;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            r += x[q].re * y[q].re + x[q].im * y[q].im;
            m += x[q].re * y[q].im - x[q].im * y[q].re;
        }
        re = r;
        im = m;
    }
    re = block_sum<BLAS_BS>(re, sh);
    im = block_sum<BLAS_BS>(im, sh);
    const int nb = gridDim.x;
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = re;
        partial[2 * blockIdx.x + 1] = im;
        __threadfence();
        am_last = atomicAdd(counter, 1u) == (unsigned)(nb - 1);
    }
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    double tr = 0.0, ti = 0.0;
    for (int k = threadIdx.x; k < nb; k += BLAS_BS) {
        tr += ((volatile double*)partial)[2 * k];
        ti += ((volatile double*)partial)[2 * k + 1];
    }
    tr = block_sum<BLAS_BS>(tr, sh);
    ti = block_sum<BLAS_BS>(ti, sh);
    if (threadIdx.x == 0) {
        *counter = 0u;
        dst2[0] = tr;
        dst2[1] = ti;
    }
}

// y += (ar + i ai) x
__global__ void __launch_bounds__(BLAS_BS) k_caxpy32(void* y, const void* x, float ar, float ai, long vh) {
    const long i = (long)blockIdx.x * BLAS_BS + threadIdx.x;
    if (i >= vh) return;
    cpx<float> a[12], b[12];
    load_spinor<P32, 12>(y, vh, i, a);
    load_spinor<P32, 12>(x, vh, i, b);
    const cpx<float> s = C(ar, ai);
#pragma unroll
    for (int q = 0; q < 12; ++q) cfma(a[q], s, b[q]);
    store_spinor<P32, 12>(y, vh, i, a);
}

// y = x + (br + i bi) y
__global__ void __launch_bounds__(BLAS_BS) k_cxpay32(void* y, const void* x, float br, float bi, long vh) {
    const long i = (long)blockIdx.x * BLAS_BS + threadIdx.x;
    if (i >= vh) return;
    cpx<float> a[12], b[12];
    load_spinor<P32, 12>(y, vh, i, a);
    load_spinor<P32, 12>(x, vh, i, b);
    const cpx<float> s = C(br, bi);
#pragma unroll
    for (int q = 0; q < 12; ++q) a[q] = b[q] + s * a[q];
    store_spinor<P32, 12>(y, vh, i, a);
}

cudaError_t launch_cdot32(const void* a, const void* b, long vh, double* partial, unsigned int* counter,
                          double* dst2, cudaStream_t st) {
    k_cdot32<<<(unsigned)((vh + BLAS_BS - 1) / BLAS_BS), BLAS_BS, 0, st>>>(a, b, vh, partial, counter, dst2);
    return cudaGetLastError();
}
cudaError_t launch_caxpy32(void* y, const void* x, double ar, double ai, long vh, cudaStream_t st) {
    k_caxpy32<<<(unsigned)((vh + BLAS_BS - 1) / BLAS_BS), BLAS_BS, 0, st>>>(y, x, (float)ar, (float)ai, vh);
    return cudaGetLastError();
}
cudaError_t launch_cxpay32(void* y, const void* x, double br, double bi, long vh, cudaStream_t st) {
    k_cxpay32<<<(unsigned)((vh + BLAS_BS - 1) / BLAS_BS), BLAS_BS, 0, st>>>(y, x, (float)br, (float)bi, vh);
    return cudaGetLastError();
}

}  // namespace tmk
