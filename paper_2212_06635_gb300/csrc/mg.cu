// Two-level aggregation multigrid on the full twisted-mass clover operator, and
// the GCR solver it preconditions (Sec. 4.1: the light sector's hardest solves
// run a multigrid-preconditioned outer GCR, about a hundred times faster than
// mixed-precision CG at the physical mass; the paper gives no further detail of
// the method).  The textbook Galerkin form for Wilson-type operators:
//
//   full operator  M(s) psi = A psi + i s 2 kappa mu g5 psi - kappa H psi on both
//                  parities (one thread per site, hop as in the Schur kernels);
//   aggregates     lattice blocks of B[0..3] sites, each split by chirality
//                  (spins 0,1 / 2,3): aggregate a = 2 k + h, k the block's
//                  lexicographic index on the block lattice;
//   near-null      nvec given fields, each smoothed by minimal-residual steps on
//                  M v = 0 and normalised;
//   prolongator    per aggregate, the Gram-Schmidt orthonormalisation of the
//                  vectors' restrictions (one CUDA block per aggregate, modified
//                  Gram-Schmidt applied twice); stored [a][j][spin2 colour3][site]
//                  so that a warp's loads of one column are contiguous;
//   coarse op.     M_c = P^+ M P, nearest neighbour on the block lattice: per block
//                  9 dense (2 nvec)^2 complex blocks (self, +x, -x, ..., -t), stored
//                  column-major so that the rows of a column are contiguous, built
//                  directly (CUDA block per (block, source column): the column's
//                  fine image under the local term and every hop, split by the
//                  block the hop starts from, dotted with the block's columns);
//   preconditioner z = P M_c^-1 P^+ r with the coarse system solved by GCR to a
//                  relative residual, then minimal-residual smoothing on M z = r.
//
// Vectors of either level are flat complex arrays in the level's precision
// (FP64 double2, FP32 float2): a full fine field is the even-parity native field
// followed by the odd one, and native spinors are SoA runs of complex numbers, so
// BLAS-1 kernels treat both levels alike.  Reductions are deterministic (fixed
// grid, per-block partials summed in block order by the last block), in FP64.
// Solver scalars (GCR alpha and projections, MR alpha, the residual and stop
// flags) stay on the device in a control word per level; the host reads a
// level's word once per iteration (fine) or per restart cycle (coarse).
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <vector>

#include "tm_host.h"
#include "dslash_common.cuh"

namespace tmk {
tm_status tmk_failf(tm_status s, const char* fmt, ...);
tm_status tmk_ensure_prec(tm_ctx* c, int P, cudaStream_t st);
tm_status tmk_ws_get(tm_ctx* c, int id, size_t bytes, void** out);
}  // namespace tmk

using namespace tmk;

#define MCK(...)                                                                                            \
    do {                                                                                                    \
        cudaError_t e_ = (__VA_ARGS__);                                                                     \
        if (e_ != cudaSuccess)                                                                              \
            return tmk_failf(e_ == cudaErrorMemoryAllocation ? TM_ERR_OOM : TM_ERR_CUDA, "%s: %s (%s:%d)", \
                             #__VA_ARGS__, cudaGetErrorString(e_), __FILE__, __LINE__);                     \
    } while (0)
#define MCKS(...)                     \
    do {                              \
        tm_status s_ = (__VA_ARGS__); \
        if (s_ != TM_OK) return s_;   \
    } while (0)

namespace tmk {

constexpr int MG_MAX_NVEC = 16;
constexpr int MG_MAX_RESTART = 16;
constexpr int MG_BS = 256;
constexpr int MG_GRID_CAP = 608;         // 4 blocks of 256 on each of 152 SMs: grid of every flat-vector kernel
constexpr int MG_NSLOT = 9;              // self, +x, -x, +y, -y, +z, -z, +t, -t
constexpr int MG_NDOT = MG_MAX_RESTART + 1;
constexpr int MG_PART_W = 2 * MG_NDOT;   // doubles per block partial

// ---------------------------------------------------------------------------
// control word of one solver level (device memory)
// ---------------------------------------------------------------------------
struct MgCtl {
    double dot[2 * MG_NDOT];   // complex results of the last pair-dot reduction
    double alpha[2];           // complex step (MR or GCR)
    double na;                 // GCR: ||A z|| before normalisation
    double rr;                 // residual norm^2
    double stop_rr;            // stop when rr < stop_rr
    double nrm2;
    double tol2;               // relative tolerance squared (MGF_RRB sets stop_rr from it)
    int iter, maxiter, flag, pad;
};

enum MgFin { MGF_DOTS = 0, MGF_MR = 1, MGF_GCR = 2, MGF_RR = 3, MGF_NRM = 4, MGF_RR0 = 5, MGF_RRB = 6 };

__device__ inline void mg_finalize(int fin, const double* t, int np, MgCtl* c) {
    switch (fin) {
        case MGF_DOTS:
            for (int q = 0; q < 2 * np; ++q) c->dot[q] = t[q];
            break;
        case MGF_MR: {   // pairs (mr, r), (mr, mr): alpha = <mr, r> / <mr, mr>
            const double den = t[2];
            if (den > 0.0 && isfinite(den)) {
                c->alpha[0] = t[0] / den;
                c->alpha[1] = t[1] / den;
            } else {
                c->alpha[0] = 0.0;
                c->alpha[1] = 0.0;
            }
            break;
        }
        case MGF_GCR: {  // pairs (az, az), (az, r): na = ||az||, alpha = <az, r> / na
            const double n2 = t[0];
            if (!(n2 > 0.0) || !isfinite(n2)) {
                c->flag = CTL_BREAKDOWN;
                c->na = 1.0;
                c->alpha[0] = 0.0;
                c->alpha[1] = 0.0;
            } else {
                const double na = sqrt(n2);
                c->na = na;
                c->alpha[0] = t[2] / na;
                c->alpha[1] = t[3] / na;
            }
            break;
        }
        case MGF_RR:
            c->rr = t[0];
            c->iter += 1;
            if (!isfinite(t[0])) c->flag = CTL_BREAKDOWN;
            else if (t[0] < c->stop_rr) c->flag = CTL_STOP;
            else if (c->iter >= c->maxiter) c->flag = CTL_MAXITER;
            break;
        case MGF_RR0:    // true residual at a restart: no iteration counted
            c->rr = t[0];
            if (!isfinite(t[0])) c->flag = CTL_BREAKDOWN;
            else if (t[0] < c->stop_rr) c->flag = CTL_STOP;
            break;
        case MGF_NRM:
            c->nrm2 = t[0];
            break;
        case MGF_RRB:    // start of a solve from x = 0: r = b, stop relative to ||b||
            c->rr = t[0];
            c->stop_rr = c->tol2 * t[0];
            if (!(t[0] > 0.0) || !isfinite(t[0])) c->flag = CTL_STOP;   // b = 0 (x = 0 is the solution) or not finite
            break;
        default:
            break;
    }
}

// ---------------------------------------------------------------------------
// flat complex vectors
// ---------------------------------------------------------------------------
template <int P> struct CE;
template <> struct CE<P64> { using T = double2; using R = double; };
template <> struct CE<P32> { using T = float2; using R = float; };

template <int P>
__device__ __forceinline__ cpx<typename CE<P>::R> ldc(const void* v, long i) {
    const auto q = __ldg(reinterpret_cast<const typename CE<P>::T*>(v) + i);
    return C(q.x, q.y);
}
template <int P>
__device__ __forceinline__ void stc(void* v, long i, cpx<typename CE<P>::R> z) {
    typename CE<P>::T q;
    q.x = z.re;
    q.y = z.im;
    reinterpret_cast<typename CE<P>::T*>(v)[i] = q;
}
// plain (cached) load for vectors written earlier in the same kernel
template <int P>
__device__ __forceinline__ cpx<typename CE<P>::R> ldw(const void* v, long i) {
    const auto q = reinterpret_cast<const typename CE<P>::T*>(v)[i];
    return C(q.x, q.y);
}

static int flat_grid(long n) {
    const long b = (n + MG_BS - 1) / MG_BS;
    return (int)(b < MG_GRID_CAP ? (b > 0 ? b : 1) : MG_GRID_CAP);
}

// Block-wide sums of NV doubles held per thread; the totals land in out[0..NV)
// (shared memory) for every thread after the call.
template <int NV>
__device__ __forceinline__ void block_sums(double (&v)[NV], double* red, double* out) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double t = v[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
        if (l == 0) red[w * NV + q] = t;
    }
    __syncthreads();
    for (int q = threadIdx.x; q < NV; q += blockDim.x) {
        double t = 0.0;
        for (int k = 0; k < nw; ++k) t += red[k * NV + q];
        out[q] = t;
    }
    __syncthreads();
}

// Pair dots: t_q = <u_q, v_q> = sum_i conj(u_q[i]) v_q[i], q < np <= NP; the
// finaliser `fin` consumes them.  Per-thread sums in the vector precision per
// element, FP64 across elements, threads and blocks.
template <int NP>
struct PairDots {
    long n;
    int np;
    int fin;
    const void* u[NP];
    const void* v[NP];
    MgCtl* ctl;
    const MgCtl* gate;    // early exit when gate->flag != CTL_RUN (may be null)
    double* partial;
    unsigned int* counter;
};

template <int P, int NP>
__global__ void __launch_bounds__(MG_BS) k_pairdots(const __grid_constant__ PairDots<NP> a) {
    using R = typename CE<P>::R;
    if (a.gate && a.gate->flag != CTL_RUN) return;
    double acc[2 * NP];
#pragma unroll
    for (int q = 0; q < 2 * NP; ++q) acc[q] = 0.0;
    for (long i = (long)blockIdx.x * MG_BS + threadIdx.x; i < a.n; i += (long)gridDim.x * MG_BS) {
#pragma unroll
        for (int q = 0; q < NP; ++q) {
            if (q < a.np) {
                const cpx<R> u = ldc<P>(a.u[q], i), v = ldc<P>(a.v[q], i);
                acc[2 * q] += (double)(u.re * v.re + u.im * v.im);
                acc[2 * q + 1] += (double)(u.re * v.im - u.im * v.re);
            }
        }
    }
    __shared__ double red[(MG_BS / 32) * 2 * NP];
    __shared__ double tot[2 * NP];
    block_sums<2 * NP>(acc, red, tot);
    __shared__ int am_last;
    if (threadIdx.x < 2 * a.np) a.partial[(long)blockIdx.x * MG_PART_W + threadIdx.x] = tot[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    // every thread sums a fixed stride of the block partials, then one block sum:
    // the same order for a given grid
#pragma unroll
    for (int q = 0; q < 2 * NP; ++q) acc[q] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += MG_BS) {
#pragma unroll
        for (int q = 0; q < 2 * NP; ++q)
            if (q < 2 * a.np) acc[q] += ((volatile double*)a.partial)[(long)b * MG_PART_W + q];
    }
    block_sums<2 * NP>(acc, red, tot);
    if (threadIdx.x == 0) {
        *a.counter = 0u;
        mg_finalize(a.fin, tot, a.np, a.ctl);
    }
}

// a level's control word at the start of a device-driven solve
__global__ void k_ctl_start(MgCtl* c, int maxiter, double tol2) {
    c->iter = 0;
    c->maxiter = maxiter;
    c->tol2 = tol2;
    c->flag = CTL_RUN;
    c->na = 1.0;
}

// y = ca x + cw w (real host scalars; x or w may be null)
template <int P>
__global__ void __launch_bounds__(MG_BS) k_axpby(long n, void* y, double ca, const void* x, double cw, const void* w,
                                                  const MgCtl* gate) {
    using R = typename CE<P>::R;
    if (gate && gate->flag != CTL_RUN) return;
    for (long i = (long)blockIdx.x * MG_BS + threadIdx.x; i < n; i += (long)gridDim.x * MG_BS) {
        cpx<R> t = C((R)0, (R)0);
        if (x) t = t + (R)ca * ldc<P>(x, i);
        if (w) t = t + (R)cw * ldc<P>(w, i);
        stc<P>(y, i, t);
    }
}

// dst (PD) = scale * src (PS), flat (coarse vectors: one complex per element in both precisions)
template <int PD, int PS>
__global__ void __launch_bounds__(MG_BS) k_convert(long n, void* dst, const void* src, double scale) {
    using RD = typename CE<PD>::R;
    for (long i = (long)blockIdx.x * MG_BS + threadIdx.x; i < n; i += (long)gridDim.x * MG_BS) {
        const auto s = ldc<PS>(src, i);
        stc<PD>(dst, i, C((RD)(scale * (double)s.re), (RD)(scale * (double)s.im)));
    }
}

// Full fields of different precisions differ in layout (FP64 keeps one complex
// number per 16-byte vector, FP32 two), so conversions go site by site:
// dst (PD) = scale * src (PS), and y (FP64) += scale * x (PS).
template <int PD, int PS>
__global__ void __launch_bounds__(MG_BS) k_full_convert(void* dst, const void* src, long vh, size_t half_d,
                                                         size_t half_s, double scale) {
    using RS = typename PT<PS>::R;
    using RD = typename PT<PD>::R;
    const long gi = (long)blockIdx.x * MG_BS + threadIdx.x;
    if (gi >= 2 * vh) return;
    const int par = gi >= vh ? 1 : 0;
    const long i = gi - par * vh;
    cpx<RS> s[12];
    load_spinor<PS, 12>(reinterpret_cast<const char*>(src) + par * half_s, vh, i, s);
    cpx<RD> d[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) d[k] = C((RD)(scale * (double)s[k].re), (RD)(scale * (double)s[k].im));
    store_spinor<PD, 12>(reinterpret_cast<char*>(dst) + par * half_d, vh, i, d);
}

template <int PS>
__global__ void __launch_bounds__(MG_BS) k_full_add64(void* y, const void* x, long vh, size_t half_s, double scale) {
    using RS = typename PT<PS>::R;
    const long gi = (long)blockIdx.x * MG_BS + threadIdx.x;
    if (gi >= 2 * vh) return;
    const int par = gi >= vh ? 1 : 0;
    const long i = gi - par * vh;
    const size_t half64 = (size_t)vh * 12 * 16;
    cpx<RS> s[12];
    load_spinor<PS, 12>(reinterpret_cast<const char*>(x) + par * half_s, vh, i, s);
    cpx<double> t[12];
    char* yp = reinterpret_cast<char*>(y) + par * half64;
    load_spinor<P64, 12>(yp, vh, i, t);
#pragma unroll
    for (int k = 0; k < 12; ++k) t[k] = C(t[k].re + scale * (double)s[k].re, t[k].im + scale * (double)s[k].im);
    store_spinor<P64, 12>(yp, vh, i, t);
}

// v *= 1 / sqrt(ctl->nrm2)
template <int P>
__global__ void __launch_bounds__(MG_BS) k_normalize(long n, void* v, const MgCtl* ctl) {
    using R = typename CE<P>::R;
    const R s = (R)(1.0 / sqrt(ctl->nrm2));
    for (long i = (long)blockIdx.x * MG_BS + threadIdx.x; i < n; i += (long)gridDim.x * MG_BS)
        stc<P>(v, i, s * ldw<P>(v, i));
}

// minimal residual step: z += alpha r, r -= alpha mr   (alpha from ctl)
template <int P>
__global__ void __launch_bounds__(MG_BS) k_mr_update(long n, void* z, void* r, const void* mr, const MgCtl* ctl) {
    using R = typename CE<P>::R;
    const cpx<R> al = C((R)ctl->alpha[0], (R)ctl->alpha[1]);
    for (long i = (long)blockIdx.x * MG_BS + threadIdx.x; i < n; i += (long)gridDim.x * MG_BS) {
        const cpx<R> rv = ldw<P>(r, i);
        stc<P>(z, i, ldw<P>(z, i) + al * rv);
        stc<P>(r, i, rv - al * ldc<P>(mr, i));
    }
}

struct PtrList {
    void* q[MG_MAX_RESTART];
};

// GCR orthogonalisation (classical Gram-Schmidt against the stored directions):
// z -= sum_j d_j p_j,  az -= sum_j d_j ap_j,  d_j = <ap_j, az> from ctl->dot
template <int P>
__global__ void __launch_bounds__(MG_BS) k_gcr_orth(long n, int m, void* z, void* az, const __grid_constant__ PtrList p,
                                                     const __grid_constant__ PtrList ap, const MgCtl* ctl) {
    using R = typename CE<P>::R;
    if (ctl->flag != CTL_RUN) return;
    __shared__ double d[2 * MG_MAX_RESTART];
    if (threadIdx.x < 2 * m) d[threadIdx.x] = ctl->dot[threadIdx.x];
    __syncthreads();
    for (long i = (long)blockIdx.x * MG_BS + threadIdx.x; i < n; i += (long)gridDim.x * MG_BS) {
        cpx<R> zz = ldw<P>(z, i), aa = ldw<P>(az, i);
        for (int j = 0; j < m; ++j) {
            const cpx<R> dj = C((R)d[2 * j], (R)d[2 * j + 1]);
            zz = zz - dj * ldc<P>(p.q[j], i);
            aa = aa - dj * ldc<P>(ap.q[j], i);
        }
        stc<P>(z, i, zz);
        stc<P>(az, i, aa);
    }
}

// GCR step: p = z / na, ap = az / na (in place), x += alpha p, r -= alpha ap,
// ||r||^2 -> MGF_RR (iteration count, stop flags)
template <int P>
__global__ void __launch_bounds__(MG_BS) k_gcr_update(long n, void* z, void* az, void* x, void* r, MgCtl* ctl,
                                                       double* partial, unsigned int* counter) {
    using R = typename CE<P>::R;
    if (ctl->flag != CTL_RUN) return;
    const R inv = (R)(1.0 / ctl->na);
    const cpx<R> al = C((R)ctl->alpha[0], (R)ctl->alpha[1]);
    double acc[1] = {0.0};
    for (long i = (long)blockIdx.x * MG_BS + threadIdx.x; i < n; i += (long)gridDim.x * MG_BS) {
        const cpx<R> pz = inv * ldw<P>(z, i), pa = inv * ldw<P>(az, i);
        stc<P>(z, i, pz);
        stc<P>(az, i, pa);
        stc<P>(x, i, ldw<P>(x, i) + al * pz);
        const cpx<R> rn = ldw<P>(r, i) - al * pa;
        stc<P>(r, i, rn);
        acc[0] += (double)norm2(rn);
    }
    __shared__ double red[MG_BS / 32];
    __shared__ double tot[1];
    block_sums<1>(acc, red, tot);
    __shared__ int am_last;
    if (threadIdx.x == 0) partial[(long)blockIdx.x * MG_PART_W] = tot[0];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    acc[0] = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += MG_BS) acc[0] += ((volatile double*)partial)[(long)b * MG_PART_W];
    block_sums<1>(acc, red, tot);
    if (threadIdx.x == 0) {
        *counter = 0u;
        mg_finalize(MGF_RR, tot, 1, ctl);
    }
}

// ---------------------------------------------------------------------------
// full operator, canonical <-> native full fields
// ---------------------------------------------------------------------------
struct FullOp {
    Geom g;
    float bc_t;
    double kappa;
    double tw;               // sign * 2 kappa mu
    const void* gauge[2];
    const void* A[2];        // packed hermitian chirality blocks, 72 reals per site and parity
    const void* in;
    void* out;
    size_t half;             // bytes of one parity half of a full field
    const MgCtl* gate;       // early exit when gate->flag != CTL_RUN (may be null)
    MgCtl* mr;               // non-null: fuse the minimal-residual dots <out, in>, <out, out> (MGF_MR)
    double* partial;         // per-block partials of the fused dots (3 per block)
    unsigned int* counter;
};

template <int P, int MU>
__device__ __forceinline__ void full_hop(cpx<typename PT<P>::R> (&acc)[4][3], const FullOp& a, const Coord& c,
                                         long i, int po) {
    using R = typename PT<P>::R;
    const Geom& g = a.g;
    int xf = c.x, yf = c.y, zf = c.z, tf = c.t;
    int xb = c.x, yb = c.y, zb = c.z, tb = c.t;
    R ph_f = (R)1, ph_b = (R)1;
    if (MU == 0) { xf = (c.x + 1 == g.X) ? 0 : c.x + 1; xb = (c.x == 0) ? g.X - 1 : c.x - 1; }
    if (MU == 1) { yf = (c.y + 1 == g.Y) ? 0 : c.y + 1; yb = (c.y == 0) ? g.Y - 1 : c.y - 1; }
    if (MU == 2) { zf = (c.z + 1 == g.Z) ? 0 : c.z + 1; zb = (c.z == 0) ? g.Z - 1 : c.z - 1; }
    if (MU == 3) {
        if (c.t + 1 == g.T) { tf = 0; ph_f = (R)a.bc_t; } else tf = c.t + 1;
        if (c.t == 0) { tb = g.T - 1; ph_b = (R)a.bc_t; } else tb = c.t - 1;
    }
    const char* src = reinterpret_cast<const char*>(a.in) + (size_t)(1 - po) * a.half;
    cpx<R> u[9];
    cpx<R> psi[12];
    load_spinor<P, 12>(src, g.vh, cb_index(g, xf, yf, zf, tf), psi);
    load_link<P>(a.gauge[po], g.vh, MU, i, u);
    hop_dir<R, MU, -1, false>(acc, psi, u, ph_f);
    const long nb = cb_index(g, xb, yb, zb, tb);
    load_spinor<P, 12>(src, g.vh, nb, psi);
    load_link<P>(a.gauge[1 - po], g.vh, MU, nb, u);
    hop_dir<R, MU, +1, true>(acc, psi, u, ph_b);
}

template <int P>
__device__ __forceinline__ void full_op_site(const FullOp& a, long gi, double (&d)[3]);

// out(x) = A(x) psi(x) + i tw g5 psi(x) - kappa (H psi)(x), one thread per site of
// either parity; optionally the minimal-residual step's dots of (out, psi) fused
template <int P>
__global__ void __launch_bounds__(128) k_full_op(const __grid_constant__ FullOp a) {
    if (a.gate && a.gate->flag != CTL_RUN) return;
    const long gi = (long)blockIdx.x * 128 + threadIdx.x;
    double d[3] = {0.0, 0.0, 0.0};
    if (gi < 2 * a.g.vh) full_op_site<P>(a, gi, d);
    if (!a.mr) return;
    __shared__ double red[(128 / 32) * 3];
    __shared__ double tot[3];
    block_sums<3>(d, red, tot);
    __shared__ int am_last;
    if (threadIdx.x < 3) a.partial[(long)blockIdx.x * 3 + threadIdx.x] = tot[threadIdx.x];
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) am_last = (atomicAdd(a.counter, 1u) == gridDim.x - 1);
    __syncthreads();
    if (!am_last) return;
    __threadfence();
    d[0] = d[1] = d[2] = 0.0;
    for (long b = threadIdx.x; b < (long)gridDim.x; b += 128)
#pragma unroll
        for (int q = 0; q < 3; ++q) d[q] += ((volatile double*)a.partial)[b * 3 + q];
    block_sums<3>(d, red, tot);
    if (threadIdx.x == 0) {
        *a.counter = 0u;
        mg_finalize(MGF_MR, tot, 2, a.mr);
    }
}

template <int P>
__device__ __forceinline__ void full_op_site(const FullOp& a, long gi, double (&d)[3]) {
    using R = typename PT<P>::R;
    const int po = gi >= a.g.vh ? 1 : 0;
    const long i = gi - po * a.g.vh;
    const Coord c = cb_coords(a.g, i, po);
    cpx<R> acc[4][3];
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[s][k] = C((R)0, (R)0);
    full_hop<P, 0>(acc, a, c, i, po);
    full_hop<P, 1>(acc, a, c, i, po);
    full_hop<P, 2>(acc, a, c, i, po);
    full_hop<P, 3>(acc, a, c, i, po);
    cpx<R> psi[12];
    load_spinor<P, 12>(reinterpret_cast<const char*>(a.in) + (size_t)po * a.half, a.g.vh, i, psi);
    R m[72];
    load_reals<P, 72>(a.A[po], a.g.vh, i, 0, m);
    const R kap = (R)a.kappa, tw = (R)a.tw;
    cpx<R> out[12];
#pragma unroll
    for (int cb = 0; cb < 2; ++cb) {
        cpx<R> v[6], w[6];
        const R sc = cb == 0 ? (R)1 : (R)-1;
#pragma unroll
        for (int j = 0; j < 6; ++j) {
            v[j] = psi[6 * cb + j];
            w[j] = (tw * sc) * mul_i(v[j]) - kap * acc[2 * cb + j / 3][j % 3];
        }
        herm6_mv_acc<R>(w, m + 36 * cb, v);
#pragma unroll
        for (int j = 0; j < 6; ++j) out[6 * cb + j] = w[j];
    }
    store_spinor<P, 12>(reinterpret_cast<char*>(a.out) + (size_t)po * a.half, a.g.vh, i, out);
    if (a.mr) {
        R t0 = (R)0, t1 = (R)0, t2 = (R)0;
#pragma unroll
        for (int q = 0; q < 12; ++q) {
            t0 += out[q].re * psi[q].re + out[q].im * psi[q].im;
            t1 += out[q].re * psi[q].im - out[q].im * psi[q].re;
            t2 += norm2(out[q]);
        }
        d[0] = (double)t0;
        d[1] = (double)t1;
        d[2] = (double)t2;
    }
}

// canonical full field [lex][spin][colour] (FP64) <-> native full field
template <int P>
__global__ void __launch_bounds__(MG_BS) k_full_import(void* dst, const double* src, Geom g, size_t half) {
    using R = typename PT<P>::R;
    const long lex = (long)blockIdx.x * MG_BS + threadIdx.x;
    if (lex >= 2 * g.vh) return;
    long r = lex;
    const int x = (int)(r % g.X); r /= g.X;
    const int y = (int)(r % g.Y); r /= g.Y;
    const int z = (int)(r % g.Z);
    const int t = (int)(r / g.Z);
    const int par = (x + y + z + t) & 1;
    cpx<R> s[12];
    const double2* q = reinterpret_cast<const double2*>(src) + lex * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 v = q[k];
        s[k] = C((R)v.x, (R)v.y);
    }
    store_spinor<P, 12>(reinterpret_cast<char*>(dst) + (size_t)par * half, g.vh, lex >> 1, s);
}

template <int P>
__global__ void __launch_bounds__(MG_BS) k_full_export(double* dst, const void* src, Geom g, size_t half) {
    using R = typename PT<P>::R;
    const long lex = (long)blockIdx.x * MG_BS + threadIdx.x;
    if (lex >= 2 * g.vh) return;
    long r = lex;
    const int x = (int)(r % g.X); r /= g.X;
    const int y = (int)(r % g.Y); r /= g.Y;
    const int z = (int)(r % g.Z);
    const int t = (int)(r / g.Z);
    const int par = (x + y + z + t) & 1;
    cpx<R> s[12];
    load_spinor<P, 12>(reinterpret_cast<const char*>(src) + (size_t)par * half, g.vh, lex >> 1, s);
    double2* q = reinterpret_cast<double2*>(dst) + lex * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = make_double2((double)s[k].re, (double)s[k].im);
}

// ---------------------------------------------------------------------------
// aggregates
// ---------------------------------------------------------------------------
struct MgGeom {
    Geom g;
    int B[4];        // block extents
    int nb[4];       // block-lattice extents
    int Vb;          // sites per block
    int Nb;          // blocks
    int nvec;
    size_t half;     // bytes of one parity half of a fine field
};

__device__ __forceinline__ void block_site(const MgGeom& m, int k, int s, int (&x)[4]) {
    int kk = k, ss = s;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int bc = kk % m.nb[d];
        kk /= m.nb[d];
        const int w = ss % m.B[d];
        ss /= m.B[d];
        x[d] = bc * m.B[d] + w;
    }
}
__device__ __forceinline__ int block_of(const MgGeom& m, const int (&x)[4]) {
    return (((x[3] / m.B[3]) * m.nb[2] + x[2] / m.B[2]) * m.nb[1] + x[1] / m.B[1]) * m.nb[0] + x[0] / m.B[0];
}
__device__ __forceinline__ int site_in_block(const MgGeom& m, const int (&x)[4]) {
    return (((x[3] % m.B[3]) * m.B[2] + x[2] % m.B[2]) * m.B[1] + x[1] % m.B[1]) * m.B[0] + x[0] % m.B[0];
}
// neighbour block of k in slot d (0 = k, 1 + 2 mu = +mu, 2 + 2 mu = -mu)
__device__ __forceinline__ int block_nbr(const MgGeom& m, int k, int d) {
    if (d == 0) return k;
    const int mu = (d - 1) >> 1, dir = ((d - 1) & 1) ? -1 : 1;
    int bc[4], kk = k;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        bc[q] = kk % m.nb[q];
        kk /= m.nb[q];
    }
    bc[mu] = (bc[mu] + dir + m.nb[mu]) % m.nb[mu];
    return ((bc[3] * m.nb[2] + bc[2]) * m.nb[1] + bc[1]) * m.nb[0] + bc[0];
}
__device__ __forceinline__ long lex_of(const Geom& g, const int (&x)[4]) {
    return (((long)x[3] * g.Z + x[2]) * g.Y + x[1]) * g.X + x[0];
}
// prolongator element (aggregate a, vector j, component c of the chirality's
// 2 spins x 3 colours, site s of the block)
__device__ __forceinline__ long p_index(const MgGeom& m, int a, int j, int c, int s) {
    return (((long)a * m.nvec + j) * 6 + c) * m.Vb + s;
}

// gather the near-null vectors' restrictions: P[a][j][c][s] = v_j(site s of block k)[spins 2h, 2h+1]
template <int P>
__global__ void __launch_bounds__(MG_BS) k_mg_gather(void* Pm, const void* vecs, size_t field_bytes, MgGeom m) {
    using R = typename PT<P>::R;
    const long gi = (long)blockIdx.x * MG_BS + threadIdx.x;
    if (gi >= (long)m.Nb * m.Vb) return;
    const int k = (int)(gi / m.Vb), s = (int)(gi % m.Vb);
    int x[4];
    block_site(m, k, s, x);
    const long lex = lex_of(m.g, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    for (int j = 0; j < m.nvec; ++j) {
        cpx<R> v[12];
        load_spinor<P, 12>(reinterpret_cast<const char*>(vecs) + (size_t)j * field_bytes + (size_t)par * m.half,
                           m.g.vh, lex >> 1, v);
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int c = 0; c < 6; ++c) stc<P>(Pm, p_index(m, 2 * k + h, j, c, s), v[6 * h + c]);
    }
}

// Gram-Schmidt on every aggregate (one CUDA block each): column j loses its
// components along columns 0..j-1 (modified Gram-Schmidt, the sweep run twice
// for orthogonality to rounding), then is normalised.  FP64 sums.
template <int P>
__global__ void __launch_bounds__(MG_BS) k_mg_orth(void* Pm, MgGeom m) {
    using R = typename CE<P>::R;
    const int a = blockIdx.x;
    const int L = 6 * m.Vb;
    const long base = (long)a * m.nvec * L;
    __shared__ double red[(MG_BS / 32) * 2];
    __shared__ double tot[2];
    for (int j = 0; j < m.nvec; ++j) {
        for (int sweep = 0; sweep < 2; ++sweep) {
            for (int i = 0; i < j; ++i) {
                double acc[2] = {0.0, 0.0};
                for (int e = threadIdx.x; e < L; e += blockDim.x) {
                    const cpx<R> u = ldw<P>(Pm, base + (long)i * L + e), v = ldw<P>(Pm, base + (long)j * L + e);
                    acc[0] += (double)u.re * v.re + (double)u.im * v.im;
                    acc[1] += (double)u.re * v.im - (double)u.im * v.re;
                }
                block_sums<2>(acc, red, tot);
                const cpx<R> d = C((R)tot[0], (R)tot[1]);
                for (int e = threadIdx.x; e < L; e += blockDim.x) {
                    const long q = base + (long)j * L + e;
                    stc<P>(Pm, q, ldw<P>(Pm, q) - d * ldw<P>(Pm, base + (long)i * L + e));
                }
                __syncthreads();
            }
        }
        double acc[2] = {0.0, 0.0};
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const cpx<R> v = ldw<P>(Pm, base + (long)j * L + e);
            acc[0] += (double)v.re * v.re + (double)v.im * v.im;
        }
        block_sums<2>(acc, red, tot);
        const R inv = (R)(1.0 / sqrt(tot[0]));
        for (int e = threadIdx.x; e < L; e += blockDim.x) {
            const long q = base + (long)j * L + e;
            stc<P>(Pm, q, inv * ldw<P>(Pm, q));
        }
        __syncthreads();
    }
}

// coarse = P^+ fine: one CUDA block per lattice block k with one warp per row
// r = h nvec + j (2 nvec warps).  The block's fine sites are staged in shared
// memory (component-major, a chunk of sites at a time); each warp's lanes stride
// over the entries of its prolongator column, which are contiguous in the
// [a][j][c][s] layout, and the row sum is a warp shuffle reduction in FP64.
template <int P>
__global__ void __launch_bounds__(1024) k_mg_restrict(void* coarse, const void* fine, const void* Pm, MgGeom m,
                                                       const MgCtl* gate) {
    using R = typename PT<P>::R;
    constexpr int CH = P == P64 ? 128 : 256;   // sites per staged chunk (24 KB either way)
    if (gate && gate->flag != CTL_RUN) return;
    __shared__ cpx<R> sf[12 * CH];
    const int k = blockIdx.x;
    const int nv = m.nvec;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int h = warp / nv, j = warp % nv;
    const long col = p_index(m, 2 * k + h, j, 0, 0);
    cpx<R> acc = C((R)0, (R)0);
    for (int s0 = 0; s0 < m.Vb; s0 += CH) {
        const int ns = min(CH, m.Vb - s0);
        __syncthreads();
        for (int t = threadIdx.x; t < ns; t += blockDim.x) {
            int x[4];
            block_site(m, k, s0 + t, x);
            const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
            cpx<R> v[12];
            load_spinor<P, 12>(reinterpret_cast<const char*>(fine) + (size_t)par * m.half, m.g.vh,
                               lex_of(m.g, x) >> 1, v);
#pragma unroll
            for (int q = 0; q < 12; ++q) sf[q * CH + t] = v[q];
        }
        __syncthreads();
        for (int e = lane; e < 6 * ns; e += 32) {
            const int c = e / ns, sl = e - c * ns;
            cfma_cj(acc, ldc<P>(Pm, col + (long)c * m.Vb + s0 + sl), sf[(6 * h + c) * CH + sl]);
        }
    }
    double re = (double)acc.re, im = (double)acc.im;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_xor_sync(0xffffffffu, re, o);
        im += __shfl_xor_sync(0xffffffffu, im, o);
    }
    if (lane == 0)
        stc<P>(coarse, (long)k * 2 * nv + warp, C((typename CE<P>::R)re, (typename CE<P>::R)im));
}

// fine = P coarse: one thread per (block, site)
template <int P>
__global__ void __launch_bounds__(MG_BS) k_mg_prolong(void* fine, const void* coarse, const void* Pm, MgGeom m,
                                                       const MgCtl* gate) {
    using R = typename PT<P>::R;
    if (gate && gate->flag != CTL_RUN) return;
    const long gi = (long)blockIdx.x * MG_BS + threadIdx.x;
    if (gi >= (long)m.Nb * m.Vb) return;
    const int k = (int)(gi / m.Vb), s = (int)(gi % m.Vb);
    int x[4];
    block_site(m, k, s, x);
    const int par = (x[0] + x[1] + x[2] + x[3]) & 1;
    cpx<R> v[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = C((R)0, (R)0);
    for (int h = 0; h < 2; ++h)
        for (int j = 0; j < m.nvec; ++j) {
            const cpx<R> u = ldc<P>(coarse, (long)(2 * k + h) * m.nvec + j);
#pragma unroll
            for (int c = 0; c < 6; ++c) cfma(v[6 * h + c], ldc<P>(Pm, p_index(m, 2 * k + h, j, c, s)), u);
        }
    store_spinor<P, 12>(reinterpret_cast<char*>(fine) + (size_t)par * m.half, m.g.vh, lex_of(m.g, x) >> 1, v);
}

// out = M_c in: one thread per (block k, row r); M_c stored [k][slot][c][r], so
// that a warp's loads of one column are contiguous
template <int P>
__global__ void __launch_bounds__(MG_BS) k_mg_coarse(void* out, const void* in, const void* Mc, MgGeom m,
                                                      const MgCtl* gate) {
    using R = typename CE<P>::R;
    if (gate && gate->flag != CTL_RUN) return;
    const int n2 = 2 * m.nvec;
    const long gi = (long)blockIdx.x * MG_BS + threadIdx.x;
    if (gi >= (long)m.Nb * n2) return;
    const int k = (int)(gi / n2), r = (int)(gi % n2);
    cpx<R> acc = C((R)0, (R)0);
    for (int d = 0; d < MG_NSLOT; ++d) {
        const int kn = block_nbr(m, k, d);
        const long base = ((long)k * MG_NSLOT + d) * n2 * n2 + r;
        for (int c = 0; c < n2; ++c) cfma(acc, ldc<P>(Mc, base + (long)c * n2), ldc<P>(in, (long)kn * n2 + c));
    }
    stc<P>(out, gi, acc);
}

// Galerkin coarse operator.  CUDA block (k, column cs = hs nvec + js): for every
// site x of lattice block k, the image W(x) of column cs (a fine field living on
// one aggregate) under the local term (A + i tw g5, chirality-diagonal) and each
// hop -kappa (1 -+ g_mu) U psi(x +- mu), split by the block the hop starts from:
// slot 0 collects the local term and the hops from inside block k, slot 1 + 2 mu
// (2 + 2 mu) the hops from the block in +mu (-mu).  Row r = h nvec + j of slot d
// is <P_{2k+h, j}, W_d> summed over the block's sites.
struct BuildArgs {
    MgGeom m;
    float bc_t;
    double kappa;
    double tw;
    const void* gauge[2];
    const void* A[2];
    const void* Pm;
    void* Mc;
};

template <int P>
__device__ __forceinline__ void col_at(const BuildArgs& b, int cs, const int (&y)[4], cpx<typename PT<P>::R> (&v)[12]) {
    using R = typename PT<P>::R;
    const MgGeom& m = b.m;
    const int hs = cs / m.nvec, js = cs % m.nvec;
    const int ky = block_of(m, y), sy = site_in_block(m, y);
#pragma unroll
    for (int q = 0; q < 12; ++q) v[q] = C((R)0, (R)0);
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        const cpx<R> e = ldc<P>(b.Pm, p_index(m, 2 * ky + hs, js, c, sy));
        if (hs == 0) v[c] = e; else v[6 + c] = e;
    }
}

template <int P, int MU, int S>
__device__ __forceinline__ void build_hop(const BuildArgs& b, int cs, const int (&x)[4], long ix, int px,
                                          cpx<typename PT<P>::R> (&acc)[4][3], int want_slot, int k) {
    // S = -1: forward hop from y = x + mu;  S = +1: backward hop from y = x - mu
    using R = typename PT<P>::R;
    const MgGeom& m = b.m;
    int y[4] = {x[0], x[1], x[2], x[3]};
    const int L = MU == 0 ? m.g.X : MU == 1 ? m.g.Y : MU == 2 ? m.g.Z : m.g.T;
    R ph = (R)1;
    if (S < 0) {
        y[MU] = x[MU] + 1 == L ? 0 : x[MU] + 1;
        if (MU == 3 && x[MU] + 1 == L) ph = (R)b.bc_t;
    } else {
        y[MU] = x[MU] == 0 ? L - 1 : x[MU] - 1;
        if (MU == 3 && x[MU] == 0) ph = (R)b.bc_t;
    }
    const int ky = block_of(m, y);
    const int slot = ky == k ? 0 : (S < 0 ? 1 + 2 * MU : 2 + 2 * MU);
    if (slot != want_slot) return;
    cpx<R> psi[12], u[9];
    col_at<P>(b, cs, y, psi);
    if (S < 0) {
        load_link<P>(b.gauge[px], m.g.vh, MU, ix, u);
        hop_dir<R, MU, -1, false>(acc, psi, u, ph);
    } else {
        const long iy = lex_of(m.g, y) >> 1;
        load_link<P>(b.gauge[1 - px], m.g.vh, MU, iy, u);
        hop_dir<R, MU, +1, true>(acc, psi, u, ph);
    }
}

template <int P, int NV>
__global__ void __launch_bounds__(MG_BS) k_mg_build(const __grid_constant__ BuildArgs b) {
    using R = typename PT<P>::R;
    const MgGeom& m = b.m;
    const int k = blockIdx.x;
    const int cs = blockIdx.y;
    const int nv = m.nvec, n2 = 2 * nv;
    __shared__ double red[(MG_BS / 32) * 4 * NV];
    __shared__ double tot[4 * NV];
    for (int d = 0; d < MG_NSLOT; ++d) {
        double acc[4 * NV];
#pragma unroll
        for (int q = 0; q < 4 * NV; ++q) acc[q] = 0.0;
        for (int s = threadIdx.x; s < m.Vb; s += blockDim.x) {
            int x[4];
            block_site(m, k, s, x);
            const int px = (x[0] + x[1] + x[2] + x[3]) & 1;
            const long ix = lex_of(m.g, x) >> 1;
            cpx<R> h[4][3];
#pragma unroll
            for (int q = 0; q < 4; ++q)
#pragma unroll
                for (int c = 0; c < 3; ++c) h[q][c] = C((R)0, (R)0);
            build_hop<P, 0, -1>(b, cs, x, ix, px, h, d, k);
            build_hop<P, 0, +1>(b, cs, x, ix, px, h, d, k);
            build_hop<P, 1, -1>(b, cs, x, ix, px, h, d, k);
            build_hop<P, 1, +1>(b, cs, x, ix, px, h, d, k);
            build_hop<P, 2, -1>(b, cs, x, ix, px, h, d, k);
            build_hop<P, 2, +1>(b, cs, x, ix, px, h, d, k);
            build_hop<P, 3, -1>(b, cs, x, ix, px, h, d, k);
            build_hop<P, 3, +1>(b, cs, x, ix, px, h, d, k);
            cpx<R> w[12];
            const R kap = (R)b.kappa;
#pragma unroll
            for (int q = 0; q < 12; ++q) w[q] = -kap * h[q / 3][q % 3];
            if (d == 0) {
                // local term on the column's own chirality block
                const int hs = cs / nv;
                cpx<R> v[12];
                col_at<P>(b, cs, x, v);
                R mm[72];
                load_reals<P, 72>(b.A[px], m.g.vh, ix, 0, mm);
                cpx<R> lv[6], ww[6];
                const R sc = hs == 0 ? (R)1 : (R)-1;
#pragma unroll
                for (int q = 0; q < 6; ++q) {
                    lv[q] = v[6 * hs + q];
                    ww[q] = ((R)b.tw * sc) * mul_i(lv[q]);
                }
                herm6_mv_acc<R>(ww, mm + 36 * hs, lv);
#pragma unroll
                for (int q = 0; q < 6; ++q) w[6 * hs + q] = w[6 * hs + q] + ww[q];
            }
#pragma unroll
            for (int hr = 0; hr < 2; ++hr)
#pragma unroll
                for (int j = 0; j < NV; ++j) {
                    if (j < nv) {
                        cpx<R> t = C((R)0, (R)0);
#pragma unroll
                        for (int c = 0; c < 6; ++c)
                            cfma_cj(t, ldc<P>(b.Pm, p_index(m, 2 * k + hr, j, c, s)), w[6 * hr + c]);
                        acc[2 * (hr * NV + j)] += (double)t.re;
                        acc[2 * (hr * NV + j) + 1] += (double)t.im;
                    }
                }
        }
        block_sums<4 * NV>(acc, red, tot);
        if (threadIdx.x < n2) {
            const int hr = threadIdx.x / nv, j = threadIdx.x % nv;
            const long q = (((long)k * MG_NSLOT + d) * n2 + cs) * n2 + threadIdx.x;   // [k][slot][column][row]
            stc<P>(b.Mc, q, C((typename CE<P>::R)tot[2 * (hr * NV + j)], (typename CE<P>::R)tot[2 * (hr * NV + j) + 1]));
        }
    }
}

}  // namespace tmk

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
struct tm_mg {
    tm_ctx* c = nullptr;
    tm_mg_params p{};
    int P = P32;
    MgGeom m{};
    long nfine = 0;      // complex elements of a fine field
    long ncoarse = 0;    // complex elements of a coarse vector
    size_t fbytes = 0;   // bytes of a fine field
    long setup_gen = -1, setup_stamp = -1;
    bool ready = false;
    void* Pm = nullptr;
    void* Mc = nullptr;
    void* vecs = nullptr;                    // nvec smoothed near-null fields
    std::vector<void*> cvec;                 // coarse GCR: x, r, b, t, p[restart], ap[restart]
    void* fz = nullptr;                      // preconditioner fine temporaries
    void* frs = nullptr;
    void* fmr = nullptr;
    double* op_partial = nullptr;            // block partials of the fused minimal-residual dots
    MgCtl* ctl = nullptr;                    // [0] fine GCR, [1] coarse GCR, [2] minimal residual
    MgCtl* h_ctl = nullptr;
    double* partial = nullptr;
    unsigned int* counter = nullptr;
    cudaStream_t cap = nullptr;              // private stream for graph capture
    cudaGraphExec_t coarse_graph = nullptr;  // the whole coarse solve (restrict output -> x)
};

namespace {

enum { WS_MG_IN = 600, WS_MG_OUT, WS_MG_X64, WS_MG_B64, WS_MG_R64, WS_MG_T64, WS_MG_E, WS_MG_R, WS_MG_P = 650,
       WS_MG_AP = 700, WS_MG_CTL = 750 };

inline cudaStream_t Sx(void* s) { return reinterpret_cast<cudaStream_t>(s); }

bool dev_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t full_bytes(int P, long vh) { return 2 * spinor_bytes(P, 12, vh); }

// even-site A in storage precision P (lazily; odd A comes with tmk_ensure_prec)
tm_status ensure_full(tm_ctx* c, int P, cudaStream_t st) {
    MCKS(tmk_ensure_prec(c, P, st));
    if (P == P64) return TM_OK;
    if (c->clovAeP_stamp[P] != c->clover_stamp) {
        if (!c->clovAeP[P]) MCK(cudaMalloc(&c->clovAeP[P], (size_t)prec_esz(P) * CLOV_ODD_REALS * c->vh));
        MCK(launch_clover_from64<P32>(c->clovAeP[P], c->clovA64[0], c->vh, CLOV_ODD_REALS, st));
        c->clovAeP_stamp[P] = c->clover_stamp;
    }
    return TM_OK;
}

FullOp full_args(const tm_ctx* c, int P, int sign, void* out, const void* in, const MgCtl* gate) {
    FullOp a{};
    a.g = c->g;
    a.bc_t = (float)c->params.bc_t;
    a.kappa = c->params.kappa;
    a.tw = sign * 2.0 * c->params.kappa * c->params.mu;
    for (int p = 0; p < 2; ++p) a.gauge[p] = P == P64 ? c->gauge64[p] : c->gaugeP[P][p];
    a.A[0] = P == P64 ? (const void*)c->clovA64[0] : c->clovAeP[P];
    a.A[1] = P == P64 ? (const void*)c->clovA64[1] : c->clovAP[P];
    a.in = in;
    a.out = out;
    a.half = spinor_bytes(P, 12, c->vh);
    a.gate = gate;
    return a;
}

// blocks of the full-operator kernel
long full_op_blocks(const tm_ctx* c) { return (2 * c->vh + 127) / 128; }

// mr non-null: fuse the minimal-residual dots (partial: 3 doubles per block)
cudaError_t full_op(const tm_ctx* c, int P, int sign, void* out, const void* in, const MgCtl* gate, cudaStream_t st,
                    MgCtl* mr = nullptr, double* partial = nullptr, unsigned int* counter = nullptr) {
    FullOp a = full_args(c, P, sign, out, in, gate);
    a.mr = mr;
    a.partial = partial;
    a.counter = counter;
    const unsigned nb = (unsigned)((2 * c->vh + 127) / 128);
    if (P == P64) k_full_op<P64><<<nb, 128, 0, st>>>(a);
    else k_full_op<P32><<<nb, 128, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t full_import(const tm_ctx* c, int P, void* dst, const double* src, cudaStream_t st) {
    const unsigned nb = (unsigned)((2 * c->vh + MG_BS - 1) / MG_BS);
    const size_t half = spinor_bytes(P, 12, c->vh);
    if (P == P64) k_full_import<P64><<<nb, MG_BS, 0, st>>>(dst, src, c->g, half);
    else k_full_import<P32><<<nb, MG_BS, 0, st>>>(dst, src, c->g, half);
    return cudaGetLastError();
}

cudaError_t full_export(const tm_ctx* c, int P, double* dst, const void* src, cudaStream_t st) {
    const unsigned nb = (unsigned)((2 * c->vh + MG_BS - 1) / MG_BS);
    const size_t half = spinor_bytes(P, 12, c->vh);
    if (P == P64) k_full_export<P64><<<nb, MG_BS, 0, st>>>(dst, src, c->g, half);
    else k_full_export<P32><<<nb, MG_BS, 0, st>>>(dst, src, c->g, half);
    return cudaGetLastError();
}

// flat-vector kernels of precision P
template <int NP>
cudaError_t pairdots(int P, long n, int np, const void* const* u, const void* const* v, int fin, MgCtl* ctl,
                     const MgCtl* gate, double* partial, unsigned int* counter, cudaStream_t st) {
    PairDots<NP> a{};
    a.n = n;
    a.np = np;
    a.fin = fin;
    for (int q = 0; q < np; ++q) {
        a.u[q] = u[q];
        a.v[q] = v[q];
    }
    a.ctl = ctl;
    a.gate = gate;
    a.partial = partial;
    a.counter = counter;
    if (P == P64) k_pairdots<P64, NP><<<flat_grid(n), MG_BS, 0, st>>>(a);
    else k_pairdots<P32, NP><<<flat_grid(n), MG_BS, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t dots_any(int P, long n, int np, const void* const* u, const void* const* v, int fin, MgCtl* ctl,
                     const MgCtl* gate, double* partial, unsigned int* counter, cudaStream_t st) {
    if (np <= 2) return pairdots<2>(P, n, np, u, v, fin, ctl, gate, partial, counter, st);
    if (np <= 4) return pairdots<4>(P, n, np, u, v, fin, ctl, gate, partial, counter, st);
    if (np <= 8) return pairdots<8>(P, n, np, u, v, fin, ctl, gate, partial, counter, st);
    return pairdots<MG_MAX_RESTART>(P, n, np, u, v, fin, ctl, gate, partial, counter, st);
}

cudaError_t axpby(int P, long n, void* y, double ca, const void* x, double cw, const void* w, const MgCtl* gate,
                  cudaStream_t st) {
    if (P == P64) k_axpby<P64><<<flat_grid(n), MG_BS, 0, st>>>(n, y, ca, x, cw, w, gate);
    else k_axpby<P32><<<flat_grid(n), MG_BS, 0, st>>>(n, y, ca, x, cw, w, gate);
    return cudaGetLastError();
}

// ----- multigrid pieces -------------------------------------------------------
int nv_bucket(int nvec) { return nvec <= 4 ? 4 : nvec <= 8 ? 8 : nvec <= 12 ? 12 : 16; }

template <int P>
cudaError_t restrict_t(const tm_mg* g, void* coarse, const void* fine, const MgCtl* gate, cudaStream_t st) {
    k_mg_restrict<P><<<g->m.Nb, 64 * g->p.nvec, 0, st>>>(coarse, fine, g->Pm, g->m, gate);   // 2 nvec warps
    return cudaGetLastError();
}

cudaError_t mg_restrict(const tm_mg* g, void* coarse, const void* fine, const MgCtl* gate, cudaStream_t st) {
    return g->P == P64 ? restrict_t<P64>(g, coarse, fine, gate, st) : restrict_t<P32>(g, coarse, fine, gate, st);
}

cudaError_t mg_prolong(const tm_mg* g, void* fine, const void* coarse, const MgCtl* gate, cudaStream_t st) {
    const unsigned nb = (unsigned)(((long)g->m.Nb * g->m.Vb + MG_BS - 1) / MG_BS);
    if (g->P == P64) k_mg_prolong<P64><<<nb, MG_BS, 0, st>>>(fine, coarse, g->Pm, g->m, gate);
    else k_mg_prolong<P32><<<nb, MG_BS, 0, st>>>(fine, coarse, g->Pm, g->m, gate);
    return cudaGetLastError();
}

cudaError_t mg_coarse(const tm_mg* g, void* out, const void* in, const MgCtl* gate, cudaStream_t st) {
    const unsigned nb = (unsigned)((g->ncoarse + MG_BS - 1) / MG_BS);
    if (g->P == P64) k_mg_coarse<P64><<<nb, MG_BS, 0, st>>>(out, in, g->Mc, g->m, gate);
    else k_mg_coarse<P32><<<nb, MG_BS, 0, st>>>(out, in, g->Mc, g->m, gate);
    return cudaGetLastError();
}

template <int P>
cudaError_t build_t(const tm_mg* g, const BuildArgs& b, cudaStream_t st) {
    const int nb = nv_bucket(g->p.nvec);
    const int bs = g->m.Vb >= MG_BS ? MG_BS : ((g->m.Vb + 31) / 32) * 32;
    const dim3 grid(g->m.Nb, 2 * g->p.nvec);
    if (nb == 4) k_mg_build<P, 4><<<grid, bs, 0, st>>>(b);
    else if (nb == 8) k_mg_build<P, 8><<<grid, bs, 0, st>>>(b);
    else if (nb == 12) k_mg_build<P, 12><<<grid, bs, 0, st>>>(b);
    else k_mg_build<P, 16><<<grid, bs, 0, st>>>(b);
    return cudaGetLastError();
}

tm_status read_ctl(tm_mg* g, int level, cudaStream_t st) {
    MCK(cudaMemcpyAsync(g->h_ctl + level, g->ctl + level, sizeof(MgCtl), cudaMemcpyDeviceToHost, st));
    MCK(cudaStreamSynchronize(st));
    return TM_OK;
}

tm_status reset_ctl(tm_mg* g, int level, double stop_rr, int maxiter, cudaStream_t st) {
    MgCtl h{};
    h.stop_rr = stop_rr;
    h.maxiter = maxiter;
    h.flag = CTL_RUN;
    h.na = 1.0;
    g->h_ctl[level] = h;
    MCK(cudaMemcpyAsync(g->ctl + level, g->h_ctl + level, sizeof(MgCtl), cudaMemcpyHostToDevice, st));
    return TM_OK;
}

// Operator of one GCR level
struct Level {
    long n;
    int P;
    MgCtl* ctl;
    // y = A x
    virtual tm_status apply(void* y, const void* x, cudaStream_t st) = 0;
    // z = K r (preconditioner); default: copy
    virtual tm_status precond(void* z, const void* r, cudaStream_t st) {
        MCK(axpby(P, n, z, 1.0, r, 0.0, nullptr, ctl, st));
        return TM_OK;
    }
    virtual ~Level() {}
};

struct GcrWork {
    void* x;
    void* r;
    void* b;
    void* t;
    void* p[MG_MAX_RESTART];
    void* ap[MG_MAX_RESTART];
};

// Restarted GCR on A x = b from x = 0 (the oracle's gcr): every iteration
// preconditions the residual, orthogonalises A z against the stored directions,
// normalises and updates x and r; each restart recomputes r = b - A x.  Stops
// when ||r||^2 < stop_rr or after maxiter iterations.  check_each: read the
// control word after every iteration (levels whose preconditioner does its own
// work), else once per restart cycle.  Returns the final control word in
// g->h_ctl[level].
tm_status gcr_run(tm_mg* g, Level& L, int level, GcrWork& w, int restart, double stop_rr, int maxiter,
                  bool check_each, cudaStream_t st) {
    const long n = L.n;
    const int P = L.P;
    MgCtl* ctl = g->ctl + level;
    MCKS(reset_ctl(g, level, stop_rr, maxiter, st));
    MCK(axpby(P, n, w.x, 0.0, nullptr, 0.0, nullptr, nullptr, st));
    MCK(axpby(P, n, w.r, 1.0, w.b, 0.0, nullptr, nullptr, st));
    {
        const void* u[1] = {w.r};
        MCK(dots_any(P, n, 1, u, u, MGF_RR0, ctl, nullptr, g->partial, g->counter, st));
    }
    MCKS(read_ctl(g, level, st));
    if (g->h_ctl[level].flag != CTL_RUN) return TM_OK;
    for (;;) {
        for (int i = 0; i < restart; ++i) {
            MCKS(L.precond(w.p[i], w.r, st));
            MCKS(L.apply(w.ap[i], w.p[i], st));
            if (i > 0) {
                const void* u[MG_MAX_RESTART];
                const void* v[MG_MAX_RESTART];
                PtrList pl{}, al{};
                for (int j = 0; j < i; ++j) {
                    u[j] = w.ap[j];
                    v[j] = w.ap[i];
                    pl.q[j] = w.p[j];
                    al.q[j] = w.ap[j];
                }
                MCK(dots_any(P, n, i, u, v, MGF_DOTS, ctl, ctl, g->partial, g->counter, st));
                if (P == P64) k_gcr_orth<P64><<<flat_grid(n), MG_BS, 0, st>>>(n, i, w.p[i], w.ap[i], pl, al, ctl);
                else k_gcr_orth<P32><<<flat_grid(n), MG_BS, 0, st>>>(n, i, w.p[i], w.ap[i], pl, al, ctl);
                MCK(cudaGetLastError());
            }
            const void* u[2] = {w.ap[i], w.ap[i]};
            const void* v[2] = {w.ap[i], w.r};
            MCK(dots_any(P, n, 2, u, v, MGF_GCR, ctl, ctl, g->partial, g->counter, st));
            if (P == P64)
                k_gcr_update<P64><<<flat_grid(n), MG_BS, 0, st>>>(n, w.p[i], w.ap[i], w.x, w.r, ctl, g->partial, g->counter);
            else
                k_gcr_update<P32><<<flat_grid(n), MG_BS, 0, st>>>(n, w.p[i], w.ap[i], w.x, w.r, ctl, g->partial, g->counter);
            MCK(cudaGetLastError());
            if (check_each) {
                MCKS(read_ctl(g, level, st));
                if (g->h_ctl[level].flag != CTL_RUN) return TM_OK;
            }
        }
        MCKS(read_ctl(g, level, st));
        if (g->h_ctl[level].flag != CTL_RUN) return TM_OK;
        // restart from the true residual
        MCKS(L.apply(w.t, w.x, st));
        MCK(axpby(P, n, w.r, 1.0, w.b, -1.0, w.t, ctl, st));
        const void* u[1] = {w.r};
        MCK(dots_any(P, n, 1, u, u, MGF_RR0, ctl, ctl, g->partial, g->counter, st));
    }
}

// minimal-residual steps on M z = r from the given z (the oracle's minimal_residual)
tm_status mr_steps(tm_mg* g, void* z, const void* r, int steps, cudaStream_t st) {
    tm_ctx* c = g->c;
    const int P = g->P;
    const long n = g->nfine;
    MgCtl* ctl = g->ctl + 2;
    MCK(full_op(c, P, g->p.sign, g->fmr, z, nullptr, st));
    MCK(axpby(P, n, g->frs, 1.0, r, -1.0, g->fmr, nullptr, st));
    for (int k = 0; k < steps; ++k) {
        // mr = M r with <mr, r> and <mr, mr> reduced in the same kernel (alpha in ctl)
        MCK(full_op(c, P, g->p.sign, g->fmr, g->frs, nullptr, st, ctl, g->op_partial, g->counter));
        if (P == P64) k_mr_update<P64><<<flat_grid(n), MG_BS, 0, st>>>(n, z, g->frs, g->fmr, ctl);
        else k_mr_update<P32><<<flat_grid(n), MG_BS, 0, st>>>(n, z, g->frs, g->fmr, ctl);
        MCK(cudaGetLastError());
    }
    return TM_OK;
}

// z = P M_c^-1 P^+ r (coarse GCR to coarse_tol), then smooth_steps MR steps
// The coarse solve is launch-bound (kernels of a few microseconds on vectors of
// ~1e6 complex entries), so the whole of it is one CUDA graph: control word
// reset, x = 0, r = b, ||b||^2 (stop threshold set on the device), then
// ceil(coarse_maxiter / restart) restart cycles of GCR iterations and true
// residuals.  Every kernel is gated on the coarse control word, so the
// iterations after convergence or the iteration bound exit at entry.  Captured
// once per hierarchy on its private stream; its vectors are the hierarchy's own.
tm_status coarse_graph(tm_mg* g) {
    if (g->coarse_graph) return TM_OK;
    const int P = g->P;
    const long n = g->ncoarse;
    const int R = g->p.coarse_restart;
    const int ncyc = (g->p.coarse_maxiter + R - 1) / R;
    MgCtl* ctl = g->ctl + 1;
    GcrWork w{};
    w.x = g->cvec[0];
    w.r = g->cvec[1];
    w.b = g->cvec[2];
    w.t = g->cvec[3];
    for (int i = 0; i < R; ++i) {
        w.p[i] = g->cvec[4 + i];
        w.ap[i] = g->cvec[4 + R + i];
    }
    const cudaStream_t st = g->cap;
    cudaGraph_t graph = nullptr;
    MCK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    auto body = [&]() -> cudaError_t {
        k_ctl_start<<<1, 1, 0, st>>>(ctl, g->p.coarse_maxiter, g->p.coarse_tol * g->p.coarse_tol);
        cudaError_t e = cudaGetLastError();
        if (!e) e = axpby(P, n, w.x, 0.0, nullptr, 0.0, nullptr, nullptr, st);
        if (!e) e = axpby(P, n, w.r, 1.0, w.b, 0.0, nullptr, nullptr, st);
        const void* ub[1] = {w.r};
        if (!e) e = dots_any(P, n, 1, ub, ub, MGF_RRB, ctl, nullptr, g->partial, g->counter, st);
        for (int cyc = 0; cyc < ncyc && !e; ++cyc) {
            for (int i = 0; i < R && !e; ++i) {
                e = axpby(P, n, w.p[i], 1.0, w.r, 0.0, nullptr, ctl, st);   // no coarse preconditioner
                if (!e) e = mg_coarse(g, w.ap[i], w.p[i], ctl, st);
                if (i > 0 && !e) {
                    const void* u[MG_MAX_RESTART];
                    const void* v[MG_MAX_RESTART];
                    PtrList pl{}, al{};
                    for (int j = 0; j < i; ++j) {
                        u[j] = w.ap[j];
                        v[j] = w.ap[i];
                        pl.q[j] = w.p[j];
                        al.q[j] = w.ap[j];
                    }
                    e = dots_any(P, n, i, u, v, MGF_DOTS, ctl, ctl, g->partial, g->counter, st);
                    if (!e) {
                        if (P == P64) k_gcr_orth<P64><<<flat_grid(n), MG_BS, 0, st>>>(n, i, w.p[i], w.ap[i], pl, al, ctl);
                        else k_gcr_orth<P32><<<flat_grid(n), MG_BS, 0, st>>>(n, i, w.p[i], w.ap[i], pl, al, ctl);
                        e = cudaGetLastError();
                    }
                }
                const void* u2[2] = {w.ap[i], w.ap[i]};
                const void* v2[2] = {w.ap[i], w.r};
                if (!e) e = dots_any(P, n, 2, u2, v2, MGF_GCR, ctl, ctl, g->partial, g->counter, st);
                if (!e) {
                    if (P == P64)
                        k_gcr_update<P64><<<flat_grid(n), MG_BS, 0, st>>>(n, w.p[i], w.ap[i], w.x, w.r, ctl, g->partial, g->counter);
                    else
                        k_gcr_update<P32><<<flat_grid(n), MG_BS, 0, st>>>(n, w.p[i], w.ap[i], w.x, w.r, ctl, g->partial, g->counter);
                    e = cudaGetLastError();
                }
            }
            if (cyc + 1 < ncyc && !e) {   // restart from the true residual
                e = mg_coarse(g, w.t, w.x, ctl, st);
                if (!e) e = axpby(P, n, w.r, 1.0, w.b, -1.0, w.t, ctl, st);
                const void* u[1] = {w.r};
                if (!e) e = dots_any(P, n, 1, u, u, MGF_RR0, ctl, ctl, g->partial, g->counter, st);
            }
        }
        return e;
    };
    const cudaError_t e = body();
    const cudaError_t e2 = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        return tmk_failf(TM_ERR_CUDA, "multigrid: capture of the coarse solve: %s",
                         cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    const cudaError_t e3 = cudaGraphInstantiate(&g->coarse_graph, graph, 0);
    cudaGraphDestroy(graph);
    if (e3 != cudaSuccess) {
        g->coarse_graph = nullptr;
        return tmk_failf(TM_ERR_CUDA, "multigrid: coarse graph: %s", cudaGetErrorString(e3));
    }
    return TM_OK;
}

// z = P M_c^-1 P^+ r (coarse GCR to coarse_tol), then smooth_steps MR steps
tm_status mg_apply(tm_mg* g, void* z, const void* r, cudaStream_t st) {
    MCKS(coarse_graph(g));
    MCK(mg_restrict(g, g->cvec[2], r, nullptr, st));
    MCK(cudaGraphLaunch(g->coarse_graph, st));
    MCK(mg_prolong(g, z, g->cvec[0], nullptr, st));
    if (g->p.smooth_steps > 0) MCKS(mr_steps(g, z, r, g->p.smooth_steps, st));
    return TM_OK;
}

struct FineLevel : Level {
    tm_mg* g = nullptr;   // preconditioner (null: none)
    tm_ctx* c = nullptr;
    int sign = 1;
    tm_status apply(void* y, const void* x, cudaStream_t st) override {
        MCK(full_op(c, P, sign, y, x, ctl, st));
        return TM_OK;
    }
    tm_status precond(void* z, const void* r, cudaStream_t st) override {
        if (!g) return Level::precond(z, r, st);
        return mg_apply(g, z, r, st);
    }
};

tm_status check_mg_ready(tm_mg* g) {
    if (!g->ready) return tmk_failf(TM_ERR_ARG, "multigrid: tm_mg_setup has not run");
    if (g->c->gauge_gen != g->setup_gen || g->c->clover_stamp != g->setup_stamp)
        return tmk_failf(TM_ERR_STALE, "multigrid: the gauge field or clover term changed since tm_mg_setup");
    return TM_OK;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" tm_status tm_apply_full(tm_ctx* c, int sign, tm_prec prec, double* out, const double* in, void* stream) {
    if (!c || !out || !in || (sign != 1 && sign != -1)) return tmk_failf(TM_ERR_ARG, "tm_apply_full: bad argument");
    if (prec != TM_F64 && prec != TM_F32) return tmk_failf(TM_ERR_ARG, "tm_apply_full: precision must be TM_F64 or TM_F32");
    if (((uintptr_t)out & 15) || ((uintptr_t)in & 15)) return tmk_failf(TM_ERR_ARG, "tm_apply_full: misaligned pointer");
    MCK(cudaSetDevice(c->device));
    if (!dev_ptr(out) || !dev_ptr(in)) return tmk_failf(TM_ERR_ARG, "tm_apply_full: fields must be device pointers");
    const cudaStream_t st = Sx(stream);
    MCKS(ensure_full(c, prec, st));
    void *a, *b;
    MCKS(tmk_ws_get(c, WS_MG_IN, full_bytes(prec, c->vh), &a));
    MCKS(tmk_ws_get(c, WS_MG_OUT, full_bytes(prec, c->vh), &b));
    MCK(full_import(c, prec, a, in, st));
    MCK(full_op(c, prec, sign, b, a, nullptr, st));
    MCK(full_export(c, prec, out, b, st));
    return TM_OK;
}

extern "C" tm_status tm_mg_create(tm_mg** out, tm_ctx* c, const tm_mg_params* p) {
    if (!out || !c || !p) return tmk_failf(TM_ERR_ARG, "tm_mg_create: null argument");
    const int L[4] = {c->g.X, c->g.Y, c->g.Z, c->g.T};
    int Vb = 1;
    for (int d = 0; d < 4; ++d) {
        if (p->block[d] < 1 || L[d] % p->block[d])
            return tmk_failf(TM_ERR_ARG, "tm_mg_create: block extent %d = %d must divide the lattice extent %d", d,
                             p->block[d], L[d]);
        Vb *= p->block[d];
    }
    if (p->nvec < 1 || p->nvec > MG_MAX_NVEC || p->nvec > 6 * Vb)
        return tmk_failf(TM_ERR_ARG, "tm_mg_create: need 1 <= nvec <= %d and nvec <= 6 x block volume", MG_MAX_NVEC);
    if (p->prec != TM_F64 && p->prec != TM_F32) return tmk_failf(TM_ERR_ARG, "tm_mg_create: prec must be TM_F64 or TM_F32");
    if (p->sign != 1 && p->sign != -1) return tmk_failf(TM_ERR_ARG, "tm_mg_create: sign must be +1 or -1");
    if (p->coarse_restart < 1 || p->coarse_restart > MG_MAX_RESTART || p->coarse_maxiter < 1 || !(p->coarse_tol > 0.0) ||
        p->setup_steps < 0 || p->smooth_steps < 0)
        return tmk_failf(TM_ERR_ARG, "tm_mg_create: bad solver parameters");
    MCK(cudaSetDevice(c->device));
    tm_mg* g = new tm_mg();
    g->c = c;
    g->p = *p;
    g->P = p->prec == TM_F64 ? P64 : P32;
    g->m.g = c->g;
    for (int d = 0; d < 4; ++d) {
        g->m.B[d] = p->block[d];
        g->m.nb[d] = L[d] / p->block[d];
    }
    g->m.Vb = Vb;
    g->m.Nb = (int)(2 * c->vh / Vb);
    g->m.nvec = p->nvec;
    g->m.half = spinor_bytes(g->P, 12, c->vh);
    g->nfine = 24 * c->vh;
    g->ncoarse = (long)g->m.Nb * 2 * p->nvec;
    g->fbytes = full_bytes(g->P, c->vh);
    const size_t ce = g->P == P64 ? 16 : 8;
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaMalloc(&g->Pm, ce * (size_t)g->nfine * p->nvec);   // 12 V nvec complex
    e = e ? e : cudaMalloc(&g->Mc, ce * (size_t)g->m.Nb * MG_NSLOT * 4 * p->nvec * p->nvec);
    e = e ? e : cudaMalloc(&g->vecs, g->fbytes * p->nvec);
    g->cvec.assign(4 + 2 * p->coarse_restart, nullptr);
    for (auto& v : g->cvec) e = e ? e : cudaMalloc(&v, ce * g->ncoarse);
    e = e ? e : cudaMalloc(&g->fz, g->fbytes);
    e = e ? e : cudaMalloc(&g->frs, g->fbytes);
    e = e ? e : cudaMalloc(&g->fmr, g->fbytes);
    e = e ? e : cudaMalloc(&g->ctl, 3 * sizeof(MgCtl));
    e = e ? e : cudaMallocHost(&g->h_ctl, 3 * sizeof(MgCtl));
    e = e ? e : cudaMalloc(&g->partial, sizeof(double) * MG_GRID_CAP * MG_PART_W);
    e = e ? e : cudaMalloc(&g->op_partial, sizeof(double) * 3 * full_op_blocks(c));
    e = e ? e : cudaMalloc(&g->counter, sizeof(unsigned int));
    e = e ? e : cudaMemset(g->counter, 0, sizeof(unsigned int));
    e = e ? e : cudaMemset(g->ctl, 0, 3 * sizeof(MgCtl));
    e = e ? e : cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        tm_mg_destroy(g);
        return tmk_failf(e == cudaErrorMemoryAllocation ? TM_ERR_OOM : TM_ERR_CUDA, "tm_mg_create: %s",
                         cudaGetErrorString(e));
    }
    *out = g;
    return TM_OK;
}

extern "C" tm_status tm_mg_destroy(tm_mg* g) {
    if (!g) return TM_OK;
    cudaSetDevice(g->c->device);
    cudaDeviceSynchronize();
    cudaFree(g->Pm);
    cudaFree(g->Mc);
    cudaFree(g->vecs);
    for (void* v : g->cvec) cudaFree(v);
    cudaFree(g->fz);
    cudaFree(g->frs);
    cudaFree(g->fmr);
    cudaFree(g->ctl);
    cudaFreeHost(g->h_ctl);
    if (g->coarse_graph) cudaGraphExecDestroy(g->coarse_graph);
    if (g->cap) cudaStreamDestroy(g->cap);
    cudaFree(g->partial);
    cudaFree(g->op_partial);
    cudaFree(g->counter);
    delete g;
    return TM_OK;
}

extern "C" tm_status tm_mg_coarse_size(const tm_mg* g, size_t* n) {
    if (!g || !n) return tmk_failf(TM_ERR_ARG, "tm_mg_coarse_size: null argument");
    *n = (size_t)g->ncoarse;
    return TM_OK;
}

extern "C" tm_status tm_mg_setup(tm_mg* g, const double* init, void* stream) {
    if (!g || !init) return tmk_failf(TM_ERR_ARG, "tm_mg_setup: null argument");
    tm_ctx* c = g->c;
    MCK(cudaSetDevice(c->device));
    if (!dev_ptr(init)) return tmk_failf(TM_ERR_ARG, "tm_mg_setup: init must be a device pointer");
    const cudaStream_t st = Sx(stream);
    MCKS(ensure_full(c, g->P, st));
    const int P = g->P;
    const long n = g->nfine;
    const size_t canon = (size_t)2 * c->vh * 24;   // doubles per canonical full field
    // near-null vectors: x = v, r = -M v, setup_steps MR steps on M x = 0, normalise
    for (int j = 0; j < g->p.nvec; ++j) {
        void* x = reinterpret_cast<char*>(g->vecs) + (size_t)j * g->fbytes;
        MCK(full_import(c, P, x, init + (size_t)j * canon, st));
        MCK(axpby(P, n, g->frs, 0.0, nullptr, 0.0, nullptr, nullptr, st));   // b = 0
        MCK(axpby(P, n, g->fz, 0.0, nullptr, 0.0, nullptr, nullptr, st));
        MCKS(mr_steps(g, x, g->fz, g->p.setup_steps, st));
        const void* u[1] = {x};
        MCK(dots_any(P, n, 1, u, u, MGF_NRM, g->ctl + 2, nullptr, g->partial, g->counter, st));
        if (P == P64) k_normalize<P64><<<flat_grid(n), MG_BS, 0, st>>>(n, x, g->ctl + 2);
        else k_normalize<P32><<<flat_grid(n), MG_BS, 0, st>>>(n, x, g->ctl + 2);
        MCK(cudaGetLastError());
    }
    // prolongator
    const unsigned nbs = (unsigned)(((long)g->m.Nb * g->m.Vb + MG_BS - 1) / MG_BS);
    if (P == P64) {
        k_mg_gather<P64><<<nbs, MG_BS, 0, st>>>(g->Pm, g->vecs, g->fbytes, g->m);
        k_mg_orth<P64><<<2 * g->m.Nb, MG_BS, 0, st>>>(g->Pm, g->m);
    } else {
        k_mg_gather<P32><<<nbs, MG_BS, 0, st>>>(g->Pm, g->vecs, g->fbytes, g->m);
        k_mg_orth<P32><<<2 * g->m.Nb, MG_BS, 0, st>>>(g->Pm, g->m);
    }
    MCK(cudaGetLastError());
    // Galerkin coarse operator
    BuildArgs b{};
    b.m = g->m;
    const FullOp fa = full_args(c, P, g->p.sign, nullptr, nullptr, nullptr);
    b.bc_t = fa.bc_t;
    b.kappa = fa.kappa;
    b.tw = fa.tw;
    for (int q = 0; q < 2; ++q) {
        b.gauge[q] = fa.gauge[q];
        b.A[q] = fa.A[q];
    }
    b.Pm = g->Pm;
    b.Mc = g->Mc;
    MCK(P == P64 ? build_t<P64>(g, b, st) : build_t<P32>(g, b, st));
    MCK(cudaStreamSynchronize(st));
    g->setup_gen = c->gauge_gen;
    g->setup_stamp = c->clover_stamp;
    g->ready = true;
    return TM_OK;
}

// the smoothed, normalised near-null vectors as canonical full FP64 fields (device)
extern "C" tm_status tm_mg_vectors(tm_mg* g, double* out, void* stream) {
    if (!g || !out) return tmk_failf(TM_ERR_ARG, "tm_mg_vectors: null argument");
    MCKS(check_mg_ready(g));
    MCK(cudaSetDevice(g->c->device));
    if (!dev_ptr(out)) return tmk_failf(TM_ERR_ARG, "tm_mg_vectors: out must be a device pointer");
    const size_t canon = (size_t)2 * g->c->vh * 24;
    for (int j = 0; j < g->p.nvec; ++j)
        MCK(full_export(g->c, g->P, out + j * canon, reinterpret_cast<const char*>(g->vecs) + (size_t)j * g->fbytes,
                        Sx(stream)));
    return TM_OK;
}

// coarse vectors of the C ABI are complex FP64; in FP32 mode they are converted
static tm_status coarse_in(tm_mg* g, void* dst, const double* src, cudaStream_t st) {
    if (g->P == P64) MCK(cudaMemcpyAsync(dst, src, 16 * (size_t)g->ncoarse, cudaMemcpyDeviceToDevice, st));
    else {
        k_convert<P32, P64><<<flat_grid(g->ncoarse), MG_BS, 0, st>>>(g->ncoarse, dst, src, 1.0);
        MCK(cudaGetLastError());
    }
    return TM_OK;
}
static tm_status coarse_out(tm_mg* g, double* dst, const void* src, cudaStream_t st) {
    if (g->P == P64) MCK(cudaMemcpyAsync(dst, src, 16 * (size_t)g->ncoarse, cudaMemcpyDeviceToDevice, st));
    else {
        k_convert<P64, P32><<<flat_grid(g->ncoarse), MG_BS, 0, st>>>(g->ncoarse, dst, src, 1.0);
        MCK(cudaGetLastError());
    }
    return TM_OK;
}

static tm_status mg_io_check(tm_mg* g, const void* a, const void* b, const char* who) {
    if (!g || !a || !b) return tmk_failf(TM_ERR_ARG, "%s: null argument", who);
    MCKS(check_mg_ready(g));
    MCK(cudaSetDevice(g->c->device));
    if (!dev_ptr(a) || !dev_ptr(b)) return tmk_failf(TM_ERR_ARG, "%s: vectors must be device pointers", who);
    if (((uintptr_t)a & 15) || ((uintptr_t)b & 15)) return tmk_failf(TM_ERR_ARG, "%s: misaligned pointer", who);
    return TM_OK;
}

extern "C" tm_status tm_mg_prolong(tm_mg* g, double* fine, const double* coarse, void* stream) {
    MCKS(mg_io_check(g, fine, coarse, "tm_mg_prolong"));
    const cudaStream_t st = Sx(stream);
    MCKS(coarse_in(g, g->cvec[0], coarse, st));
    MCK(mg_prolong(g, g->fz, g->cvec[0], nullptr, st));
    MCK(full_export(g->c, g->P, fine, g->fz, st));
    return TM_OK;
}

extern "C" tm_status tm_mg_restrict(tm_mg* g, double* coarse, const double* fine, void* stream) {
    MCKS(mg_io_check(g, coarse, fine, "tm_mg_restrict"));
    const cudaStream_t st = Sx(stream);
    MCK(full_import(g->c, g->P, g->fz, fine, st));
    MCK(mg_restrict(g, g->cvec[0], g->fz, nullptr, st));
    MCKS(coarse_out(g, coarse, g->cvec[0], st));
    return TM_OK;
}

extern "C" tm_status tm_mg_coarse_apply(tm_mg* g, double* out, const double* in, void* stream) {
    MCKS(mg_io_check(g, out, in, "tm_mg_coarse_apply"));
    const cudaStream_t st = Sx(stream);
    MCKS(coarse_in(g, g->cvec[0], in, st));
    MCK(mg_coarse(g, g->cvec[1], g->cvec[0], nullptr, st));
    MCKS(coarse_out(g, out, g->cvec[1], st));
    return TM_OK;
}

extern "C" tm_status tm_mg_precondition(tm_mg* g, double* z, const double* r, int* coarse_iters, void* stream) {
    MCKS(mg_io_check(g, z, r, "tm_mg_precondition"));
    const cudaStream_t st = Sx(stream);
    void* rn;
    MCKS(tmk_ws_get(g->c, WS_MG_IN, g->fbytes, &rn));
    MCK(full_import(g->c, g->P, rn, r, st));
    MCKS(mg_apply(g, g->fz, rn, st));
    MCK(full_export(g->c, g->P, z, g->fz, st));
    MCKS(read_ctl(g, 1, st));
    if (coarse_iters) *coarse_iters = g->h_ctl[1].iter;
    return TM_OK;
}

// Solve M(sign) x = b to FP64 true relative residual sp->tol.  Outer loop in FP64:
// r = b - M x with the FP64 operator; if not converged, the inner flexible GCR
// (precision of mg, or sp->sloppy without mg) solves M e = r / ||r|| to relative
// residual inner_tol, and x += ||r|| e.  FP64 inner solves aim straight at the
// target.
extern "C" tm_status tm_solve_gcr(tm_ctx* c, int sign, tm_mg* g, const tm_solve_params* sp, double* x,
                                  const double* b, tm_solve_info* info, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!c || !sp || !x || !b || !info || (sign != 1 && sign != -1)) return tmk_failf(TM_ERR_ARG, "tm_solve_gcr: bad argument");
    if (!(sp->tol > 0.0) || sp->maxiter < 1) return tmk_failf(TM_ERR_ARG, "tm_solve_gcr: need tol > 0, maxiter >= 1");
    const int restart = sp->chunk > 0 ? sp->chunk : 8;
    if (restart > MG_MAX_RESTART) return tmk_failf(TM_ERR_ARG, "tm_solve_gcr: restart (chunk) at most %d", MG_MAX_RESTART);
    if (g && (g->c != c || g->p.sign != sign))
        return tmk_failf(TM_ERR_ARG, "tm_solve_gcr: the multigrid belongs to another context or sign");
    const int P = g ? g->P : (sp->sloppy == TM_F64 ? P64 : P32);
    if (!g && sp->sloppy != TM_F64 && sp->sloppy != TM_F32)
        return tmk_failf(TM_ERR_ARG, "tm_solve_gcr: sloppy precision must be TM_F64 or TM_F32");
    if (g) MCKS(check_mg_ready(g));
    MCK(cudaSetDevice(c->device));
    if (!dev_ptr(x) || !dev_ptr(b)) return tmk_failf(TM_ERR_ARG, "tm_solve_gcr: x and b must be device pointers");
    *info = tm_solve_info{};
    const cudaStream_t st = Sx(stream);
    MCKS(ensure_full(c, P64, st));
    MCKS(ensure_full(c, P, st));
    tm_mg* gw = g;
    tm_mg scratch;   // control words and reduction scratch when no multigrid is given
    if (!gw) {
        gw = &scratch;
        gw->c = c;
        gw->P = P;
        MCKS(tmk_ws_get(c, WS_MG_CTL, 3 * sizeof(MgCtl), reinterpret_cast<void**>(&gw->ctl)));
        MCKS(tmk_ws_get(c, WS_MG_CTL + 1, sizeof(double) * MG_GRID_CAP * MG_PART_W, reinterpret_cast<void**>(&gw->partial)));
        MCKS(tmk_ws_get(c, WS_MG_CTL + 2, sizeof(unsigned int), reinterpret_cast<void**>(&gw->counter)));
        MCK(cudaMemsetAsync(gw->counter, 0, sizeof(unsigned int), st));
        MCK(cudaMallocHost(&gw->h_ctl, 3 * sizeof(MgCtl)));
    }
    struct HostFree {
        tm_mg* s;
        bool own;
        ~HostFree() { if (own && s->h_ctl) cudaFreeHost(s->h_ctl); s->h_ctl = nullptr; }
    } hf{&scratch, gw == &scratch};
    const long n = 24 * c->vh;
    const size_t b64 = full_bytes(P64, c->vh), bp = full_bytes(P, c->vh);
    void *x64, *bb64, *r64, *t64;
    MCKS(tmk_ws_get(c, WS_MG_X64, b64, &x64));
    MCKS(tmk_ws_get(c, WS_MG_B64, b64, &bb64));
    MCKS(tmk_ws_get(c, WS_MG_R64, b64, &r64));
    MCKS(tmk_ws_get(c, WS_MG_T64, b64, &t64));
    GcrWork w{};
    MCKS(tmk_ws_get(c, WS_MG_E, bp, &w.x));
    MCKS(tmk_ws_get(c, WS_MG_R, bp, &w.r));
    MCKS(tmk_ws_get(c, WS_MG_E + 20, bp, &w.b));
    MCKS(tmk_ws_get(c, WS_MG_E + 21, bp, &w.t));
    for (int i = 0; i < restart; ++i) {
        MCKS(tmk_ws_get(c, WS_MG_P + i, bp, &w.p[i]));
        MCKS(tmk_ws_get(c, WS_MG_AP + i, bp, &w.ap[i]));
    }
    MCK(full_import(c, P64, x64, x, st));
    MCK(full_import(c, P64, bb64, b, st));
    const void* ub[1] = {bb64};
    MCK(dots_any(P64, n, 1, ub, ub, MGF_NRM, gw->ctl + 2, nullptr, gw->partial, gw->counter, st));
    MCKS(read_ctl(gw, 2, st));
    const double bnorm2 = gw->h_ctl[2].nrm2;
    if (!(bnorm2 > 0.0) || !std::isfinite(bnorm2)) {
        info->status = std::isfinite(bnorm2) ? TM_OK : TM_ERR_BREAKDOWN;
        if (bnorm2 == 0.0) {
            MCK(cudaMemsetAsync(x, 0, (size_t)n * 16, st));
            MCK(cudaStreamSynchronize(st));
        }
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        return info->status == TM_OK ? TM_OK : tmk_failf(TM_ERR_BREAKDOWN, "tm_solve_gcr: b is not finite");
    }
    FineLevel L;
    L.g = g;
    L.c = c;
    L.sign = sign;
    L.n = n;
    L.P = P;
    L.ctl = gw->ctl;
    const double inner_tol = P == P64 ? 0.0 : (sp->delta > 0.0 ? sp->delta : 1e-5);
    tm_status status = TM_ERR_NOT_CONVERGED;
    double rr = 0.0;
    for (int cycle = 0; cycle < 200; ++cycle) {
        MCK(full_op(c, P64, sign, t64, x64, nullptr, st));
        MCK(axpby(P64, n, r64, 1.0, bb64, -1.0, t64, nullptr, st));
        const void* u[1] = {r64};
        MCK(dots_any(P64, n, 1, u, u, MGF_NRM, gw->ctl + 2, nullptr, gw->partial, gw->counter, st));
        MCKS(read_ctl(gw, 2, st));
        rr = gw->h_ctl[2].nrm2;
        if (!std::isfinite(rr)) { status = TM_ERR_BREAKDOWN; break; }
        if (rr <= sp->tol * sp->tol * bnorm2) { status = TM_OK; break; }
        if (info->iters >= sp->maxiter) break;
        info->reliable_updates += 1;
        const double rn = std::sqrt(rr);
        if (P == P64) {
            MCK(axpby(P64, n, w.b, 1.0 / rn, r64, 0.0, nullptr, nullptr, st));
        } else {
            k_full_convert<P32, P64><<<(unsigned)((2 * c->vh + MG_BS - 1) / MG_BS), MG_BS, 0, st>>>(
                w.b, r64, c->vh, spinor_bytes(P32, 12, c->vh), spinor_bytes(P64, 12, c->vh), 1.0 / rn);
            MCK(cudaGetLastError());
        }
        // inner target: relative inner_tol (FP32) or the outer target itself (FP64)
        const double itol = P == P64 ? 0.9 * sp->tol * std::sqrt(bnorm2) / rn : inner_tol;
        MCKS(gcr_run(gw, L, 0, w, restart, itol * itol, sp->maxiter - info->iters, true, st));
        info->iters += gw->h_ctl[0].iter;
        if (gw->h_ctl[0].flag == CTL_BREAKDOWN) { status = TM_ERR_BREAKDOWN; break; }
        if (P == P64) {
            MCK(axpby(P64, n, x64, 1.0, x64, rn, w.x, nullptr, st));
        } else {
            k_full_add64<P32><<<(unsigned)((2 * c->vh + MG_BS - 1) / MG_BS), MG_BS, 0, st>>>(
                x64, w.x, c->vh, spinor_bytes(P32, 12, c->vh), rn);
            MCK(cudaGetLastError());
        }
    }
    MCK(full_export(c, P64, x, x64, st));
    MCK(cudaStreamSynchronize(st));
    info->true_rel_res = std::sqrt(rr / bnorm2);
    info->status = status;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (status != TM_OK)
        return tmk_failf(status, "tm_solve_gcr: %s", status == TM_ERR_BREAKDOWN ? "breakdown" : "not converged");
    return TM_OK;
}
