// Internal types shared by the library's translation units: complex arithmetic,
// storage-precision traits, native field layouts, problem descriptors for the
// batched kernels, and solver control words.
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/tm.h"
#include "fastdiv.h"
#include "df64.h"

namespace tmk {

// ---------------------------------------------------------------------------
// complex
// ---------------------------------------------------------------------------
template <typename R>
struct cpx {
    R re, im;
};

template <typename R> __host__ __device__ __forceinline__ cpx<R> C(R a, R b) { return cpx<R>{a, b}; }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator-(cpx<R> a) { return {-a.re, -a.im}; }
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __host__ __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> __host__ __device__ __forceinline__ cpx<R> cj(cpx<R> a) { return {a.re, -a.im}; }
template <typename R> __host__ __device__ __forceinline__ cpx<R> mul_i(cpx<R> a) { return {-a.im, a.re}; }   // i*a
// a += b*c
template <typename R> __host__ __device__ __forceinline__ void cfma(cpx<R>& a, cpx<R> b, cpx<R> c) {
    a.re = fma(b.re, c.re, a.re); a.re = fma(-b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im); a.im = fma(b.im, c.re, a.im);
}
// a += conj(b)*c
template <typename R> __host__ __device__ __forceinline__ void cfma_cj(cpx<R>& a, cpx<R> b, cpx<R> c) {
    a.re = fma(b.re, c.re, a.re); a.re = fma(b.im, c.im, a.re);
    a.im = fma(b.re, c.im, a.im); a.im = fma(-b.im, c.re, a.im);
}
template <typename R> __host__ __device__ __forceinline__ R norm2(cpx<R> a) { return a.re * a.re + a.im * a.im; }

// ---------------------------------------------------------------------------
// storage precisions and native layouts
//
// Every native array is a structure of arrays over the Vh sites of one parity:
// element (vector v, site i) lives at v*Vh + i, a vector holding W reals
// (W = 2 for FP64 double2, 4 for FP32 float4, 8 for 16-bit uint4).
//   spinor (nc complex per site: 12 light, 24 heavy): vectors 0 .. 2nc/W-1, in
//     (flavour, spin, colour) order; 16-bit fields append a float scale per site
//     after the vectors (value = stored * scale, |stored| <= 1).
//   links  per parity p and direction mu: 9 complex, W_link = 2 reals per vector
//     (double2 / float2 / 2x16-bit), element (mu*9 + k)*Vh + i.
//   clover per parity, a flat list of reals (multiples of 8) in W-wide vectors.
// ---------------------------------------------------------------------------
enum Prec { P64 = 0, P32 = 1, PB16 = 2, PF16 = 3 };
// Kernel-internal precision of the reliable updates: FP64 storage layouts and
// sizes, double-word arithmetic (df64.h).  Links, clover blocks and spinors are
// held as (hi, lo) FP32 pairs, a float4 per two reals (the FP64 double2 slot).
constexpr int PDF = 4;

template <int P> struct PT;
template <> struct PT<P64> { using R = double; static constexpr int W = 2; static constexpr int ESZ = 8; };
template <> struct PT<P32> { using R = float;  static constexpr int W = 4; static constexpr int ESZ = 4; };
template <> struct PT<PB16> { using R = float; static constexpr int W = 8; static constexpr int ESZ = 2; };
template <> struct PT<PF16> { using R = float; static constexpr int W = 8; static constexpr int ESZ = 2; };
template <> struct PT<PDF> { using R = df; static constexpr int W = 2; static constexpr int ESZ = 8; };

__host__ __device__ inline int prec_esz(int p) { return (p == P64 || p == PDF) ? 8 : (p == P32 ? 4 : 2); }
__host__ __device__ inline int prec_w(int p) { return (p == P64 || p == PDF) ? 2 : (p == P32 ? 4 : 8); }

// bytes of a native spinor field of nc complex components per site
__host__ __device__ inline size_t spinor_bytes(int p, int nc, long vh) {
    size_t b = (size_t)vh * nc * 2 * prec_esz(p);
    if (p == PB16 || p == PF16) b += (size_t)vh * sizeof(float);
    return b;
}
// FP64 and BF16 links store 18 reals, FP32 / FP16 links 12 (two rows; see load_link)
__host__ __device__ inline size_t link_bytes_parity(int p, long vh) {
    return (size_t)vh * 4 * ((p == P32 || p == PF16) ? 12 : 18) * prec_esz(p);
}

template <int P> __device__ __forceinline__ float h2f(uint16_t v);
template <> __device__ __forceinline__ float h2f<PF16>(uint16_t v) { return __half2float(__ushort_as_half(v)); }
template <> __device__ __forceinline__ float h2f<PB16>(uint16_t v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
template <int P> __device__ __forceinline__ uint16_t f2h(float v);
template <> __device__ __forceinline__ uint16_t f2h<PF16>(float v) { return __half_as_ushort(__float2half_rn(v)); }
template <> __device__ __forceinline__ uint16_t f2h<PB16>(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }

// paired conversions of a 32-bit word holding two 16-bit values (low half first)
template <int P> __device__ __forceinline__ float2 h2f2(uint32_t w);
template <> __device__ __forceinline__ float2 h2f2<PF16>(uint32_t w) {
    __half2 h;
    memcpy(&h, &w, 4);
    return __half22float2(h);
}
template <> __device__ __forceinline__ float2 h2f2<PB16>(uint32_t w) {
    // a BF16 value is the upper 16 bits of the FP32 value
    return make_float2(__uint_as_float(w << 16), __uint_as_float(w & 0xffff0000u));
}
template <int P> __device__ __forceinline__ uint32_t f2h2(float lo, float hi);
template <> __device__ __forceinline__ uint32_t f2h2<PF16>(float lo, float hi) {
    const __half2 h = __floats2half2_rn(lo, hi);
    uint32_t w;
    memcpy(&w, &h, 4);
    return w;
}
template <> __device__ __forceinline__ uint32_t f2h2<PB16>(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    uint32_t w;
    memcpy(&w, &h, 4);
    return w;
}

// Load NR reals (NR multiple of W) starting at real offset OFF of site i.
template <int P, int NR>
__device__ __forceinline__ void load_reals(const void* base, long vh, long i, int off,
                                           typename PT<P>::R* dst) {
    constexpr int W = PT<P>::W;
    const int v0 = off / W;
#pragma unroll
    for (int v = 0; v < NR / W; ++v) {
        const long e = (long)(v0 + v) * vh + i;
        if constexpr (P == P64) {
            double2 q = __ldg(reinterpret_cast<const double2*>(base) + e);
            dst[2 * v] = q.x; dst[2 * v + 1] = q.y;
        } else if constexpr (P == PDF) {
            float4 q = __ldg(reinterpret_cast<const float4*>(base) + e);
            dst[2 * v] = df(q.x, q.y); dst[2 * v + 1] = df(q.z, q.w);
        } else if constexpr (P == P32) {
            float4 q = __ldg(reinterpret_cast<const float4*>(base) + e);
            dst[4 * v] = q.x; dst[4 * v + 1] = q.y; dst[4 * v + 2] = q.z; dst[4 * v + 3] = q.w;
        } else {
            uint4 q = __ldg(reinterpret_cast<const uint4*>(base) + e);
            const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const float2 f = h2f2<P>(w[k]);
                dst[8 * v + 2 * k] = f.x;
                dst[8 * v + 2 * k + 1] = f.y;
            }
        }
    }
}

template <int P, int NR>
__device__ __forceinline__ void store_reals(void* base, long vh, long i, int off,
                                            const typename PT<P>::R* src) {
    constexpr int W = PT<P>::W;
    const int v0 = off / W;
#pragma unroll
    for (int v = 0; v < NR / W; ++v) {
        const long e = (long)(v0 + v) * vh + i;
        if constexpr (P == P64) {
            reinterpret_cast<double2*>(base)[e] = make_double2(src[2 * v], src[2 * v + 1]);
        } else if constexpr (P == PDF) {
            reinterpret_cast<float4*>(base)[e] = make_float4(src[2 * v].h, src[2 * v].l, src[2 * v + 1].h, src[2 * v + 1].l);
        } else if constexpr (P == P32) {
            reinterpret_cast<float4*>(base)[e] =
                make_float4(src[4 * v], src[4 * v + 1], src[4 * v + 2], src[4 * v + 3]);
        } else {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                w[k] = f2h2<P>(src[8 * v + 2 * k], src[8 * v + 2 * k + 1]);
            reinterpret_cast<uint4*>(base)[e] = make_uint4(w[0], w[1], w[2], w[3]);
        }
    }
}

// Spinor of NC complex components at site i.
template <int P, int NC>
__device__ __forceinline__ void load_spinor(const void* base, long vh, long i,
                                            cpx<typename PT<P>::R>* s) {
    using R = typename PT<P>::R;
    load_reals<P, 2 * NC>(base, vh, i, 0, reinterpret_cast<R*>(s));
    if constexpr (P == PB16 || P == PF16) {
        const float* nrm = reinterpret_cast<const float*>(
            reinterpret_cast<const char*>(base) + (size_t)vh * NC * 2 * 2);
        const float sc = __ldg(nrm + i);
#pragma unroll
        for (int k = 0; k < NC; ++k) { s[k].re *= sc; s[k].im *= sc; }
    }
}

// as load_spinor, but 16-bit spinors stay unscaled and their per-site scale is
// returned in sc (1 for FP32 / FP64)
template <int P, int NC>
__device__ __forceinline__ void load_spinor_unscaled(const void* base, long vh, long i,
                                                     cpx<typename PT<P>::R>* s, float& sc) {
    using R = typename PT<P>::R;
    load_reals<P, 2 * NC>(base, vh, i, 0, reinterpret_cast<R*>(s));
    sc = 1.f;
    if constexpr (P == PB16 || P == PF16) {
        const float* nrm = reinterpret_cast<const float*>(
            reinterpret_cast<const char*>(base) + (size_t)vh * NC * 2 * 2);
        sc = __ldg(nrm + i);
    }
}

template <int P, int NC>
__device__ __forceinline__ void store_spinor(void* base, long vh, long i,
                                             const cpx<typename PT<P>::R>* s) {
    using R = typename PT<P>::R;
    if constexpr (P == PB16 || P == PF16) {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < NC; ++k) m = fmaxf(m, fmaxf(fabsf(s[k].re), fabsf(s[k].im)));
        const float inv = m > 0.f ? 1.f / m : 0.f;
        R t[2 * NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) { t[2 * k] = s[k].re * inv; t[2 * k + 1] = s[k].im * inv; }
        store_reals<P, 2 * NC>(base, vh, i, 0, t);
        float* nrm = reinterpret_cast<float*>(reinterpret_cast<char*>(base) + (size_t)vh * NC * 2 * 2);
        nrm[i] = m;
    } else {
        store_reals<P, 2 * NC>(base, vh, i, 0, reinterpret_cast<const R*>(s));
    }
}

// Complex entries stored per link: FP32 and FP16 keep the first two rows only (12
// reals) and rebuild the third from unitarity with det U = 1.  FP64 keeps all 9
// (its passes are bound by FP64 arithmetic, not bytes), and so does BF16: a third
// row rebuilt from two rows rounded to BF16's 8-bit significand exceeds the 3e-3
// operator error budget.
template <int P> struct LinkStore { static constexpr int N = (P == P32 || P == PF16) ? 6 : 9; };

// row 2 of an SU(3) matrix = conj(row 0 x row 1)
template <typename R>
__device__ __forceinline__ void su3_third_row(cpx<R>* u) {
    u[6] = cj(u[1] * u[5] - u[2] * u[4]);
    u[7] = cj(u[2] * u[3] - u[0] * u[5]);
    u[8] = cj(u[0] * u[4] - u[1] * u[3]);
}

// SU(3) link (9 complex, row major) of direction mu at site i of one parity;
// element k of direction mu lives at (mu * LinkStore<P>::N + k) * vh + i.
template <int P>
__device__ __forceinline__ void load_link(const void* base, long vh, int mu, long i,
                                          cpx<typename PT<P>::R>* u) {
    constexpr int N = LinkStore<P>::N;
#pragma unroll
    for (int k = 0; k < N; ++k) {
        const long e = (long)(mu * N + k) * vh + i;
        if constexpr (P == P64) {
            double2 q = __ldg(reinterpret_cast<const double2*>(base) + e);
            u[k] = C(q.x, q.y);
        } else if constexpr (P == PDF) {
            float4 q = __ldg(reinterpret_cast<const float4*>(base) + e);
            u[k] = C(df(q.x, q.y), df(q.z, q.w));
        } else if constexpr (P == P32) {
            float2 q = __ldg(reinterpret_cast<const float2*>(base) + e);
            u[k] = C(q.x, q.y);
        } else {
            uint32_t q = __ldg(reinterpret_cast<const unsigned int*>(base) + e);
            const float2 f = h2f2<P>(q);
            u[k] = C(f.x, f.y);
        }
    }
    if constexpr (N == 6) su3_third_row(u);
}

// ---------------------------------------------------------------------------
// clover layouts (reals per site)
//   hermitian 6x6 block: 6 real diagonal entries, then the 15 strictly-lower
//   entries (i>j, row by row) as (re, im): 36 reals.
//   full 6x6 block: row major complex: 72 reals.
//   odd  A:       [A0 herm 36][A1 herm 36]                          72 reals
//   even light:   [B0 full 72][B1 full 72]  B_c = (A_c + i s_c mu_t)^-1   144 reals
//   even heavy:   [A0-1 herm 36][D0-1 herm 36][A1-1 herm 36][D1-1 herm 36]  144 reals
//                 D_c = (A_c^2 + mubar_t^2 - epsbar_t^2)^-1; the block inverse
//                 [[(A_c - i s_c mubar_t) D_c, epsbar_t D_c], [epsbar_t D_c, (A_c + i s_c mubar_t) D_c]]
//                 is applied from A_c and D_c (they commute)
// (s_c = +1 for chirality 0 = spins 0,1 and -1 for spins 2,3.)
// ---------------------------------------------------------------------------
constexpr int CLOV_ODD_REALS = 72;
constexpr int CLOV_EVEN_LIGHT_REALS = 144;
constexpr int CLOV_EVEN_HEAVY_REALS = 144;

__host__ __device__ constexpr int herm_off(int i, int j) {   // i > j
    return 6 + 2 * (i * (i - 1) / 2 + j);
}

// ---------------------------------------------------------------------------
// solver control word (device memory, one per problem)
// ---------------------------------------------------------------------------
enum CtlFlag { CTL_RUN = 0, CTL_STOP = 1, CTL_BREAKDOWN = 2, CTL_MAXITER = 3 };

struct SolverCtl {
    double rr;        // current iterated ||r||^2
    double rr_old;    // ||r||^2 of the previous iteration
    double pAp;       // <p, A p>
    double alpha;
    double beta;
    double stop_rr;   // stop the chunk when rr < stop_rr
    double result;    // generic reduction result
    double shift;     // constant shift added to A (multishift base shift / refinement)
    int iter;
    int maxiter;
    int flag;
    int pad;
};

// Multishift state (one per multishift solve), up to MAX_SHIFTS shifts.
constexpr int MAX_SHIFTS = 16;
struct MsCtl {
    double zeta[MAX_SHIFTS], zeta_old[MAX_SHIFTS];
    double alpha_s[MAX_SHIFTS], beta_s[MAX_SHIFTS];
    double dshift[MAX_SHIFTS];     // sigma_k - sigma_0
    double alpha_old, beta_old;
    double stop_rr;                // per shift: zeta^2 rr < stop_rr => frozen
    int active[MAX_SHIFTS];
    int nshift;
    int n_active;
};

// ---------------------------------------------------------------------------
// problem descriptors for batched kernels (one block belongs to one problem)
// ---------------------------------------------------------------------------
constexpr int MAXP = 32;

struct Geom {
    int X, Y, Z, T;
    long vh;                 // sites per parity; the volume 2 vh is below 2^31
    FastDiv dxh, dy, dz;     // division by X/2, Y, Z (geom_init)
};

inline void geom_init(Geom& g, int X, int Y, int Z, int T) {
    g.X = X; g.Y = Y; g.Z = Z; g.T = T;
    g.vh = (long)X * Y * Z * T / 2;
    g.dxh = make_fastdiv((uint32_t)(X / 2));
    g.dy = make_fastdiv((uint32_t)Y);
    g.dz = make_fastdiv((uint32_t)Z);
}

struct OpProb {
    Geom g;
    int nblk;
    float bc_t;
    const void* gauge[2];    // native links of parity 0 / 1
    const void* clov;        // clover array of the output parity
    const void* in;          // hopping input (other parity)
    const void* loc;         // K2: odd-site input for the local term
    void* out;
    double kappa;
    double tw;               // light: sign*mu_t; heavy: sign*mubar_t (K2 local term)
    double eps;              // heavy: epsbar_t
    double rho;              // odd pass: out += i rho psi (W_hat: sign * 2 kappa rho; else 0)
    int sign;                // +1 / -1 (which inverse / adjoint)
    SolverCtl* ctl;          // early exit when ctl->flag != 0 (may be null)
    MsCtl* ms;               // multishift state for FIN_MS_ALPHA (may be null)
    double* partial;         // per-block partial sums for the fused norm (may be null)
    unsigned int* counter;   // last-block counter for the fused norm
};

template <int NP>
struct OpBatch {
    int n;
    int fin;                 // finalisation of the fused norm (FinOp)
    int blk_start[NP + 1];
    OpProb p[NP];
};

enum FinOp { FIN_NONE = 0, FIN_STORE = 1, FIN_CG_ALPHA = 2, FIN_MS_ALPHA = 3 };

template <int NP>
__device__ __forceinline__ int find_problem(const OpBatch<NP>& b, int blk) {
    int k = 0;
#pragma unroll 1
    while (k + 1 < b.n && blk >= b.blk_start[k + 1]) ++k;
    return k;
}

// site coordinates of checkerboard index i of parity par
struct Coord {
    int x, y, z, t;
};
// (32-bit arithmetic throughout: the volume is below 2^31)
__device__ __forceinline__ Coord cb_coords(const Geom& g, long i, int par) {
    const uint32_t u = (uint32_t)i;
    const uint32_t r = fdiv(u, g.dxh);       // i / (X/2)
    const uint32_t q = fdiv(r, g.dy);
    const uint32_t t = fdiv(q, g.dz);
    Coord c;
    c.y = (int)(r - q * g.dy.d);
    c.z = (int)(q - t * g.dz.d);
    c.t = (int)t;
    c.x = 2 * (int)(u - r * g.dxh.d) + ((c.y + c.z + c.t + par) & 1);
    return c;
}
__device__ __forceinline__ long cb_index(const Geom& g, int x, int y, int z, int t) {
    return (long)((((t * g.Z + z) * g.Y + y) * g.X + x) >> 1);
}

}  // namespace tmk
