// Gauge-field import, low-precision link copies, and the clover term with its
// site-local inverses (Sec. 2: the clover term and the even-site blocks
// (M_ee +- i mu g5)^-1 of eq:hQpm and (M_ee + i mubar g5 tau3 - epsbar tau1)^-1
// of eq:hQh).  All clover arithmetic is FP64; stored copies are converted to the
// requested storage precision afterwards.
#include "tm_internal.h"
#include "tm_kernels.h"

namespace tmk {

// canonical [t][z][y][x][mu][3][3] complex FP64 -> native FP64 [parity][mu*9+k][vh] double2
__global__ void k_gauge_import(void* dst0, void* dst1, const double* __restrict__ src, Geom g) {
    const long V = 2 * g.vh;
    const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * V) return;
    const long lex = idx >> 2;
    const int mu = (int)(idx & 3);
    long r = lex;
    const int x = (int)(r % g.X); r /= g.X;
    const int y = (int)(r % g.Y); r /= g.Y;
    const int z = (int)(r % g.Z);
    const int t = (int)(r / g.Z);
    const int par = (x + y + z + t) & 1;
    const long cb = lex >> 1;
    double2* d = reinterpret_cast<double2*>(par ? dst1 : dst0);
    const double2* s = reinterpret_cast<const double2*>(src) + idx * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) d[(long)(mu * 9 + k) * g.vh + cb] = s[k];
}

// native FP64 links of one parity (9 complex per direction) -> native precision P
// (the first LinkStore<P>::N complex per direction; FP32/16-bit keep rows 0, 1)
template <int P>
__global__ void k_links_from64(void* dst, const double2* __restrict__ src, long vh) {
    constexpr int N = LinkStore<P>::N;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // destination element
    if (e >= 4 * N * vh) return;
    const long w = e / vh, i = e - w * vh;
    const int mu = (int)(w / N), k = (int)(w % N);
    const double2 v = src[(long)(mu * 9 + k) * vh + i];
    if constexpr (P == P32) {
        reinterpret_cast<float2*>(dst)[e] = make_float2((float)v.x, (float)v.y);
    } else if constexpr (P == P64) {
        reinterpret_cast<double2*>(dst)[e] = v;
    } else {
        const uint32_t w = f2h2<P>((float)v.x, (float)v.y);
        reinterpret_cast<unsigned int*>(dst)[e] = w;
    }
}

// native FP64 clover reals (nreal per site, double2 vectors) -> native precision P
template <int P>
__global__ void k_clover_from64(void* dst, const double* __restrict__ src, long vh, int nreal) {
    constexpr int W = PT<P>::W;
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;   // target vector index
    const long nvec = (long)(nreal / W) * vh;
    if (e >= nvec) return;
    const long v = e / vh, i = e - v * vh;
    typename PT<P>::R buf[W];
#pragma unroll
    for (int c = 0; c < W; ++c) {
        const long r = v * W + c;                       // real index within the site
        buf[c] = (typename PT<P>::R)src[((r >> 1) * vh + i) * 2 + (r & 1)];
    }
    store_reals<P, W>(dst, vh, i, (int)(v * W), buf);
}

// ---------------------------------------------------------------------------
// clover term
// ---------------------------------------------------------------------------
using cd = cpx<double>;

struct M3 {
    cd m[9];
};

__device__ __forceinline__ M3 mm(const M3& a, const M3& b) {   // a b
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cd s = C(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cfma(s, a.m[3 * i + k], b.m[3 * k + j]);
            c.m[3 * i + j] = s;
        }
    return c;
}
__device__ __forceinline__ M3 mmd(const M3& a, const M3& b) {  // a b^+
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cd s = C(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) s = s + a.m[3 * i + k] * cj(b.m[3 * j + k]);
            c.m[3 * i + j] = s;
        }
    return c;
}
__device__ __forceinline__ M3 mdm(const M3& a, const M3& b) {  // a^+ b
    M3 c;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cd s = C(0.0, 0.0);
#pragma unroll
            for (int k = 0; k < 3; ++k) cfma_cj(s, a.m[3 * k + i], b.m[3 * k + j]);
            c.m[3 * i + j] = s;
        }
    return c;
}

__device__ __forceinline__ M3 link_at(const Geom& g, const void* const* gauge, int mu,
                                      int x, int y, int z, int t) {
    x = (x + g.X) % g.X; y = (y + g.Y) % g.Y; z = (z + g.Z) % g.Z; t = (t + g.T) % g.T;
    const int par = (x + y + z + t) & 1;
    M3 u;
    load_link<P64>(gauge[par], g.vh, mu, cb_index(g, x, y, z, t), u.m);
    return u;
}

// F_munu(x) = (1/8)(Q - Q^+) - (1/3) tr, Q = sum of the four leaves in the (mu,nu) plane
__device__ M3 clover_leaf(const Geom& g, const void* const* gauge, int mu, int nu, const int* xc) {
    int e_mu[4] = {0, 0, 0, 0}, e_nu[4] = {0, 0, 0, 0};
    e_mu[mu] = 1;
    e_nu[nu] = 1;
    auto L = [&](int d, int dm, int dn) {   // U_d(x + dm mu + dn nu)
        return link_at(g, gauge, d, xc[0] + dm * e_mu[0] + dn * e_nu[0], xc[1] + dm * e_mu[1] + dn * e_nu[1],
                       xc[2] + dm * e_mu[2] + dn * e_nu[2], xc[3] + dm * e_mu[3] + dn * e_nu[3]);
    };
    // leaf 1: U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    M3 q = mmd(mmd(mm(L(mu, 0, 0), L(nu, 1, 0)), L(mu, 0, 1)), L(nu, 0, 0));
    // leaf 2: U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    M3 l2 = mm(mmd(mmd(L(nu, 0, 0), L(mu, -1, 1)), L(nu, -1, 0)), L(mu, -1, 0));
    // leaf 3: U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu) = (b a)^+ c d
    M3 l3;
    {
        const M3 a = L(mu, -1, 0), b = L(nu, -1, -1), c = L(mu, -1, -1), d = L(nu, 0, -1);
        l3 = mm(mdm(mm(b, a), c), d);
    }
    // leaf 4: U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    M3 l4 = mmd(mm(mdm(L(nu, 0, -1), L(mu, 0, -1)), L(nu, 1, -1)), L(mu, 0, 0));
#pragma unroll
    for (int k = 0; k < 9; ++k) q.m[k] = q.m[k] + l2.m[k] + l3.m[k] + l4.m[k];
    M3 f;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) f.m[3 * i + j] = 0.125 * (q.m[3 * i + j] - cj(q.m[3 * j + i]));
    const double tr_im = (f.m[0].im + f.m[4].im + f.m[8].im) / 3.0;   // trace is imaginary
#pragma unroll
    for (int i = 0; i < 3; ++i) f.m[4 * i].im -= tr_im;
    return f;
}

// inverse of a 6x6 hermitian positive definite matrix (Cholesky), in place
__device__ void hpd6_inverse(cd (&h)[36]) {
    cd L[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) L[k] = C(0.0, 0.0);
    for (int j = 0; j < 6; ++j) {
        double d = h[6 * j + j].re;
        for (int k = 0; k < j; ++k) d -= norm2(L[6 * j + k]);
        const double ljj = sqrt(d);
        L[6 * j + j] = C(ljj, 0.0);
        for (int i = j + 1; i < 6; ++i) {
            cd s = h[6 * i + j];
            for (int k = 0; k < j; ++k) s = s - L[6 * i + k] * cj(L[6 * j + k]);
            L[6 * i + j] = (1.0 / ljj) * s;
        }
    }
    cd Li[36];
#pragma unroll
    for (int k = 0; k < 36; ++k) Li[k] = C(0.0, 0.0);
    for (int i = 0; i < 6; ++i) {
        Li[6 * i + i] = C(1.0 / L[6 * i + i].re, 0.0);
        for (int j = 0; j < i; ++j) {
            cd s = C(0.0, 0.0);
            for (int k = j; k < i; ++k) s = s + L[6 * i + k] * Li[6 * k + j];
            Li[6 * i + j] = (-1.0 / L[6 * i + i].re) * s;
        }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) {
            cd s = C(0.0, 0.0);
            const int k0 = i > j ? i : j;
            for (int k = k0; k < 6; ++k) cfma_cj(s, Li[6 * k + i], Li[6 * k + j]);
            h[6 * i + j] = s;
        }
}

__device__ __forceinline__ void put_real(double* base, long vh, long i, int r, double v) {
    base[((long)(r >> 1) * vh + i) * 2 + (r & 1)] = v;
}

// One thread per site of parity `par`:
//   A_c = 1 - kappa csw [ i s1 (x) a1 + i s2 (x) a2 + i s3 (x) a3 ],
//   a1 = F_yz + s F_xt,  a2 = -F_xz + s F_yt,  a3 = F_xy + s F_zt  (s = +1 / -1 per chirality),
// which is the chirality-block form of 1 - kappa csw sum_{mu<nu} g_mu g_nu F_munu.
// Writes A (packed hermitian, 72 reals/site); on even sites also the light inverse
// blocks B_c = (A_c + i s mu_t)^-1 (144 reals) and/or the heavy A_c, D_c (144).
__global__ void k_clover(Geom g, const void* g0, const void* g1, int par, double kappa, double csw,
                         double mu_t, double mubar_t, double epsbar_t, double* outA,
                         double* outB, double* outH) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.vh) return;
    const void* gauge[2] = {g0, g1};
    const Coord c = cb_coords(g, i, par);
    const int xc[4] = {c.x, c.y, c.z, c.t};
    const double kc = kappa * csw;
    M3 F[6];
    int n = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu) F[n++] = clover_leaf(g, gauge, mu, nu, xc);
    // plane order: 0 xy, 1 xz, 2 xt, 3 yz, 4 yt, 5 zt
    for (int cb = 0; cb < 2; ++cb) {
        const double s = cb == 0 ? 1.0 : -1.0;
        cd A[36];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                const cd a1 = F[3].m[3 * a + b] + s * F[2].m[3 * a + b];
                const cd a2 = s * F[4].m[3 * a + b] - F[1].m[3 * a + b];
                const cd a3 = F[0].m[3 * a + b] + s * F[5].m[3 * a + b];
                const double id = (a == b) ? 1.0 : 0.0;
                // S = [[ i a3, i a1 + a2 ], [ i a1 - a2, -i a3 ]]
                A[6 * (0 + a) + (0 + b)] = C(id, 0.0) - kc * mul_i(a3);
                A[6 * (0 + a) + (3 + b)] = -kc * (mul_i(a1) + a2);
                A[6 * (3 + a) + (0 + b)] = -kc * (mul_i(a1) - a2);
                A[6 * (3 + a) + (3 + b)] = C(id, 0.0) + kc * mul_i(a3);
            }
        // packed hermitian store
        for (int r = 0; r < 6; ++r) put_real(outA, g.vh, i, 36 * cb + r, A[7 * r].re);
        for (int r = 1; r < 6; ++r)
            for (int j = 0; j < r; ++j) {
                put_real(outA, g.vh, i, 36 * cb + herm_off(r, j), A[6 * r + j].re);
                put_real(outA, g.vh, i, 36 * cb + herm_off(r, j) + 1, A[6 * r + j].im);
            }
        if (par != 0) continue;
        // A^2 (hermitian)
        cd A2[36];
        for (int r = 0; r < 6; ++r)
            for (int j = 0; j < 6; ++j) {
                cd t = C(0.0, 0.0);
                for (int k = 0; k < 6; ++k) cfma(t, A[6 * r + k], A[6 * k + j]);
                A2[6 * r + j] = t;
            }
        if (outB != nullptr) {
            cd D[36];
            for (int k = 0; k < 36; ++k) D[k] = A2[k];
            for (int r = 0; r < 6; ++r) D[7 * r].re += mu_t * mu_t;
            hpd6_inverse(D);
            // B = (A - i s mu_t) D
            for (int r = 0; r < 6; ++r)
                for (int j = 0; j < 6; ++j) {
                    cd t = C(0.0, 0.0);
                    for (int k = 0; k < 6; ++k) {
                        cd a = A[6 * r + k];
                        if (k == r) a.im -= s * mu_t;
                        cfma(t, a, D[6 * k + j]);
                    }
                    put_real(outB, g.vh, i, 72 * cb + 2 * (6 * r + j), t.re);
                    put_real(outB, g.vh, i, 72 * cb + 2 * (6 * r + j) + 1, t.im);
                }
        }
        if (outH != nullptr) {
            cd D[36];
            for (int k = 0; k < 36; ++k) D[k] = A2[k];
            for (int r = 0; r < 6; ++r) D[7 * r].re += mubar_t * mubar_t - epsbar_t * epsbar_t;
            hpd6_inverse(D);
            // [A_c - 1 36][D_c - 1 36] per chirality, both packed hermitian (the
            // deviation from the identity keeps 16-bit rounding relative to it)
            for (int r = 0; r < 6; ++r) {
                put_real(outH, g.vh, i, 72 * cb + r, A[7 * r].re - 1.0);
                put_real(outH, g.vh, i, 72 * cb + 36 + r, D[7 * r].re - 1.0);
            }
            for (int r = 1; r < 6; ++r)
                for (int j = 0; j < r; ++j) {
                    put_real(outH, g.vh, i, 72 * cb + herm_off(r, j), A[6 * r + j].re);
                    put_real(outH, g.vh, i, 72 * cb + herm_off(r, j) + 1, A[6 * r + j].im);
                    put_real(outH, g.vh, i, 72 * cb + 36 + herm_off(r, j), D[6 * r + j].re);
                    put_real(outH, g.vh, i, 72 * cb + 36 + herm_off(r, j) + 1, D[6 * r + j].im);
                }
        }
    }
}

// unpack the packed hermitian A of one parity to [site][2][6][6] complex (debug export)
__global__ void k_clover_unpack(double2* out, const double* __restrict__ A, long vh) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    auto get = [&](int r) { return A[((long)(r >> 1) * vh + i) * 2 + (r & 1)]; };
    for (int cb = 0; cb < 2; ++cb)
        for (int r = 0; r < 6; ++r)
            for (int j = 0; j < 6; ++j) {
                double re, im;
                if (r == j) { re = get(36 * cb + r); im = 0.0; }
                else if (r > j) { re = get(36 * cb + herm_off(r, j)); im = get(36 * cb + herm_off(r, j) + 1); }
                else { re = get(36 * cb + herm_off(j, r)); im = -get(36 * cb + herm_off(j, r) + 1); }
                out[((i * 2 + cb) * 6 + r) * 6 + j] = make_double2(re, im);
            }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
cudaError_t launch_gauge_import(void* d0, void* d1, const double* src, const Geom& g, cudaStream_t st) {
    const long n = 8 * g.vh;
    k_gauge_import<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(d0, d1, src, g);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_links_from64(void* dst, const void* src64, long vh, cudaStream_t st) {
    const long n = 4 * LinkStore<P>::N * vh;
    k_links_from64<P><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst, reinterpret_cast<const double2*>(src64), vh);
    return cudaGetLastError();
}

template <int P>
cudaError_t launch_clover_from64(void* dst, const double* src, long vh, int nreal, cudaStream_t st) {
    const long n = (long)(nreal / PT<P>::W) * vh;
    k_clover_from64<P><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(dst, src, vh, nreal);
    return cudaGetLastError();
}

cudaError_t launch_clover(const Geom& g, const void* g0, const void* g1, int par, double kappa, double csw,
                          double mu_t, double mubar_t, double epsbar_t, double* outA, double* outB,
                          double* outH, cudaStream_t st) {
    k_clover<<<(unsigned)((g.vh + 63) / 64), 64, 0, st>>>(g, g0, g1, par, kappa, csw, mu_t, mubar_t,
                                                          epsbar_t, outA, outB, outH);
    return cudaGetLastError();
}

cudaError_t launch_clover_unpack(double* out, const double* A, long vh, cudaStream_t st) {
    k_clover_unpack<<<(unsigned)((vh + 127) / 128), 128, 0, st>>>(reinterpret_cast<double2*>(out), A, vh);
    return cudaGetLastError();
}

// FP64 arrays (a double2 per two reals: links, clover blocks, spinors) <->
// double-word arrays (a float4 (h, l, h, l) per two reals), n 16-byte elements;
// in place is allowed (each thread reads and writes only its own element)
__global__ void k_f64_to_df(float4* dst, const double2* src, long n) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 v = src[e];
    const df x(v.x), y(v.y);
    dst[e] = make_float4(x.h, x.l, y.h, y.l);
}
__global__ void k_df_to_f64(double2* dst, const float4* src, long n) {
    const long e = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float4 q = src[e];
    dst[e] = make_double2((double)df(q.x, q.y), (double)df(q.z, q.w));
}
cudaError_t launch_f64_to_df(void* dst, const void* src, long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_f64_to_df<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<float4*>(dst),
                                                              reinterpret_cast<const double2*>(src), n);
    return cudaGetLastError();
}
cudaError_t launch_df_to_f64(void* dst, const void* src, long n, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_df_to_f64<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(reinterpret_cast<double2*>(dst),
                                                              reinterpret_cast<const float4*>(src), n);
    return cudaGetLastError();
}

template cudaError_t launch_links_from64<P32>(void*, const void*, long, cudaStream_t);
template cudaError_t launch_links_from64<PB16>(void*, const void*, long, cudaStream_t);
template cudaError_t launch_links_from64<PF16>(void*, const void*, long, cudaStream_t);
template cudaError_t launch_clover_from64<P32>(void*, const double*, long, int, cudaStream_t);
template cudaError_t launch_clover_from64<PB16>(void*, const double*, long, int, cudaStream_t);
template cudaError_t launch_clover_from64<PF16>(void*, const double*, long, int, cudaStream_t);

}  // namespace tmk
