// Gauge-equivariant parallel-transport network (PTC) used as a learned
// preconditioner in flexible CG: forward layer, input- and weight-gradient
// kernels, loss, Adam, and the training-pair generator.
//
// One layer maps C_in to C_out channels of full-lattice spinor fields:
//   out^a(x) = sum_{p in P} sum_b W_p^{ab} (T_p in^b)(x),
//   P = {1, +x,+y,+z,+t, -x,-y,-z,-t},  (T_{+mu} f)(x) = U_mu(x) f(x+mu),
//   (T_{-mu} f)(x) = U_mu(x-mu)^dag f(x-mu),  W_p^{ab} a complex 4x4 spin matrix.
// Because W acts on (channel, spin) and T on (site, colour), a tile of sites is
// a real GEMM per path: with every complex number split into (re, im),
//   Out[64 x 3S] += A_p[64 x 64] * V_p[64 x 3S],
//   rows (re/im, a<8, s<4), K = (re/im, b<8, t<4), columns (site, colour),
//   A_p = [[Re W, -Im W], [Im W, Re W]] (BF16), V_p = T_p in (BF16), FP32 accumulate.
// The transport (gather of neighbour activations, SU(3) multiply) fills V_p in
// shared memory and mma.sync m16n8k16 (BF16 in, FP32 accumulate) does the mixing.
// Channel counts below 8 are zero-padded in A_p.  Activations are BF16, layout
// [channel][3 x 16-B vectors of 4 complex (spin, colour)][V] in lexicographic site
// order.  The input gradient of a layer is the same layer run with the adjoint
// weights W'_p = (W_{rev p})^H (T_p^dag = T_{rev p}); the weight gradient is the
// site reduction G_p = sum_{x,c} delta(x) v_p(x)^H, again a BF16 tensor-core GEMM.
#include "tm_internal.h"
#include "tm_kernels.h"
#include "ptc.h"

namespace tmk {

__device__ __forceinline__ float bf(uint16_t v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
__device__ __forceinline__ uint16_t fb(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi) { return (uint32_t)fb(lo) | ((uint32_t)fb(hi) << 16); }

__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void site_coords(const PtcGeom& g, long x, int& cx, int& cy, int& cz, int& ct) {
    long r = x;
    cx = (int)(r % g.X); r /= g.X;
    cy = (int)(r % g.Y); r /= g.Y;
    cz = (int)(r % g.Z);
    ct = (int)(r / g.Z);
}

// neighbour site, link and phase of path p at lex site x; dag = use U^dagger
__device__ __forceinline__ long path_site(const PtcGeom& g, long x, int p, cpx<float> (&u)[9], bool& dag,
                                          float& ph) {
    int c[4];
    site_coords(g, x, c[0], c[1], c[2], c[3]);
    const int L[4] = {g.X, g.Y, g.Z, g.T};
    const int mu = (p - 1) & 3;
    const bool fwd = p <= 4;
    ph = 1.f;
    int y[4] = {c[0], c[1], c[2], c[3]};
    if (fwd) {
        y[mu] = (c[mu] + 1 == L[mu]) ? 0 : c[mu] + 1;
        if (mu == 3 && c[3] + 1 == g.T) ph = g.bc_t;
    } else {
        y[mu] = (c[mu] == 0) ? L[mu] - 1 : c[mu] - 1;
        if (mu == 3 && c[3] == 0) ph = g.bc_t;
    }
    const long ly = (((long)y[3] * g.Z + y[2]) * g.Y + y[1]) * g.X + y[0];
    const long ls = fwd ? x : ly;                       // site that owns the link
    const int* cs = fwd ? c : y;
    const int par = (cs[0] + cs[1] + cs[2] + cs[3]) & 1;
    load_link<PF16>(g.gauge[par], g.vh, mu, ls >> 1, u);
    dag = !fwd;
    return ly;
}

// 12 complex (spin, colour) of channel b at site y
__device__ __forceinline__ void act_load(const uint4* a, long V, int b, long y, cpx<float> (&v)[12]) {
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const uint4 w = __ldg(a + ((long)b * 3 + q) * V + y);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) v[4 * q + k] = C(bf((uint16_t)(ws[k] & 0xffffu)), bf((uint16_t)(ws[k] >> 16)));
    }
}

// Transport channels [b0, b0 + n) of `in` along path p to site x: the link and
// the neighbour index are computed once for the whole channel group; each
// transported 12-complex (spin, colour) spinor is handed to sink(b, w).
template <int NMAX, typename Sink>
__device__ __forceinline__ void transport_channels(const PtcGeom& g, const uint4* in, long x, int p, int b0,
                                                   int n, Sink&& sink) {
    cpx<float> u[9];
    bool dag = false;
    float ph = 1.f;
    long y = x;
    if (p != 0) y = path_site(g, x, p, u, dag, ph);
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
        if (k >= n) break;
        const int b = b0 + k;
        cpx<float> v[12], w[12];
        act_load(in, g.V, b, y, v);
        if (p == 0) {
#pragma unroll
            for (int q = 0; q < 12; ++q) w[q] = v[q];
        } else {
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    cpx<float> t = C(0.f, 0.f);
#pragma unroll
                    for (int d = 0; d < 3; ++d) {
                        if (dag) cfma_cj(t, u[3 * d + c], v[3 * sp + d]);
                        else cfma(t, u[3 * c + d], v[3 * sp + d]);
                    }
                    w[3 * sp + c] = ph * t;
                }
        }
        sink(b, w);
    }
}

// ---------------------------------------------------------------------------
// forward layer (also the input-gradient layer with adjoint weights)
// Tile of PTC_LTILE = 64 sites (192 GEMM columns); thread t transports site
// t % 64 for the channel group t / 64, so each (site, path) link is rebuilt by
// at most two threads.  Warp w owns columns [48 w, 48 w + 48): 4 m-tiles x 6
// n-tiles of m16n8 accumulators.
// ---------------------------------------------------------------------------
constexpr int LDW = 36;   // padded row length in 32-bit words (72 bf16)

template <int CIN, int COUT>
__global__ void __launch_bounds__(PTC_BS, 2) ptc_layer_kernel(PtcGeom g, const uint4* __restrict__ in,
                                                             uint4* __restrict__ out,
                                                             const uint4* __restrict__ wemb, long ntiles) {
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t* Wsm = sm;                                // 9 x 64 rows x LDW words
    uint32_t* Vsm = Wsm + 9 * 64 * LDW;                // 192 columns x LDW words
    uint32_t* Osm = Vsm;                               // output staging reuses the V tile:
                                                       // 64 sites x 8 ch x 12 complex (bf16 pairs)
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    constexpr int CPG = (CIN + 1) / 2;                 // channels per transport group

    // weights: 9 x 64 x 64 bf16 = 9*64 rows of 8 uint4
    for (int e = tid; e < 9 * 64 * 8; e += PTC_BS) {
        const uint4 v = __ldg(wemb + e);
        const int row = e >> 3, q = e & 7;
        uint32_t* d = Wsm + row * LDW + 4 * q;
        d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
    }
    __syncthreads();

    for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const long x0 = tile * PTC_LTILE;
        // rows of absent input channels must read as zero (the tile also served as
        // output staging for the previous tile)
        if (CIN < 8) {
            for (int e = tid; e < PTC_LN * LDW; e += PTC_BS) Vsm[e] = 0u;
            __syncthreads();
        }
        float acc[4][6][4];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 6; ++b)
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

        const int j = tid % PTC_LTILE, grp = tid / PTC_LTILE;
        const long x = x0 + j;
        const int b0 = grp * CPG, nb = min(CPG, CIN - b0);
#pragma unroll 1
        for (int p = 0; p < 9; ++p) {
            auto sink = [&](int b, const cpx<float> (&w)[12]) {
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    uint32_t* col = Vsm + (3 * j + c) * LDW;
#pragma unroll
                    for (int h = 0; h < 2; ++h) {   // spins (2h, 2h+1)
                        col[2 * b + h] = pack2(w[3 * (2 * h) + c].re, w[3 * (2 * h + 1) + c].re);
                        col[16 + 2 * b + h] = pack2(w[3 * (2 * h) + c].im, w[3 * (2 * h + 1) + c].im);
                    }
                }
            };
            if (nb > 0) {
                if (x < g.V) {
                    transport_channels<CPG>(g, in, x, p, b0, nb, sink);
                } else {
                    cpx<float> z[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) z[q] = C(0.f, 0.f);
                    for (int k = 0; k < nb; ++k) sink(b0 + k, z);
                }
            }
            __syncthreads();
            const uint32_t* Wp = Wsm + p * 64 * LDW;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                uint32_t a[4][4];
#pragma unroll
                for (int mt = 0; mt < 4; ++mt) {
                    const uint32_t* r0 = Wp + (16 * mt + gq) * LDW + 8 * kk + tq;
                    a[mt][0] = r0[0];
                    a[mt][1] = r0[8 * LDW];
                    a[mt][2] = r0[4];
                    a[mt][3] = r0[8 * LDW + 4];
                }
#pragma unroll
                for (int nt = 0; nt < 6; ++nt) {
                    const uint32_t* c0 = Vsm + (48 * warp + 8 * nt + gq) * LDW + 8 * kk + tq;
                    const uint32_t b0v = c0[0], b1v = c0[4];
#pragma unroll
                    for (int mt = 0; mt < 4; ++mt) mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0v, b1v);
                }
            }
            __syncthreads();
        }
        // accumulators -> Osm as complex bf16 pairs [site][channel][s*3+c]
#pragma unroll
        for (int mt = 0; mt < 2; ++mt)
#pragma unroll
            for (int nt = 0; nt < 6; ++nt)
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const int m = 16 * mt + gq + 8 * (r >> 1);      // < 32: (a, s)
                    const int n = 48 * warp + 8 * nt + 2 * tq + (r & 1);
                    const int a = m >> 2, sp = m & 3, jj = n / 3, c = n % 3;
                    Osm[(jj * 8 + a) * 12 + 3 * sp + c] = pack2(acc[mt][nt][r], acc[mt + 2][nt][r]);
                }
        __syncthreads();
        for (int it = tid; it < PTC_LTILE * COUT * 3; it += PTC_BS) {
            const int jj = it % PTC_LTILE, rest = it / PTC_LTILE, q = rest % 3, a = rest / 3;
            const long xx = x0 + jj;
            if (xx < g.V) {
                const uint32_t* o = Osm + (jj * 8 + a) * 12 + 4 * q;
                out[((long)a * 3 + q) * g.V + xx] = make_uint4(o[0], o[1], o[2], o[3]);
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// weight gradient: Q_p[m][k] = sum_n D[m][n] V_p[k][n] over all (site, colour)
// columns n; D = [Re delta; Im delta] (64 rows), V_p = [Re T_p in; Im T_p in].
// Block (p, chunk) accumulates over its range of tiles and writes a partial.
// ---------------------------------------------------------------------------
constexpr int LDG = 52;   // padded row length in words (104 bf16) for 96 columns

template <int CIN, int COUT>
__global__ void __launch_bounds__(PTC_BS) ptc_wgrad_kernel(PtcGeom g, const uint4* __restrict__ in,
                                                          const uint4* __restrict__ delta, float* partial,
                                                          long ntiles, int nchunk) {
    __shared__ __align__(16) uint32_t VT[64 * LDG];
    __shared__ __align__(16) uint32_t DS[64 * LDG];
    const int p = blockIdx.x / nchunk, chunk = blockIdx.x % nchunk;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, tq = lane & 3;
    uint16_t* VT16 = reinterpret_cast<uint16_t*>(VT);
    uint16_t* DS16 = reinterpret_cast<uint16_t*>(DS);
    for (int e = tid; e < 64 * LDG; e += PTC_BS) { VT[e] = 0u; DS[e] = 0u; }
    __syncthreads();
    float acc[8][4];
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    const long per = (ntiles + nchunk - 1) / nchunk;
    const long t0 = chunk * per, t1 = min(ntiles, t0 + per);
    for (long tile = t0; tile < t1; ++tile) {
        const long x0 = tile * PTC_TILE;
        {
            constexpr int CPG = (CIN + 3) / 4;   // channels per transport group (4 groups of 32 sites)
            const int j = tid % PTC_TILE, grp = tid / PTC_TILE;
            const long x = x0 + j;
            const int b0 = grp * CPG, nb = min(CPG, CIN - b0);
            auto sink = [&](int b, const cpx<float> (&w)[12]) {
#pragma unroll
                for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        VT16[(4 * b + sp) * 2 * LDG + 3 * j + c] = fb(w[3 * sp + c].re);
                        VT16[(32 + 4 * b + sp) * 2 * LDG + 3 * j + c] = fb(w[3 * sp + c].im);
                    }
            };
            if (nb > 0) {
                if (x < g.V) {
                    transport_channels<CPG>(g, in, x, p, b0, nb, sink);
                } else {
                    cpx<float> z[12];
#pragma unroll
                    for (int q = 0; q < 12; ++q) z[q] = C(0.f, 0.f);
                    for (int k = 0; k < nb; ++k) sink(b0 + k, z);
                }
            }
        }
        for (int it = tid; it < PTC_TILE * COUT; it += PTC_BS) {
            const int j = it % PTC_TILE, a = it / PTC_TILE;
            const long x = x0 + j;
            cpx<float> d[12];
            if (x < g.V) act_load(delta, g.V, a, x, d);
            else {
#pragma unroll
                for (int q = 0; q < 12; ++q) d[q] = C(0.f, 0.f);
            }
#pragma unroll
            for (int s = 0; s < 4; ++s)
#pragma unroll
                for (int c = 0; c < 3; ++c) {
                    DS16[(4 * a + s) * 2 * LDG + 3 * j + c] = fb(d[3 * s + c].re);
                    DS16[(32 + 4 * a + s) * 2 * LDG + 3 * j + c] = fb(d[3 * s + c].im);
                }
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
            const uint32_t* ar = DS + (16 * warp + gq) * LDG + 8 * kk + tq;
            const uint32_t a0 = ar[0], a1 = ar[8 * LDG], a2 = ar[4], a3 = ar[8 * LDG + 4];
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const uint32_t* br = VT + (8 * nt + gq) * LDG + 8 * kk + tq;
                mma_bf16(acc[nt], a0, a1, a2, a3, br[0], br[4]);
            }
        }
        __syncthreads();
    }
    float* dst = partial + (size_t)blockIdx.x * 4096;
#pragma unroll
    for (int nt = 0; nt < 8; ++nt)
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int m = 16 * warp + gq + 8 * (r >> 1);
            const int k = 8 * nt + 2 * tq + (r & 1);
            dst[m * 64 + k] = acc[nt][r];
        }
}

// G[p][a][b][s][t] (complex) += scale * combination of the summed partials
__global__ void ptc_wgrad_reduce(const float* __restrict__ partial, int nchunk, int cin, int cout,
                                 float2* grad, float scale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = 9 * cout * cin * 16;
    if (e >= n) return;
    int r = e;
    const int t = r & 3; r >>= 2;
    const int s = r & 3; r >>= 2;
    const int b = r % cin; r /= cin;
    const int a = r % cout;
    const int p = r / cout;
    const int mre = 4 * a + s, mim = 32 + 4 * a + s, kre = 4 * b + t, kim = 32 + 4 * b + t;
    double rr = 0, ii = 0, ir = 0, ri = 0;
    for (int c = 0; c < nchunk; ++c) {
        const float* q = partial + ((size_t)p * nchunk + c) * 4096;
        rr += q[mre * 64 + kre];
        ii += q[mim * 64 + kim];
        ir += q[mim * 64 + kre];
        ri += q[mre * 64 + kim];
    }
    grad[e].x += scale * (float)(rr + ii);
    grad[e].y += scale * (float)(ir - ri);
}

// ---------------------------------------------------------------------------
// weights: FP32 complex master [9][cout][cin][4][4] -> BF16 real embeddings
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rev_path(int p) { return p == 0 ? 0 : (p <= 4 ? p + 4 : p - 4); }

__global__ void ptc_embed_weights(const float2* __restrict__ W, int cin, int cout, uint16_t* fwd, uint16_t* adj) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;   // over 9 x 64 x 64
    if (e >= 9 * 64 * 64) return;
    const int k = e & 63, m = (e >> 6) & 63, p = e >> 12;
    const int rim = m >> 5, cim = k >> 5;
    {   // forward: m = (ri, a, s), k = (ri', b, t)
        const int a = (m & 31) >> 2, s = m & 3, b = (k & 31) >> 2, t = k & 3;
        float v = 0.f;
        if (a < cout && b < cin) {
            const float2 w = W[(((p * cout + a) * cin + b) * 4 + s) * 4 + t];
            v = (rim == cim) ? w.x : (rim == 0 ? -w.y : w.y);
        }
        fwd[e] = fb(v);
    }
    {   // adjoint: W'_p[b][a][t][s] = conj(W_{rev p}[a][b][s][t]); m = (ri, b, t), k = (ri', a, s)
        const int b = (m & 31) >> 2, t = m & 3, a = (k & 31) >> 2, s = k & 3;
        float v = 0.f;
        if (a < cout && b < cin) {
            const float2 w0 = W[(((rev_path(p) * cout + a) * cin + b) * 4 + s) * 4 + t];
            const float2 w = make_float2(w0.x, -w0.y);
            v = (rim == cim) ? w.x : (rim == 0 ? -w.y : w.y);
        }
        adj[e] = fb(v);
    }
}

// Adam (Kingma & Ba) on re and im parts; grad is zeroed after the step
__global__ void ptc_adam(float2* W, float2* m, float2* v, float2* grad, int n, float lr, float b1, float b2,
                         float eps, float c1, float c2) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const float2 g = grad[e];
    float2 mm = m[e], vv = v[e], w = W[e];
    mm.x = b1 * mm.x + (1.f - b1) * g.x;
    mm.y = b1 * mm.y + (1.f - b1) * g.y;
    vv.x = b2 * vv.x + (1.f - b2) * g.x * g.x;
    vv.y = b2 * vv.y + (1.f - b2) * g.y * g.y;
    w.x -= lr * (mm.x / c1) / (sqrtf(vv.x / c2) + eps);
    w.y -= lr * (mm.y / c1) / (sqrtf(vv.y / c2) + eps);
    m[e] = mm;
    v[e] = vv;
    W[e] = w;
    grad[e] = make_float2(0.f, 0.f);
}

// ---------------------------------------------------------------------------
// odd native field <-> full-lattice single-channel activation
// ---------------------------------------------------------------------------
template <int P>
__global__ void ptc_embed_odd(const void* __restrict__ r, uint4* a0, PtcGeom g) {
    const long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    int cx, cy, cz, ct;
    site_coords(g, x, cx, cy, cz, ct);
    cpx<typename PT<P>::R> v[12];
    if ((cx + cy + cz + ct) & 1) load_spinor<P, 12>(r, g.vh, x >> 1, v);
    else {
#pragma unroll
        for (int q = 0; q < 12; ++q) v[q] = C((typename PT<P>::R)0, (typename PT<P>::R)0);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        a0[(long)q * g.V + x] = make_uint4(pack2((float)v[4 * q].re, (float)v[4 * q].im),
                                           pack2((float)v[4 * q + 1].re, (float)v[4 * q + 1].im),
                                           pack2((float)v[4 * q + 2].re, (float)v[4 * q + 2].im),
                                           pack2((float)v[4 * q + 3].re, (float)v[4 * q + 3].im));
}

template <int P>
__global__ void ptc_extract_odd(const uint4* __restrict__ a, void* z, PtcGeom g) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;   // odd cb index
    if (i >= g.vh) return;
    // lex of odd site i: row = i / (X/2); x parity chosen so that the site is odd
    const int xh2 = g.X >> 1;
    long r = i / xh2;
    const int xh = (int)(i - r * xh2);
    const int y = (int)(r % g.Y);
    const long r2 = r / g.Y;
    const int zz = (int)(r2 % g.Z), t = (int)(r2 / g.Z);
    const int x = 2 * xh + ((y + zz + t + 1) & 1);
    const long lex = (((long)t * g.Z + zz) * g.Y + y) * g.X + x;
    cpx<float> v[12];
    act_load(a, g.V, 0, lex, v);
    cpx<typename PT<P>::R> o[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) o[q] = C((typename PT<P>::R)v[q].re, (typename PT<P>::R)v[q].im);
    store_spinor<P, 12>(z, g.vh, i, o);
}

// loss ||z - e||^2 (block partials) and delta = (z - e) * inv_ee on odd sites (0 on even)
__global__ void ptc_loss_delta(const uint4* __restrict__ aL, const float4* __restrict__ e, uint4* delta, PtcGeom g,
                               const double* __restrict__ ee, double* partial) {
    __shared__ double sh[8];
    const float inv_ee = (float)(1.0 / *ee);
    const long x = (long)blockIdx.x * blockDim.x + threadIdx.x;
    double s = 0.0;
    if (x < g.V) {
        int cx, cy, cz, ct;
        site_coords(g, x, cx, cy, cz, ct);
        cpx<float> d[12];
        if ((cx + cy + cz + ct) & 1) {
            cpx<float> z[12];
            act_load(aL, g.V, 0, x, z);
            const long i = x >> 1;
            float t = 0.f;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float4 ev = e[(long)q * g.vh + i];
                const cpx<float> e0 = C(ev.x, ev.y), e1 = C(ev.z, ev.w);
                const cpx<float> d0 = z[2 * q] - e0, d1 = z[2 * q + 1] - e1;
                t += norm2(d0) + norm2(d1);
                d[2 * q] = inv_ee * d0;
                d[2 * q + 1] = inv_ee * d1;
            }
            s = t;
        } else {
#pragma unroll
            for (int q = 0; q < 12; ++q) d[q] = C(0.f, 0.f);
        }
#pragma unroll
        for (int q = 0; q < 3; ++q)
            delta[(long)q * g.V + x] = make_uint4(pack2(d[4 * q].re, d[4 * q].im), pack2(d[4 * q + 1].re, d[4 * q + 1].im),
                                                  pack2(d[4 * q + 2].re, d[4 * q + 2].im),
                                                  pack2(d[4 * q + 3].re, d[4 * q + 3].im));
    }
    const double bs = block_sum<256>(s, sh);
    if (threadIdx.x == 0) partial[blockIdx.x] = bs;
}

__global__ void sum_partials(const double* __restrict__ partial, int n, double* out) {
    __shared__ double sh[8];
    double t = 0.0;
    for (int k = threadIdx.x; k < n; k += 256) t += partial[k];
    t = block_sum<256>(t, sh);
    if (threadIdx.x == 0) *out = t;
}

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) and Box-Muller: complex
// Gaussian error vectors e (re, im ~ N(0,1)) on odd sites, FP32 native layout.
// counter = (site, vector, stream lo, stream hi), key = seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__global__ void ptc_gauss_odd(float4* e, long vh, unsigned long long seed, unsigned long long stream) {
    const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= vh) return;
    const uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const uint4 r = philox4x32_10(make_uint4((uint32_t)i, (uint32_t)q | ((uint32_t)(i >> 32) << 8),
                                                 (uint32_t)stream, (uint32_t)(stream >> 32)), key);
        const float u1 = ((float)r.x + 1.f) * 2.3283064e-10f, u2 = (float)r.y * 2.3283064e-10f;
        const float u3 = ((float)r.z + 1.f) * 2.3283064e-10f, u4 = (float)r.w * 2.3283064e-10f;
        const float r1 = sqrtf(-2.f * logf(u1)), r2 = sqrtf(-2.f * logf(u3));
        float s1, c1, s2, c2;
        sincospif(2.f * u2, &s1, &c1);
        sincospif(2.f * u4, &s2, &c2);
        e[(long)q * vh + i] = make_float4(r1 * c1, r1 * s1, r2 * c2, r2 * s2);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static size_t layer_smem() { return (size_t)(9 * 64 * LDW + PTC_LN * LDW) * 4; }

template <int CIN, int COUT>
static cudaError_t layer_t(const PtcGeom& g, const void* in, void* out, const void* w, int nsm, cudaStream_t st) {
    static bool cfg = false;
    if (!cfg) {
        cudaError_t e = cudaFuncSetAttribute(ptc_layer_kernel<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)layer_smem());
        if (e != cudaSuccess) return e;
        cfg = true;
    }
    const long ntiles = (g.V + PTC_LTILE - 1) / PTC_LTILE;
    const long grid = std::min<long>(ntiles, 2L * nsm);
    ptc_layer_kernel<CIN, COUT><<<(unsigned)grid, PTC_BS, layer_smem(), st>>>(
        g, reinterpret_cast<const uint4*>(in), reinterpret_cast<uint4*>(out), reinterpret_cast<const uint4*>(w),
        ntiles);
    return cudaGetLastError();
}

cudaError_t launch_ptc_layer(int cin, int cout, const PtcGeom& g, const void* in, void* out, const void* w, int nsm,
                             cudaStream_t st) {
    if (cin == 1 && cout == 8) return layer_t<1, 8>(g, in, out, w, nsm, st);
    if (cin == 8 && cout == 8) return layer_t<8, 8>(g, in, out, w, nsm, st);
    if (cin == 8 && cout == 1) return layer_t<8, 1>(g, in, out, w, nsm, st);
    if (cin == 1 && cout == 1) return layer_t<1, 1>(g, in, out, w, nsm, st);
    if (cin == 1 && cout == 2) return layer_t<1, 2>(g, in, out, w, nsm, st);
    if (cin == 2 && cout == 2) return layer_t<2, 2>(g, in, out, w, nsm, st);
    if (cin == 2 && cout == 1) return layer_t<2, 1>(g, in, out, w, nsm, st);
    if (cin == 4 && cout == 4) return layer_t<4, 4>(g, in, out, w, nsm, st);
    if (cin == 1 && cout == 4) return layer_t<1, 4>(g, in, out, w, nsm, st);
    if (cin == 4 && cout == 1) return layer_t<4, 1>(g, in, out, w, nsm, st);
    return cudaErrorInvalidValue;
}

template <int CIN, int COUT>
static cudaError_t wgrad_t(const PtcGeom& g, const void* in, const void* delta, float* partial, int nchunk,
                           cudaStream_t st) {
    const long ntiles = (g.V + PTC_TILE - 1) / PTC_TILE;
    ptc_wgrad_kernel<CIN, COUT><<<9 * nchunk, PTC_BS, 0, st>>>(g, reinterpret_cast<const uint4*>(in),
                                                               reinterpret_cast<const uint4*>(delta), partial, ntiles,
                                                               nchunk);
    return cudaGetLastError();
}

cudaError_t launch_ptc_wgrad(int cin, int cout, const PtcGeom& g, const void* in, const void* delta, float* partial,
                             int nchunk, float2* grad, float scale, cudaStream_t st) {
    cudaError_t e;
    if (cin == 1 && cout == 8) e = wgrad_t<1, 8>(g, in, delta, partial, nchunk, st);
    else if (cin == 8 && cout == 8) e = wgrad_t<8, 8>(g, in, delta, partial, nchunk, st);
    else if (cin == 8 && cout == 1) e = wgrad_t<8, 1>(g, in, delta, partial, nchunk, st);
    else if (cin == 1 && cout == 1) e = wgrad_t<1, 1>(g, in, delta, partial, nchunk, st);
    else if (cin == 1 && cout == 2) e = wgrad_t<1, 2>(g, in, delta, partial, nchunk, st);
    else if (cin == 2 && cout == 2) e = wgrad_t<2, 2>(g, in, delta, partial, nchunk, st);
    else if (cin == 2 && cout == 1) e = wgrad_t<2, 1>(g, in, delta, partial, nchunk, st);
    else if (cin == 4 && cout == 4) e = wgrad_t<4, 4>(g, in, delta, partial, nchunk, st);
    else if (cin == 1 && cout == 4) e = wgrad_t<1, 4>(g, in, delta, partial, nchunk, st);
    else if (cin == 4 && cout == 1) e = wgrad_t<4, 1>(g, in, delta, partial, nchunk, st);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    const int n = 9 * cout * cin * 16;
    ptc_wgrad_reduce<<<(n + 255) / 256, 256, 0, st>>>(partial, nchunk, cin, cout, grad, scale);
    return cudaGetLastError();
}

cudaError_t launch_ptc_embed_weights(const float2* W, int cin, int cout, void* fwd, void* adj, cudaStream_t st) {
    ptc_embed_weights<<<9 * 64 * 64 / 256, 256, 0, st>>>(W, cin, cout, reinterpret_cast<uint16_t*>(fwd),
                                                          reinterpret_cast<uint16_t*>(adj));
    return cudaGetLastError();
}

cudaError_t launch_ptc_adam(float2* W, float2* m, float2* v, float2* grad, int n, float lr, float b1, float b2,
                            float eps, int step, cudaStream_t st) {
    const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
    ptc_adam<<<(n + 255) / 256, 256, 0, st>>>(W, m, v, grad, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_ptc_embed_odd(int prec, const void* r, void* a0, const PtcGeom& g, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.V + 255) / 256);
    if (prec == P32) ptc_embed_odd<P32><<<nb, 256, 0, st>>>(r, reinterpret_cast<uint4*>(a0), g);
    else if (prec == P64) ptc_embed_odd<P64><<<nb, 256, 0, st>>>(r, reinterpret_cast<uint4*>(a0), g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_ptc_extract_odd(int prec, const void* a, void* z, const PtcGeom& g, cudaStream_t st) {
    const unsigned nb = (unsigned)((g.vh + 255) / 256);
    if (prec == P32) ptc_extract_odd<P32><<<nb, 256, 0, st>>>(reinterpret_cast<const uint4*>(a), z, g);
    else if (prec == P64) ptc_extract_odd<P64><<<nb, 256, 0, st>>>(reinterpret_cast<const uint4*>(a), z, g);
    else return cudaErrorInvalidValue;
    return cudaGetLastError();
}

cudaError_t launch_ptc_loss_delta(const void* aL, const void* e, void* delta, const PtcGeom& g, const double* ee,
                                  double* partial, double* out, cudaStream_t st) {
    const int nb = (int)((g.V + 255) / 256);
    ptc_loss_delta<<<nb, 256, 0, st>>>(reinterpret_cast<const uint4*>(aL), reinterpret_cast<const float4*>(e),
                                        reinterpret_cast<uint4*>(delta), g, ee, partial);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    sum_partials<<<1, 256, 0, st>>>(partial, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_ptc_gauss_odd(void* e, long vh, unsigned long long seed, unsigned long long stream,
                                 cudaStream_t st) {
    ptc_gauss_odd<<<(unsigned)((vh + 255) / 256), 256, 0, st>>>(reinterpret_cast<float4*>(e), vh, seed, stream);
    return cudaGetLastError();
}

}  // namespace tmk
