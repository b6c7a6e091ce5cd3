// Gauge-equivariant parallel-transport network (PTC) used as a learned
// preconditioner in flexible CG: forward layer, input- and weight-gradient
// kernels, loss, Adam, and the training-pair generator.
//
// One layer maps C_in to C_out channels of full-lattice spinor fields:
//   out^a(x) = sum_{p in P} sum_b W_p^{ab} (T_p in^b)(x),
//   P = {1, +x,+y,+z,+t, -x,-y,-z,-t},  (T_{+mu} f)(x) = U_mu(x) f(x+mu),
//   (T_{-mu} f)(x) = U_mu(x-mu)^dag f(x-mu),  W_p^{ab} a complex 4x4 spin matrix.
// Because W acts on (channel, spin) and T on (site, colour), a tile of sites is
// a real GEMM per path and colour: with every complex number split into (re, im),
//   D[site][n] += A_p[site][k] B_p[n][k],
//   n = 8 a + 2 s + re/im (output channel, spin), k = 8 b + 2 t + re/im (input),
//   B_p the real embedding [[Re W, -Im W], [Im W, Re W]] (BF16), A_p = T_p in (BF16),
//   FP32 accumulate.
// The transport (gather of neighbour activations, SU(3) multiply with paired FP32
// FMAs, links from a per-context FP16 transport-link field) fills A_p in shared
// memory; the mixing runs on the tcgen05 tensor cores with the accumulators in
// tensor memory (ptc_layer_tc).  Layers with one output channel mix first and
// transport one channel per path (ptc_layer_tc<.., MIX> + ptc_tsum).  The weight
// gradient G_p = sum_{x,c} delta(x) v_p(x)^H is the same product reduced over
// sites, also on tcgen05 (ptc_wgrad_tc); the input gradient of a layer is the
// layer run with the adjoint weights W'_p = (W_{rev p})^H (T_p^dag = T_{rev p}).
// Activations are BF16, layout [channel][3 x 16-B vectors of 4 complex (spin,
// colour)][V] in lexicographic site order.
#include "tm_internal.h"
#include "tm_kernels.h"
#include "ptc.h"

namespace tmk {

__device__ __forceinline__ float bf(uint16_t v) { return __bfloat162float(__ushort_as_bfloat16(v)); }
__device__ __forceinline__ uint16_t fb(float v) { return __bfloat16_as_ushort(__float2bfloat16_rn(v)); }
// two FP32 values rounded to nearest-even BF16 in one 32-bit word (lo in the low half)
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    uint32_t w;
    memcpy(&w, &h, 4);
    return w;
}

__device__ __forceinline__ void site_coords(const PtcGeom& g, long x, int& cx, int& cy, int& cz, int& ct) {
    long r = x;
    cx = (int)(r % g.X); r /= g.X;
    cy = (int)(r % g.Y); r /= g.Y;
    cz = (int)(r % g.Z);
    ct = (int)(r / g.Z);
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

// ---------------------------------------------------------------------------
// forward layer (also the input-gradient layer with adjoint weights) on the
// fifth-generation tensor cores.  Per tile of TC_SITES = 120 sites and per path
// p, colour c:  D_c[site][n] += A_{p,c}[site][k] * B_p[n][k]  (kind::f16, BF16
// in, FP32 accumulate in tensor memory), M = 128 rows (the last 8 unused),
// N = 8 COUT (re/im, spin, output channel), K = 8 CIN (re/im, spin, input channel).
//
// Warp roles: 15 transport warps (4 threads per site) gather and transport the
// input of one stage (one or more paths) into one of two stage buffers and
// arrive on its "full" mbarrier.  Each thread's activation words for its next
// stage are copied into a private shared-memory slot by cp.async (and its link
// words into registers) while it transports the current stage; a channel's copy
// is issued once the channel's current words have been consumed.  One MMA warp waits for
// "full", issues the stage's MMAs from one thread and commits them to the
// buffer's "empty" mbarrier, so transport and MMAs overlap.  After a tile's last
// stage the MMA warp commits to "acc_full"; all 16 warps read the accumulators
// back with tcgen05.ld (TMEM lane = site, so each thread owns one site and
// writes its output vectors directly) and arrive on "acc_empty" before the next
// tile's first MMA overwrites them.  The 9 paths' embedded weights (B) stay
// resident in shared memory.  15 + 1 warps keep 128 registers per thread (4
// warps per SM sub-partition), which a 17th warp would cut to 96.
//
// Shared-memory operand images are the canonical K-major layout without
// swizzle: core matrices of 8 rows x 16 bytes (8 BF16 along K) stored as 128
// contiguous bytes; core matrices adjacent along K are LBO = 128 bytes apart,
// 8-row groups along M/N are SBO = 128 * KCH bytes apart (KCH 16-byte K chunks,
// one per input channel: its 4 spins as (re, im) pairs).
// ---------------------------------------------------------------------------
constexpr int TC_M = 128;                  // MMA M = TMEM lanes
constexpr int TC_SITES = 120;              // sites per tile (rows 120..127 of the MMA unused)
constexpr int TC_G = 4;                    // site groups (transport threads per site)
constexpr int TC_PT = TC_G * TC_SITES;     // transport threads (15 warps)
constexpr int TC_BS = TC_PT + 32;          // + the MMA warp = 16 warps
constexpr int TC_STAGES = 2;               // transport stage buffers
constexpr long long TC_WAIT_NS = 1000000000LL;   // bound on every mbarrier wait (1 s)

// MIX: the mixing half of a layer with one output channel (see ptc_layer_mix):
// only the identity path, N = 9 paths x 8 rows (padded to 80), 9 output channels.
template <int CIN, int COUT, bool MIX = false>
struct TcShape {
    static constexpr int NPATH = MIX ? 1 : 9;                // paths transported
    static constexpr int NOUT = MIX ? 9 : COUT;              // output channels written
    static constexpr int KCH = CIN < 2 ? 2 : CIN;            // K = 8 KCH >= 16 (one MMA K step)
    static constexpr int NN = MIX ? 80 : (8 * COUT < 16 ? 16 : 8 * COUT);   // N per colour (multiple of 16)
    static constexpr int GPP = CIN < TC_G ? CIN : TC_G;      // site groups per path
    static constexpr int NPS = TC_G / GPP;                   // paths per stage (small CIN: one path per group)
    static constexpr int CPG = CIN / GPP;                    // input channels per thread
    static constexpr int NSTG = (NPATH + NPS - 1) / NPS;     // stages per tile
    static constexpr int A_COL = TC_M * 16 * KCH;            // bytes of one (path, colour) A image
    static constexpr int A_STAGE = NPS * 3 * A_COL;
    static constexpr int W_PATH = NN * 16 * KCH;             // bytes of one path's B image
    static constexpr int W_ALL = NPATH * W_PATH;
    static constexpr int TMEM_COLS = 3 * NN <= 32 ? 32 : (3 * NN <= 64 ? 64 : (3 * NN <= 128 ? 128 : 256));
    static constexpr int RAW = CPG * 3 * TC_PT * 16;         // cp.async slots: [channel][vector][thread]
    static constexpr int SMEM = W_ALL + TC_STAGES * A_STAGE + RAW + 128;   // + mbarriers, TMEM address, abort flag
    // kind::f16 instruction descriptor: D F32 (bits 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1),
    // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NN >> 3) << 17) |
                                      ((uint32_t)(TC_M >> 4) << 24);
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start, LBO, SBO (>> 4), version 1 at bit 46, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t start, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((start & 0x3FFFFu) >> 4) | ((uint64_t)((lbo & 0x3FFFFu) >> 4) << 16) |
           ((uint64_t)((sbo & 0x3FFFFu) >> 4) << 32) | (1ull << 46);
}

__device__ __forceinline__ long long global_ns() {
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_addr(b)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}

// as mbar_test, but the thread may sleep up to TC_SUSPEND_NS for the phase, so a
// waiting warp takes no issue slots from the working ones
constexpr uint32_t TC_SUSPEND_NS = 20000;
__device__ __forceinline__ bool mbar_test_sleep(uint64_t* b, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity), "r"(TC_SUSPEND_NS)
        : "memory");
    return ok != 0;
}

// Wait for the completion of the phase with this parity.  Returns false, with
// the block's abort flag set, after bound_ns or as soon as another thread has
// set the flag, so one wait that runs out ends every role of the block.  With
// abort_flag null only the time bound applies.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* abort_flag,
                                          long long bound_ns = TC_WAIT_NS) {
    if (mbar_test(b, parity)) return true;
    const long long t0 = global_ns();
    while (!mbar_test_sleep(b, parity)) {
        if (abort_flag != nullptr && *abort_flag) return false;
        if (global_ns() - t0 > bound_ns) {
            if (abort_flag != nullptr) *abort_flag = 1;
            return false;
        }
    }
    return true;
}

// Check of the bounded wait: one thread waits on an mbarrier that no thread
// arrives on.  *out = 1: the bound ran out and set the abort flag (expected);
// 0: the phase completed; 2: the wait ended without the flag.
__global__ void ptc_wait_selftest(long long bound_ns, int* out) {
    __shared__ uint64_t b;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&b, 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool done = mbar_wait(&b, 0, &abort_flag, bound_ns);
        *out = done ? 0 : (abort_flag ? 1 : 2);
    }
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tc_mma(uint32_t dtmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dtmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
        : "memory");
}

// arrive once on the mbarrier when every MMA this thread issued so far has completed
__device__ __forceinline__ void tc_commit(uint64_t* b) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_addr(b))
                 : "memory");
}

// 8 consecutive FP32 columns of this warp's 32 TMEM lanes (lane = thread)
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                 : "r"(taddr)
                 : "memory");
}

// completes the loads above; the registers are tied in so no use moves ahead of it
__device__ __forceinline__ void tmem_wait_ld(uint32_t (&a)[8], uint32_t (&b)[8], uint32_t (&c)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7]),
                   "+r"(b[0]), "+r"(b[1]), "+r"(b[2]), "+r"(b[3]), "+r"(b[4]), "+r"(b[5]), "+r"(b[6]), "+r"(b[7]),
                   "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3]), "+r"(c[4]), "+r"(c[5]), "+r"(c[6]), "+r"(c[7])
                 :
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_f32bits(uint32_t re, uint32_t im) {
    return pack2(__uint_as_float(re), __uint_as_float(im));
}

// Coordinates of one transport thread's site for the current tile (computed once
// per tile; lattices of the layer kernel have fewer than 2^31 sites).
struct TcSite {
    int x, c[4];
    bool valid;
};

__device__ __forceinline__ TcSite tc_site(const PtcGeom& g, long xl) {
    TcSite s;
    s.valid = xl < g.V;
    s.x = s.valid ? (int)xl : 0;
    int r = s.x;
    s.c[0] = r % g.X; r /= g.X;
    s.c[1] = r % g.Y; r /= g.Y;
    s.c[2] = r % g.Z;
    s.c[3] = r / g.Z;
    return s;
}

// Where one thread's transport unit (site, path p) reads: the neighbour y, the
// FP16 link words (fetched into registers one stage ahead of their use) and the
// boundary phase.  Its activation words go to shared memory by cp.async.
struct TcUnit {
    int y;
    uint32_t link[6];
    float ph;
    int flags;   // bit 0 valid, bit 1 identity path, bit 2 link daggered (backward path)
};

__device__ __forceinline__ void tc_locate(const PtcGeom& g, const TcSite& s, int p, TcUnit& f) {
    f.flags = 0;
    if (p >= 9 || !s.valid) return;
    f.y = s.x;
    f.ph = 1.f;
    if (p == 0) {
        f.flags = 3;
        return;
    }
    const int mu = (p - 1) & 3;
    const bool fwd = p <= 4;
    const int L = mu == 0 ? g.X : (mu == 1 ? g.Y : (mu == 2 ? g.Z : g.T));
    const int st = mu == 0 ? 1 : (mu == 1 ? g.X : (mu == 2 ? g.X * g.Y : g.X * g.Y * g.Z));
    const int cm = s.c[mu];
    if (fwd) {
        f.y = (cm + 1 == L) ? s.x - (L - 1) * st : s.x + st;
        if (mu == 3 && cm + 1 == L) f.ph = g.bc_t;
    } else {
        f.y = (cm == 0) ? s.x + (L - 1) * st : s.x - st;
        if (mu == 3 && cm == 0) f.ph = g.bc_t;
    }
    // the link of a forward hop lives at the site, of a backward hop at the neighbour
    // (opposite parity); checkerboard index = lexicographic index / 2
    const int par = ((s.c[0] + s.c[1] + s.c[2] + s.c[3]) & 1) ^ (fwd ? 0 : 1);
    const int owner = fwd ? s.x : f.y;
    const unsigned int* base = reinterpret_cast<const unsigned int*>(g.gauge[par]) + (owner >> 1);
#pragma unroll
    for (int k = 0; k < 6; ++k) f.link[k] = __ldg(base + (long)(mu * 6 + k) * g.vh);
    f.flags = fwd ? 1 : 5;
}

// As tc_locate, but the link comes from the transport-link field g.lp: 9 FP16
// (re, im) words of M (daggered and phased already) at the site itself.
struct TcUnitL {
    int y;
    uint32_t lw[9];
    int flags;   // bit 0 valid, bit 1 identity path
};

__device__ __forceinline__ void tc_locate_l(const PtcGeom& g, const TcSite& s, int p, TcUnitL& f) {
    f.flags = 0;
    if (p >= 9 || !s.valid) return;
    f.y = s.x;
    if (p == 0) {
        f.flags = 3;
        return;
    }
    const int mu = (p - 1) & 3;
    const int L = mu == 0 ? g.X : (mu == 1 ? g.Y : (mu == 2 ? g.Z : g.T));
    const int st = mu == 0 ? 1 : (mu == 1 ? g.X : (mu == 2 ? g.X * g.Y : g.X * g.Y * g.Z));
    const int cm = s.c[mu];
    if (p <= 4) f.y = (cm + 1 == L) ? s.x - (L - 1) * st : s.x + st;
    else f.y = (cm == 0) ? s.x + (L - 1) * st : s.x - st;
    const uint32_t* base = g.lp + (long)(p - 1) * 9 * g.V + s.x;
#pragma unroll
    for (int k = 0; k < 9; ++k) f.lw[k] = __ldg(base + (long)k * g.V);
    f.flags = 1;
}

// link words of a unit as broadcast pairs for paired FP32 FMAs: (Re M, Re M), (Im M, Im M)
__device__ __forceinline__ void tc_pairs_l(const TcUnitL& f, float2 (&mr)[9], float2 (&mi)[9]) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float2 h = h2f2<PF16>(f.lw[k]);
        mr[k] = make_float2(h.x, h.x);
        mi[k] = make_float2(h.y, h.y);
    }
}

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// SU(3) link of a located unit as 9 complex (row major; the third row rebuilt)
__device__ __forceinline__ void tc_link(const TcUnit& f, cpx<float> (&u)[9]) {
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float2 h = h2f2<PF16>(f.link[k]);
        u[k] = C(h.x, h.y);
    }
    su3_third_row(u);
}

// One channel of a unit: 12 activation words (complex (spin s, colour c) is
// word 3 s + c) -> one 16-byte chunk per colour of the A images at img (4 spins
// as BF16 (re, im) pairs): t = M v, M the path's link with its dagger and phase
// already applied.  Two spins share each paired FMA:
//   Re t = sum_d Re M Re v + Im M (-Im v),  Im t = sum_d Re M Im v + Im M Re v,
// each lane in the same order as the scalar form.
template <int A_COL>
__device__ __forceinline__ void tc_transport_channel(const uint4 (&a)[3], const float2 (&mr)[9],
                                                     const float2 (&mi)[9], uint8_t* img) {
    const uint32_t w[12] = {a[0].x, a[0].y, a[0].z, a[0].w, a[1].x, a[1].y, a[1].z, a[1].w,
                            a[2].x, a[2].y, a[2].z, a[2].w};
    uint32_t wd[3][4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {   // spins 2h, 2h + 1
        float2 vr[3], vi[3], nvi[3];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const uint32_t w0 = w[3 * (2 * h) + d], w1 = w[3 * (2 * h + 1) + d];
            vr[d] = make_float2(__uint_as_float(w0 << 16), __uint_as_float(w1 << 16));
            vi[d] = make_float2(__uint_as_float(w0 & 0xffff0000u), __uint_as_float(w1 & 0xffff0000u));
            nvi[d] = make_float2(__uint_as_float((w0 ^ 0x80000000u) & 0xffff0000u),
                                 __uint_as_float((w1 ^ 0x80000000u) & 0xffff0000u));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            float2 tr = make_float2(0.f, 0.f), ti = make_float2(0.f, 0.f);
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                tr = __ffma2_rn(mr[3 * c + d], vr[d], tr);
                tr = __ffma2_rn(mi[3 * c + d], nvi[d], tr);
                ti = __ffma2_rn(mr[3 * c + d], vi[d], ti);
                ti = __ffma2_rn(mi[3 * c + d], vr[d], ti);
            }
            wd[c][2 * h] = pack2(tr.x, ti.x);
            wd[c][2 * h + 1] = pack2(tr.y, ti.y);
        }
    }
#pragma unroll
    for (int c = 0; c < 3; ++c)
        *reinterpret_cast<uint4*>(img + c * A_COL) = make_uint4(wd[c][0], wd[c][1], wd[c][2], wd[c][3]);
}

// identity path: the words are only regrouped by colour
template <int A_COL>
__device__ __forceinline__ void tc_copy_channel(const uint4 (&a)[3], uint8_t* img) {
    const uint32_t w[12] = {a[0].x, a[0].y, a[0].z, a[0].w, a[1].x, a[1].y, a[1].z, a[1].w,
                            a[2].x, a[2].y, a[2].z, a[2].w};
#pragma unroll
    for (int c = 0; c < 3; ++c)
        *reinterpret_cast<uint4*>(img + c * A_COL) = make_uint4(w[c], w[3 + c], w[6 + c], w[9 + c]);
}

// Epilogue of one tile, run by every warp of the block: wait for the tile's
// accumulators, read this warp's TMEM lane quarter (rows 32 quarter + lane =
// sites of the tile) for its output channels, release the accumulators and
// store the BF16 output vectors.  False if the wait ran out (warp-uniform).
template <typename S, int COUT>   // COUT = output channels written
__device__ __forceinline__ bool tc_epilogue(uint32_t tmem, uint64_t* acc_full, uint64_t* acc_empty, uint32_t j,
                                            volatile int* abort_flag, int quarter, int wg, int lane, long tile,
                                            const PtcGeom& g, uint4* __restrict__ out) {
    const bool w = mbar_wait(acc_full, j & 1, abort_flag);
    if (!__all_sync(0xffffffffu, w)) return false;
    tc_fence_after();
    const int row = 32 * quarter + lane;
    const long xo = tile * TC_SITES + row;
    constexpr int CPO = (COUT + 3) / 4;                    // output channels per warp (4 warps per quarter)
    uint32_t wv[CPO][12];
#pragma unroll
    for (int k = 0; k < CPO; ++k) {
        const int a = wg * CPO + k;
        if (a < COUT) {                                     // warp-uniform
            uint32_t v0[8], v1[8], v2[8];
            const uint32_t ta = tmem + ((uint32_t)(32 * quarter) << 16) + 8 * a;
            tmem_ld8(ta, v0);
            tmem_ld8(ta + S::NN, v1);
            tmem_ld8(ta + 2 * S::NN, v2);
            tmem_wait_ld(v0, v1, v2);
            // column 8 a + 2 s + ri of colour c -> complex (s, c), word 3 s + c
#pragma unroll
            for (int s = 0; s < 4; ++s) {
                wv[k][3 * s + 0] = pack_f32bits(v0[2 * s], v0[2 * s + 1]);
                wv[k][3 * s + 1] = pack_f32bits(v1[2 * s], v1[2 * s + 1]);
                wv[k][3 * s + 2] = pack_f32bits(v2[2 * s], v2[2 * s + 1]);
            }
        }
    }
    tc_fence_before();
    mbar_arrive(acc_empty);
    if (row < TC_SITES && xo < g.V) {
#pragma unroll
        for (int k = 0; k < CPO; ++k) {
            const int a = wg * CPO + k;
            if (a < COUT) {
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    out[((long)a * 3 + q) * g.V + xo] =
                        make_uint4(wv[k][4 * q], wv[k][4 * q + 1], wv[k][4 * q + 2], wv[k][4 * q + 3]);
            }
        }
    }
    return true;
}

template <int CIN, int COUT, bool MIX>
__global__ void __launch_bounds__(TC_BS, 1) ptc_layer_tc(PtcGeom g, const uint4* __restrict__ in,
                                                        uint4* __restrict__ out, const uint4* __restrict__ wimg,
                                                        long ntiles, int* err) {
    using S = TcShape<CIN, COUT, MIX>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* Wsm = smem;                                   // 9 paths of B images
    uint8_t* Asm = smem + S::W_ALL;                        // TC_STAGES stage buffers of A images
    uint8_t* Raw = Asm + TC_STAGES * S::A_STAGE;          // activation words of each thread's next stage
    uint64_t* bar = reinterpret_cast<uint64_t*>(Raw + S::RAW);
    uint64_t* full = bar;                                  // [TC_STAGES] transport -> MMA
    uint64_t* empty = bar + TC_STAGES;                     // [TC_STAGES] MMA -> transport
    uint64_t* acc_full = bar + 2 * TC_STAGES;              // accumulators ready
    uint64_t* acc_empty = acc_full + 1;                    // accumulators read back
    uint64_t* drain = acc_full + 2;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(drain + 1);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // resident weights; the K padding chunk of one-channel inputs must read as zero
    for (int e = tid; e < S::W_ALL / 16; e += TC_BS) reinterpret_cast<uint4*>(Wsm)[e] = __ldg(wimg + e);
    if (CIN == 1) {
        for (int e = tid; e < TC_STAGES * S::NPS * 3 * TC_M; e += TC_BS) {
            const int r = e % TC_M, col = e / TC_M;   // (stage, path, colour) image, row r
            *reinterpret_cast<uint4*>(Asm + (long)col * S::A_COL + (r >> 3) * (128 * S::KCH) + 128 + (r & 7) * 16) =
                make_uint4(0u, 0u, 0u, 0u);
        }
    }
    if (tid == 0) {
        for (int k = 0; k < TC_STAGES; ++k) {
            mbar_init(full + k, TC_PT);
            mbar_init(empty + k, 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(acc_empty, TC_BS);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"((uint32_t)S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;

    const int quarter = warp & 3, wg = warp >> 2;          // epilogue: TMEM lane quarter, channel group
    if (warp == TC_PT / 32) {
        // ---- MMA warp: one thread issues; the whole warp joins each epilogue
        const uint32_t a_base = smem_addr(Asm), w_base = smem_addr(Wsm);
        constexpr uint32_t SBO = 128 * S::KCH;
        uint32_t u = 0, j = 0;
        for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
            if (lane == 0) {
                if (j > 0 && !mbar_wait(acc_empty, (j - 1) & 1, abort_flag)) ok = false;
                for (int stg = 0; stg < S::NSTG && ok; ++stg, ++u) {
                    const int buf = u % TC_STAGES;
                    if (!mbar_wait(full + buf, (u / TC_STAGES) & 1, abort_flag)) { ok = false; break; }
                    tc_fence_after();
#pragma unroll 1
                    for (int q = 0; q < S::NPS; ++q) {
                        const int pp = stg * S::NPS + q;
                        if (pp >= S::NPATH) break;
#pragma unroll
                        for (int c = 0; c < 3; ++c)
#pragma unroll
                            for (int kk = 0; kk < S::KCH / 2; ++kk) {
                                const uint32_t as = a_base + buf * S::A_STAGE + (q * 3 + c) * S::A_COL + kk * 256;
                                const uint32_t ws = w_base + pp * S::W_PATH + kk * 256;
                                tc_mma(tmem + c * S::NN, smem_desc(as, 128, SBO), smem_desc(ws, 128, SBO), S::IDESC,
                                       (pp > 0 || kk > 0) ? 1u : 0u);
                            }
                    }
                    tc_commit(empty + buf);
                }
                if (ok) tc_commit(acc_full);
            }
            ok = __shfl_sync(0xffffffffu, ok, 0);
            if (!ok) break;
            if (!tc_epilogue<S, S::NOUT>(tmem, acc_full, acc_empty, j, abort_flag, quarter, wg, lane, tile, g, out)) {
                ok = false;
                break;
            }
        }
    } else {
        // ---- transport warps
        const int r = tid % TC_SITES, grp = tid / TC_SITES;   // site r of the tile, site group
        const int pi = grp / S::GPP;                       // path slot of this group within a stage
        const int b0 = (grp % S::GPP) * S::CPG;            // first input channel of this thread
        uint32_t u = 0, j = 0;
        const uint32_t raw_base = smem_addr(Raw) + 16 * tid;
        const uint4* rawp = reinterpret_cast<const uint4*>(Raw) + tid;
        TcSite site = tc_site(g, (long)blockIdx.x * TC_SITES + r), nsite = site;
        TcUnitL nxt;
        nxt.flags = 0;
        if (pi < S::NPATH) tc_locate_l(g, site, pi, nxt);
        if (nxt.flags & 1) {
#pragma unroll
            for (int k = 0; k < S::CPG; ++k)
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    cp_async16(raw_base + (k * 3 + q) * TC_PT * 16, in + ((long)(b0 + k) * 3 + q) * g.V + nxt.y);
        }
        cp_async_commit();
        for (long tile = blockIdx.x; tile < ntiles; tile += gridDim.x, ++j) {
            for (int stg = 0; stg < S::NSTG; ++stg, ++u) {
                const int buf = u % TC_STAGES;
                const TcUnitL cur = nxt;
                {   // this thread's next stage (possibly the next tile's first)
                    const bool last = stg + 1 == S::NSTG;
                    const long nt = last ? tile + gridDim.x : tile;
                    const int np = (last ? 0 : (stg + 1) * S::NPS) + pi;
                    if (last) nsite = tc_site(g, nt * TC_SITES + r);
                    nxt.flags = 0;
                    if (nt < ntiles && np < S::NPATH) tc_locate_l(g, nsite, np, nxt);
                }
                // every lane of a warp runs the same iterations, so the vote keeps the
                // warp together on the way out and at the epilogue's aligned loads
                const bool w = u < TC_STAGES || mbar_wait(empty + buf, ((u / TC_STAGES) - 1) & 1, abort_flag);
                if (!__all_sync(0xffffffffu, w)) {
                    ok = false;
                    break;
                }
                cp_async_wait_all();
                float2 mr[9], mi[9];
                if ((cur.flags & 3) == 1) tc_pairs_l(cur, mr, mi);
                const bool copy = (cur.flags & 2) != 0;
                uint8_t* img = Asm + (long)buf * S::A_STAGE + (long)pi * 3 * S::A_COL + (r >> 3) * (128 * S::KCH) +
                               (r & 7) * 16;
#pragma unroll
                for (int k = 0; k < S::CPG; ++k) {
                    if (cur.flags & 1) {
                        uint4 a[3];
#pragma unroll
                        for (int q = 0; q < 3; ++q) a[q] = rawp[(k * 3 + q) * TC_PT];
                        uint8_t* dst = img + (b0 + k) * 128;
                        if (copy) tc_copy_channel<S::A_COL>(a, dst);
                        else tc_transport_channel<S::A_COL>(a, mr, mi, dst);
                    }
                    // the slot's current words are consumed: bring the next stage's
                    if (nxt.flags & 1) {
#pragma unroll
                        for (int q = 0; q < 3; ++q)
                            cp_async16(raw_base + (k * 3 + q) * TC_PT * 16, in + ((long)(b0 + k) * 3 + q) * g.V + nxt.y);
                    }
                }
                cp_async_commit();
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                mbar_arrive(full + buf);
            }
            if (!ok) break;
            if (!tc_epilogue<S, S::NOUT>(tmem, acc_full, acc_empty, j, abort_flag, quarter, wg, lane, tile, g, out)) {
                ok = false;
                break;
            }
        }
    }

    // drain: every copy and MMA issued by this block completes (each wait bounded,
    // also after an abort) before TMEM is released
    cp_async_wait_all();
    __syncthreads();
    if (tid == TC_PT) {
        tc_commit(drain);
        if (!mbar_wait(drain, 0, nullptr)) ok = false;
    }
    if (!ok) atomicExch(err, 1);
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::TMEM_COLS)
                     : "memory");
    }
}

// Transport links of the eight hop paths as FP16 (re, im) pairs in lexicographic
// site order: lp[(p - 1) * 9 + 3 c + d][x] = ph M[c][d], M = U_mu(x) for
// p = 1..4 (mu = p - 1) and U_mu(x - mu)^dagger for p = 5..8, ph the time
// boundary phase of the hop.  The transport kernels read the link of a (site,
// path) here (9 loads) instead of rebuilding it from the 12-real even-odd links;
// the field is rebuilt whenever the gauge field or the boundary phase changes.
__global__ void __launch_bounds__(256) ptc_links(PtcGeom g, uint32_t* __restrict__ lp) {
    const long xl = (long)blockIdx.x * 256 + threadIdx.x;
    if (xl >= g.V) return;
    const TcSite site = tc_site(g, xl);
#pragma unroll 1
    for (int p = 1; p < 9; ++p) {
        TcUnit f;
        tc_locate(g, site, p, f);
        cpx<float> u[9];
        tc_link(f, u);
        const bool dag = (f.flags & 4) != 0;
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const cpx<float> e = dag ? cj(u[3 * d + c]) : u[3 * c + d];
                lp[((long)(p - 1) * 9 + 3 * c + d) * g.V + xl] = f2h2<PF16>(f.ph * e.re, f.ph * e.im);
            }
    }
}

// ---------------------------------------------------------------------------
// Layers with one output channel and C_in > 1 (8->1, 4->1, 2->1) mix first:
// the spin-space weights commute with the colour-space transport, so
//   out(x) = sum_p T_p (sum_b W_p^{0b} in^b)(x) = sum_p (T_p z_p)(x),
// z_p = sum_b W_p^{0b} in^b at every site.  ptc_layer_tc<CIN, 1, true> computes
// the nine z_p on the tensor cores (identity path, N = 9 x 8 rows); ptc_tsum then
// transports one channel per path instead of C_in.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) ptc_tsum(PtcGeom g, const uint4* __restrict__ z, uint4* __restrict__ out) {
    const long xl = (long)blockIdx.x * 256 + threadIdx.x;
    if (xl >= g.V) return;
    const TcSite site = tc_site(g, xl);
    cpx<float> acc[12];   // complex (spin s, colour c) at 3 s + c
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        const uint4 w = __ldg(z + (long)q * g.V + xl);
        const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const float2 h = h2f2<PB16>(ws[e]);
            acc[4 * q + e] = C(h.x, h.y);
        }
    }
#pragma unroll 1
    for (int p = 1; p < 9; ++p) {
        TcUnitL f;
        tc_locate_l(g, site, p, f);
        cpx<float> u[9];   // M of the path: daggered and phased already
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 h = h2f2<PF16>(f.lw[k]);
            u[k] = C(h.x, h.y);
        }
        cpx<float> v[12];
#pragma unroll
        for (int q = 0; q < 3; ++q) {
            const uint4 w = __ldg(z + ((long)p * 3 + q) * g.V + f.y);
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 h = h2f2<PB16>(ws[e]);
                v[4 * q + e] = C(h.x, h.y);
            }
        }
#pragma unroll
        for (int sp = 0; sp < 4; ++sp)
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int d = 0; d < 3; ++d) cfma(acc[3 * sp + c], u[3 * c + d], v[3 * sp + d]);
            }
    }
#pragma unroll
    for (int q = 0; q < 3; ++q)
        out[(long)q * g.V + xl] = make_uint4(pack2(acc[4 * q].re, acc[4 * q].im), pack2(acc[4 * q + 1].re, acc[4 * q + 1].im),
                                             pack2(acc[4 * q + 2].re, acc[4 * q + 2].im),
                                             pack2(acc[4 * q + 3].re, acc[4 * q + 3].im));
}

// ---------------------------------------------------------------------------
// weight gradient on the tensor cores:
//   Q_p[m][n] = sum_{x, c} V_p[m](x, c) Delta[n](x, c),
// V_p = T_p in (rows m = 8 b + 2 t + ri: input channel b, spin t, re/im) and
// Delta the back-propagated delta (rows n = 8 a + 2 s + ri), the reduction over
// the (colour, site) pairs of the block's sites.  One MMA (M = 128) stacks the
// rows of PPM = 16 / CIN paths; NG = ceil(9 / PPM) accumulators of N = 8 COUT
// columns stay in tensor memory for the whole kernel.  A stage is (block of 32
// sites, path group): 16 transport warps, one (site, path, channel) unit per
// thread, write its A image; in a block's first stage the delta of the 32 sites
// is written too (B image, double-buffered by site block).  One MMA warp issues
// 6 MMAs of K = 16 per stage.  Both images are MN-major without swizzle: a
// 16-byte chunk holds 8 consecutive rows of one K index (k = 32 c + j), core
// matrices (8 K x 8 rows) of 128 bytes, LBO = 128 bytes between K groups, SBO =
// 12 * 128 bytes between 8-row groups.  At the end every warp reads its TMEM
// lane quarter and writes the block's partial Q_p.
// ---------------------------------------------------------------------------
constexpr int WG_S = 32;                   // sites per stage
constexpr int WG_K = 3 * WG_S;             // MMA K per stage (colour, site)
constexpr int WG_PT = 512;                 // transport threads (16 warps)
constexpr int WG_BS = WG_PT + 32;          // + the MMA warp
constexpr int WG_SBO = (WG_K / 8) * 128;   // bytes between 8-row groups of an image

template <int CIN, int COUT>
struct WgShape {
    static constexpr int PPM = 16 / CIN;                      // paths stacked per MMA
    static constexpr int NG = (9 + PPM - 1) / PPM;            // MMA groups (accumulators)
    static constexpr int NN = 8 * COUT < 16 ? 16 : 8 * COUT;  // N
    static constexpr int A_IMG = 128 / 8 * WG_SBO;            // bytes of one A image (128 rows)
    static constexpr int B_IMG = NN / 8 * WG_SBO;             // bytes of one B image
    static constexpr int RAW = 3 * WG_PT * 16;                // cp.async slots [vector][thread]
    static constexpr int COLS = NG * NN;
    static constexpr int TMEM_COLS = COLS <= 32 ? 32 : (COLS <= 64 ? 64 : (COLS <= 128 ? 128 : (COLS <= 256 ? 256 : 512)));
    static constexpr int SMEM = 2 * A_IMG + 2 * B_IMG + RAW + 128;
    // kind::f16: D F32, A and B BF16, both MN-major (bits 15, 16), N >> 3, M >> 4
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) |
                                      ((uint32_t)(NN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
};

__device__ __forceinline__ void tmem_wait_ld1(uint32_t (&a)[8]) {
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3]), "+r"(a[4]), "+r"(a[5]), "+r"(a[6]), "+r"(a[7])
                 :
                 : "memory");
}

// One (site, path, channel) unit: transport (or copy for the identity path) and
// write its 8 rows (2 t + ri) for each colour's K index as a 16-byte BF16 chunk.
__device__ __forceinline__ void wg_transport_unit(const uint4 (&a)[3], const float2 (&mr)[9], const float2 (&mi)[9],
                                                  bool copy, uint8_t* img, int j) {
    const uint32_t w[12] = {a[0].x, a[0].y, a[0].z, a[0].w, a[1].x, a[1].y, a[1].z, a[1].w,
                            a[2].x, a[2].y, a[2].z, a[2].w};
    uint32_t wd[3][4];   // [colour][spin]: (re, im) BF16
    if (copy) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int s = 0; s < 4; ++s) wd[c][s] = w[3 * s + c];
    } else {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            float2 vr[3], vi[3], nvi[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const uint32_t w0 = w[3 * (2 * h) + d], w1 = w[3 * (2 * h + 1) + d];
                vr[d] = make_float2(__uint_as_float(w0 << 16), __uint_as_float(w1 << 16));
                vi[d] = make_float2(__uint_as_float(w0 & 0xffff0000u), __uint_as_float(w1 & 0xffff0000u));
                nvi[d] = make_float2(__uint_as_float((w0 ^ 0x80000000u) & 0xffff0000u),
                                     __uint_as_float((w1 ^ 0x80000000u) & 0xffff0000u));
            }
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                float2 tr = make_float2(0.f, 0.f), ti = make_float2(0.f, 0.f);
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    tr = __ffma2_rn(mr[3 * c + d], vr[d], tr);
                    tr = __ffma2_rn(mi[3 * c + d], nvi[d], tr);
                    ti = __ffma2_rn(mr[3 * c + d], vi[d], ti);
                    ti = __ffma2_rn(mi[3 * c + d], vr[d], ti);
                }
                wd[c][2 * h] = pack2(tr.x, ti.x);
                wd[c][2 * h + 1] = pack2(tr.y, ti.y);
            }
        }
    }
    // K index k = 32 c + j: core matrix k / 8 (LBO = 128), row k % 8 (16 bytes)
#pragma unroll
    for (int c = 0; c < 3; ++c)
        *reinterpret_cast<uint4*>(img + ((WG_S * c + j) >> 3) * 128 + (j & 7) * 16) =
            make_uint4(wd[c][0], wd[c][1], wd[c][2], wd[c][3]);
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(WG_BS, 1) ptc_wgrad_tc(PtcGeom g, const uint4* __restrict__ in,
                                                        const uint4* __restrict__ delta, float* __restrict__ partial,
                                                        long nsb, int* err) {
    using S = WgShape<CIN, COUT>;
    extern __shared__ __align__(1024) uint8_t smem[];
    uint8_t* Asm = smem;                                    // 2 A images
    uint8_t* Bsm = smem + 2 * S::A_IMG;                     // 2 B images (by site-block parity)
    uint8_t* Raw = Bsm + 2 * S::B_IMG;
    uint64_t* bar = reinterpret_cast<uint64_t*>(Raw + S::RAW);
    uint64_t* full = bar;                                   // [2]
    uint64_t* empty = bar + 2;                              // [2]
    uint64_t* acc_full = bar + 4;   // every MMA of the block done
    uint64_t* drain = bar + 5;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 6);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(tslot + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // rows of absent paths (p >= 9) and the B rows beyond 8 COUT must read as zero
    for (int e = tid; e < (2 * S::A_IMG + 2 * S::B_IMG) / 16; e += WG_BS)
        reinterpret_cast<uint4*>(smem)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (tid == 0) {
        for (int k = 0; k < 2; ++k) {
            mbar_init(full + k, WG_PT);
            mbar_init(empty + k, 1);
        }
        mbar_init(acc_full, 1);
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        __syncwarp();
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(tslot)),
                     "r"((uint32_t)S::TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tslot;
    bool ok = true;
    // this block's site blocks (every block gets at least one: gridDim.x <= nsb)
    const long sb0 = blockIdx.x * nsb / gridDim.x, sb1 = (blockIdx.x + 1) * nsb / gridDim.x;
    const int nst = (int)(sb1 > sb0 ? (sb1 - sb0) * S::NG : 0);

    if (warp == WG_PT / 32) {
        // ---- MMA warp
        if (lane == 0) {
            const uint32_t a_base = smem_addr(Asm), b_base = smem_addr(Bsm);
            for (int u = 0; u < nst; ++u) {
                const int buf = u & 1, grp = u % S::NG, sbi = u / S::NG;
                if (!mbar_wait(full + buf, (u >> 1) & 1, abort_flag)) { ok = false; break; }
                tc_fence_after();
#pragma unroll
                for (int kk = 0; kk < WG_K / 16; ++kk) {
                    const uint32_t as = a_base + buf * S::A_IMG + kk * 256;
                    const uint32_t bs = b_base + (sbi & 1) * S::B_IMG + kk * 256;
                    tc_mma(tmem + grp * S::NN, smem_desc(as, 128, WG_SBO), smem_desc(bs, 128, WG_SBO), S::IDESC,
                           (sbi > 0 || kk > 0) ? 1u : 0u);
                }
                tc_commit(empty + buf);
            }
            if (ok) tc_commit(acc_full);
        }
        ok = __shfl_sync(0xffffffffu, ok, 0);
    } else {
        // ---- transport warps: unit (site j, path slot ps, channel b)
        const int j = tid % WG_S, unit = tid / WG_S;        // unit < 16
        const int ps = unit / CIN, b = unit % CIN;
        const uint32_t raw_base = smem_addr(Raw) + 16 * tid;
        const uint4* rawp = reinterpret_cast<const uint4*>(Raw) + tid;
        // site coordinates change once per site block (every NG stages)
        TcSite lsite;
        long lsb = -1;
        auto locate = [&](int u, TcUnitL& f) {
            f.flags = 0;
            if (u >= nst) return;
            const int grp = u % S::NG;
            const long sb = sb0 + u / S::NG;
            if (sb != lsb) {
                lsite = tc_site(g, sb * WG_S + j);
                lsb = sb;
            }
            tc_locate_l(g, lsite, grp * S::PPM + ps, f);
        };
        TcUnitL nxt;
        locate(0, nxt);
        if (nxt.flags & 1) {
#pragma unroll
            for (int q = 0; q < 3; ++q) cp_async16(raw_base + q * WG_PT * 16, in + ((long)b * 3 + q) * g.V + nxt.y);
        }
        cp_async_commit();
        for (int u = 0; u < nst; ++u) {
            const int buf = u & 1, grp = u % S::NG, sbi = u / S::NG;
            const TcUnitL cur = nxt;
            locate(u + 1, nxt);
            const bool w = u < 2 || mbar_wait(empty + buf, ((u >> 1) - 1) & 1, abort_flag);
            if (!__all_sync(0xffffffffu, w)) { ok = false; break; }
            // the delta of this site block (first stage of the block; its B buffer was
            // last read by MMAs that completed before the empty wait above)
            if (grp == 0 && tid < WG_S * COUT) {
                const int a = tid / WG_S;
                const long x = (sb0 + sbi) * WG_S + j;
                uint8_t* bimg = Bsm + (sbi & 1) * S::B_IMG + a * WG_SBO;
                uint32_t wd[12];
                if (x < g.V) {
#pragma unroll
                    for (int q = 0; q < 3; ++q) {
                        const uint4 v = __ldg(delta + ((long)a * 3 + q) * g.V + x);
                        wd[4 * q] = v.x; wd[4 * q + 1] = v.y; wd[4 * q + 2] = v.z; wd[4 * q + 3] = v.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 12; ++q) wd[q] = 0u;
                }
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    *reinterpret_cast<uint4*>(bimg + ((WG_S * c + j) >> 3) * 128 + (j & 7) * 16) =
                        make_uint4(wd[c], wd[3 + c], wd[6 + c], wd[9 + c]);
            }
            cp_async_wait_all();
            uint8_t* img = Asm + buf * S::A_IMG + unit * WG_SBO;
            if (cur.flags & 1) {
                uint4 a[3];
#pragma unroll
                for (int q = 0; q < 3; ++q) a[q] = rawp[q * WG_PT];
                float2 mr[9], mi[9];
                const bool copy = (cur.flags & 2) != 0;
                if (!copy) tc_pairs_l(cur, mr, mi);
                wg_transport_unit(a, mr, mi, copy, img, j);
            } else {
                // no site or no path: zero rows (an earlier stage may have left values)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                    *reinterpret_cast<uint4*>(img + ((WG_S * c + j) >> 3) * 128 + (j & 7) * 16) =
                        make_uint4(0u, 0u, 0u, 0u);
            }
            if (nxt.flags & 1) {
#pragma unroll
                for (int q = 0; q < 3; ++q) cp_async16(raw_base + q * WG_PT * 16, in + ((long)b * 3 + q) * g.V + nxt.y);
            }
            cp_async_commit();
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive(full + buf);
        }
    }

    // read back: this warp's lane quarter (rows m = 32 quarter + lane), its quarter
    // of the columns of every group; partial[block][p][n][m'] with m' = row of path p
    if (ok && nst > 0) {
        const bool w = mbar_wait(acc_full, 0, abort_flag);
        if (__all_sync(0xffffffffu, w)) {
            tc_fence_after();
            const int quarter = warp & 3, wq = warp >> 2;      // the MMA warp (wq = 4) reads nothing
            const int m = 32 * quarter + lane, ps = m / (8 * CIN), mr8 = m % (8 * CIN);
            constexpr int CW = S::NN / 4 < 8 ? 8 : S::NN / 4;  // columns per warp (x8 loads)
            for (int grp = 0; grp < S::NG; ++grp) {
                const int p = grp * S::PPM + ps;
                for (int c0 = wq * CW; c0 < (wq + 1) * CW && c0 < S::NN && wq < 4; c0 += 8) {
                    uint32_t v0[8];
                    tmem_ld8(tmem + ((uint32_t)(32 * quarter) << 16) + grp * S::NN + c0, v0);
                    tmem_wait_ld1(v0);
                    if (p < 9) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) {
                            const int n = c0 + e;
                            if (n < 8 * COUT)
                                partial[(((long)blockIdx.x * 9 + p) * 64 + n) * 64 + mr8] = __uint_as_float(v0[e]);
                        }
                    }
                }
            }
        } else {
            ok = false;
        }
    }

    // drain: copies and MMAs complete (bounded) before TMEM is released
    cp_async_wait_all();
    tc_fence_before();
    __syncthreads();
    if (tid == WG_PT) {
        tc_commit(drain);
        if (!mbar_wait(drain, 0, nullptr)) ok = false;
    }
    if (!ok) atomicExch(err, 1);
    __syncthreads();
    if (warp == 0) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)S::TMEM_COLS)
                     : "memory");
    }
}

// G[p][a][b][s][t] (complex) += scale * combination of the summed partials
// Q_p[n][m] (n = 8 a + 2 s + ri of the delta, m = 8 b + 2 t + ri' of T_p in):
//   Re G = Q[re][re] + Q[im][im],  Im G = Q[im][re] - Q[re][im]   (delta conj(v))
__global__ void ptc_wgrad_reduce(const float* __restrict__ partial, int nblk, int cin, int cout, float2* grad,
                                 float scale) {
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    const int n = 9 * cout * cin * 16;
    if (e >= n) return;
    int r = e;
    const int t = r & 3; r >>= 2;
    const int s = r & 3; r >>= 2;
    const int b = r % cin; r /= cin;
    const int a = r % cout;
    const int p = r / cout;
    const int nre = 8 * a + 2 * s, mre = 8 * b + 2 * t;
    double rr = 0, ii = 0, ir = 0, ri = 0;
    for (int c = 0; c < nblk; ++c) {
        const float* q = partial + ((size_t)c * 9 + p) * 4096;
        rr += q[nre * 64 + mre];
        ii += q[(nre + 1) * 64 + mre + 1];
        ir += q[(nre + 1) * 64 + mre];
        ri += q[nre * 64 + mre + 1];
    }
    grad[e].x += scale * (float)(rr + ii);
    grad[e].y += scale * (float)(ir - ri);
}

// ---------------------------------------------------------------------------
// weights: FP32 complex master [9][cout][cin][4][4] -> BF16 real embeddings
// ---------------------------------------------------------------------------
__device__ __forceinline__ int rev_path(int p) { return p == 0 ? 0 : (p <= 4 ? p + 4 : p - 4); }

// B image of one layer for ptc_layer_tc, layer shape cin_l -> cout_l: per path p,
// row n = 8 a + 2 s + ri (output channel a, spin s, re/im) and K index
// k = 8 b + 2 t + ri' (input channel b, spin t, re/im), stored as
// [p][n / 8][k / 8][n % 8][k % 8] BF16 with NN = max(16, 8 cout_l) rows and
// 8 max(2, cin_l) K entries, zero beyond the layer's channels.  Real embedding of
// the complex weight w: (re, re) -> Re w, (re, im) -> -Im w, (im, re) -> Im w,
// (im, im) -> Re w.  The adjoint image (input gradient) is the layer cout -> cin
// with W'_p[b][a][t][s] = conj(W_{rev p}[a][b][s][t]).
__global__ void ptc_embed_weights(const float2* __restrict__ W, int cin, int cout, int adjoint, uint16_t* img) {
    const int cin_l = adjoint ? cout : cin, cout_l = adjoint ? cin : cout;
    // a layer with fewer output than input channels (one output channel) mixes
    // first: one B image whose rows are n = 8 p + 2 s + ri over the 9 paths
    const bool mix = cin_l > cout_l;
    const int kch = cin_l < 2 ? 2 : cin_l, nn = mix ? 80 : (8 * cout_l < 16 ? 16 : 8 * cout_l);
    const int per_path = nn * 8 * kch;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (mix ? 1 : 9) * per_path) return;
    const int pb = e / per_path;
    int rem = e - pb * per_path;
    const int kr = rem & 7; rem >>= 3;   // k % 8
    const int nr = rem & 7; rem >>= 3;   // n % 8
    const int kc = rem % kch;            // k / 8
    const int ng = rem / kch;            // n / 8
    const int n = 8 * ng + nr, k = 8 * kc + kr;
    const int p = mix ? (n >> 3) : pb;                       // path
    const int ao = mix ? 0 : (n >> 3), so = (n >> 1) & 3, rim = n & 1;   // output channel, spin, re/im
    const int bi = k >> 3, si = (k >> 1) & 3, cim = k & 1;   // input channel, spin, re/im
    float v = 0.f;
    if (p < 9 && ao < cout_l && bi < cin_l) {
        float2 w;
        if (!adjoint) {
            w = W[(((p * cout + ao) * cin + bi) * 4 + so) * 4 + si];
        } else {
            const float2 w0 = W[(((rev_path(p) * cout + bi) * cin + ao) * 4 + si) * 4 + so];
            w = make_float2(w0.x, -w0.y);
        }
        v = (rim == cim) ? w.x : (rim == 0 ? -w.y : w.y);
    }
    img[e] = fb(v);
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
template <int CIN, int COUT, bool MIX = false>
static cudaError_t layer_t(const PtcGeom& g, const void* in, void* out, const void* w, int nsm, int* err,
                           cudaStream_t st) {
    using S = TcShape<CIN, COUT, MIX>;
    static_assert(S::SMEM <= 227 * 1024, "layer shared memory");
    if (g.V >= (1L << 31)) return cudaErrorInvalidValue;   // site indices of the layer kernel are 32-bit
    static int cfg_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (cfg_dev != dev) {
        e = cudaFuncSetAttribute(ptc_layer_tc<CIN, COUT, MIX>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
        if (e != cudaSuccess) return e;
        cfg_dev = dev;
    }
    const long ntiles = (g.V + TC_SITES - 1) / TC_SITES;
    const long grid = std::min<long>(ntiles, nsm);
    ptc_layer_tc<CIN, COUT, MIX><<<(unsigned)grid, TC_BS, S::SMEM, st>>>(
        g, reinterpret_cast<const uint4*>(in), reinterpret_cast<uint4*>(out), reinterpret_cast<const uint4*>(w),
        ntiles, err);
    return cudaGetLastError();
}

template <int CIN>
static cudaError_t mixed_first(const PtcGeom& g, const void* in, void* out, const void* w, int nsm, int* err,
                               void* zbuf, cudaStream_t st) {
    cudaError_t e = layer_t<CIN, 1, true>(g, in, zbuf, w, nsm, err, st);
    if (e != cudaSuccess) return e;
    ptc_tsum<<<(unsigned)((g.V + 255) / 256), 256, 0, st>>>(g, reinterpret_cast<const uint4*>(zbuf),
                                                           reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

cudaError_t launch_ptc_layer(int cin, int cout, const PtcGeom& g, const void* in, void* out, const void* w, int nsm,
                             int* err, void* zbuf, cudaStream_t st) {
    if (cin == 1 && cout == 8) return layer_t<1, 8>(g, in, out, w, nsm, err, st);
    if (cin == 8 && cout == 8) return layer_t<8, 8>(g, in, out, w, nsm, err, st);
    if (cin == 8 && cout == 1) return mixed_first<8>(g, in, out, w, nsm, err, zbuf, st);
    if (cin == 1 && cout == 1) return layer_t<1, 1>(g, in, out, w, nsm, err, st);
    if (cin == 1 && cout == 2) return layer_t<1, 2>(g, in, out, w, nsm, err, st);
    if (cin == 2 && cout == 2) return layer_t<2, 2>(g, in, out, w, nsm, err, st);
    if (cin == 2 && cout == 1) return mixed_first<2>(g, in, out, w, nsm, err, zbuf, st);
    if (cin == 4 && cout == 4) return layer_t<4, 4>(g, in, out, w, nsm, err, st);
    if (cin == 1 && cout == 4) return layer_t<1, 4>(g, in, out, w, nsm, err, st);
    if (cin == 4 && cout == 1) return mixed_first<4>(g, in, out, w, nsm, err, zbuf, st);
    return cudaErrorInvalidValue;
}

template <int CIN, int COUT>
static cudaError_t wgrad_t(const PtcGeom& g, const void* in, const void* delta, float* partial, int nblk, int* err,
                           cudaStream_t st) {
    using S = WgShape<CIN, COUT>;
    // a block that allocates all 512 TMEM columns must be alone on its SM: ask for
    // more shared memory than two blocks could share
    constexpr int SMEM = S::TMEM_COLS == 512 && S::SMEM < 120 * 1024 ? 120 * 1024 : S::SMEM;
    static_assert(SMEM <= 227 * 1024, "weight-gradient shared memory");
    if (g.V >= (1L << 31)) return cudaErrorInvalidValue;
    static int cfg_dev = -1;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (cfg_dev != dev) {
        e = cudaFuncSetAttribute(ptc_wgrad_tc<CIN, COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM);
        if (e != cudaSuccess) return e;
        cfg_dev = dev;
    }
    const long nsb = (g.V + WG_S - 1) / WG_S;
    ptc_wgrad_tc<CIN, COUT><<<nblk, WG_BS, SMEM, st>>>(g, reinterpret_cast<const uint4*>(in),
                                                       reinterpret_cast<const uint4*>(delta), partial, nsb, err);
    return cudaGetLastError();
}

cudaError_t launch_ptc_wgrad(int cin, int cout, const PtcGeom& g, const void* in, const void* delta, float* partial,
                             int nsm, float2* grad, float scale, int* err, cudaStream_t st) {
    const long nsb = (g.V + WG_S - 1) / WG_S;
    const int nblk = (int)std::min<long>(nsm, nsb);
    cudaError_t e;
    if (cin == 1 && cout == 8) e = wgrad_t<1, 8>(g, in, delta, partial, nblk, err, st);
    else if (cin == 8 && cout == 8) e = wgrad_t<8, 8>(g, in, delta, partial, nblk, err, st);
    else if (cin == 8 && cout == 1) e = wgrad_t<8, 1>(g, in, delta, partial, nblk, err, st);
    else if (cin == 1 && cout == 1) e = wgrad_t<1, 1>(g, in, delta, partial, nblk, err, st);
    else if (cin == 1 && cout == 2) e = wgrad_t<1, 2>(g, in, delta, partial, nblk, err, st);
    else if (cin == 2 && cout == 2) e = wgrad_t<2, 2>(g, in, delta, partial, nblk, err, st);
    else if (cin == 2 && cout == 1) e = wgrad_t<2, 1>(g, in, delta, partial, nblk, err, st);
    else if (cin == 4 && cout == 4) e = wgrad_t<4, 4>(g, in, delta, partial, nblk, err, st);
    else if (cin == 1 && cout == 4) e = wgrad_t<1, 4>(g, in, delta, partial, nblk, err, st);
    else if (cin == 4 && cout == 1) e = wgrad_t<4, 1>(g, in, delta, partial, nblk, err, st);
    else return cudaErrorInvalidValue;
    if (e != cudaSuccess) return e;
    const int n = 9 * cout * cin * 16;
    ptc_wgrad_reduce<<<(n + 255) / 256, 256, 0, st>>>(partial, nblk, cin, cout, grad, scale);
    return cudaGetLastError();
}

cudaError_t launch_ptc_embed_weights(const float2* W, int cin, int cout, void* fwd, void* adj, cudaStream_t st) {
    ptc_embed_weights<<<9 * 64 * 64 / 256, 256, 0, st>>>(W, cin, cout, 0, reinterpret_cast<uint16_t*>(fwd));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    ptc_embed_weights<<<9 * 64 * 64 / 256, 256, 0, st>>>(W, cin, cout, 1, reinterpret_cast<uint16_t*>(adj));
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

cudaError_t launch_ptc_links(const PtcGeom& g, uint32_t* lp, cudaStream_t st) {
    ptc_links<<<(unsigned)((g.V + 255) / 256), 256, 0, st>>>(g, lp);
    return cudaGetLastError();
}

cudaError_t launch_ptc_wait_selftest(long long bound_ns, int* out, cudaStream_t st) {
    ptc_wait_selftest<<<1, 32, 0, st>>>(bound_ns, out);
    return cudaGetLastError();
}

cudaError_t launch_ptc_gauss_odd(void* e, long vh, unsigned long long seed, unsigned long long stream,
                                 cudaStream_t st) {
    ptc_gauss_odd<<<(unsigned)((vh + 255) / 256), 256, 0, st>>>(reinterpret_cast<float4*>(e), vh, seed, stream);
    return cudaGetLastError();
}

}  // namespace tmk
