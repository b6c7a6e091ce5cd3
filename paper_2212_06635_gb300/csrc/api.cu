// C ABI of include/tm.h: context and gauge-state tracking (Sec. 3), operator
// application (eq:hQpm, eq:hQh), CG and mixed-precision CG with reliable
// updates (Sec. 4.1), multishift CG with shift-by-shift refinement (Sec. 4.2),
// batched solves and power iteration.  All arithmetic runs in the kernels of
// dslash.cu, blas.cu and gauge.cu; this file only allocates, orders launches and
// reads back solver control words.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <numeric>
#include <vector>
#include <mutex>
#include <map>
#include <string>

#include "force.h"
#include "rational.h"
#include "tm_host.h"
#include "ptc.h"

using namespace tmk;

namespace tmk {
cudaError_t launch_gauge_import(void* d0, void* d1, const double* src, const Geom& g, cudaStream_t st);
cudaError_t launch_clover(const Geom& g, const void* g0, const void* g1, int par, double kappa, double csw,
                          double mu_t, double mubar_t, double epsbar_t, double* outA, double* outB,
                          double* outH, cudaStream_t st);
cudaError_t launch_clover_unpack(double* out, const double* A, long vh, cudaStream_t st);
}  // namespace tmk

// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
static thread_local char g_err[512] = "";

static tm_status fail(tm_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}

#define CK(...)                                                                               \
    do {                                                                                      \
        cudaError_t e_ = (__VA_ARGS__);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? TM_ERR_OOM : TM_ERR_CUDA, "%s: %s (%s:%d)", \
                        #__VA_ARGS__, cudaGetErrorString(e_), __FILE__, __LINE__);                   \
    } while (0)
#define CKS(...)                             \
    do {                                     \
        tm_status s_ = (__VA_ARGS__);               \
        if (s_ != TM_OK) return s_;          \
    } while (0)

extern "C" const char* tm_last_error(void) { return g_err; }

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
static inline cudaStream_t S(void* s) { return reinterpret_cast<cudaStream_t>(s); }
static inline int nblk(long vh, int bs) { return (int)((vh + bs - 1) / bs); }
static inline int nflav(tm_op op) { return (op == TM_QH || op == TM_QH_DAG || op == TM_QH_SQ) ? 2 : 1; }
static inline bool is_what(tm_op op) { return op == TM_WHAT_PLUS || op == TM_WHAT_MINUS || op == TM_WHAT_SQ; }

static bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// native fields live in device memory: a host pointer handed to a kernel would
// fault the GPU, so the entry points reject it first
static bool device_fields(const void* a, const void* b = nullptr) {
    return is_device_ptr(a) && (b == nullptr || is_device_ptr(b));
}

// pinned (page-locked or registered) host memory: copies from / to it stay
// asynchronous, so the field calls need not synchronise
static bool is_pinned_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// next staging buffer of a ring, ordered after the work that last used it
static tm_status io_slot(tm_ctx::IoRing& r, size_t bytes, cudaStream_t st, int* slot) {
    if (r.bytes < bytes) {
        for (int k = 0; k < tm_ctx::IoRing::N; ++k) {
            if (r.free[k]) CK(cudaEventSynchronize(r.free[k]));
            cudaFree(r.buf[k]);
            r.buf[k] = nullptr;
        }
        r.bytes = 0;
        for (int k = 0; k < tm_ctx::IoRing::N; ++k) {
            CK(cudaMalloc(&r.buf[k], bytes));
            if (!r.free[k]) CK(cudaEventCreateWithFlags(&r.free[k], cudaEventDisableTiming));
        }
        r.bytes = bytes;
    }
    const int k = r.next;
    r.next = (r.next + 1) % tm_ctx::IoRing::N;
    CK(cudaStreamWaitEvent(st, r.free[k], 0));   // no-op until the event is first recorded
    *slot = k;
    return TM_OK;
}

static tm_status ws_get(tm_ctx* c, int id, size_t bytes, void** out) {
    auto it = c->ws.find(id);
    if (it != c->ws.end() && it->second.second >= bytes) {
        *out = it->second.first;
        return TM_OK;
    }
    if (it != c->ws.end()) {
        cudaFree(it->second.first);
        c->ws.erase(it);
    }
    void* p = nullptr;
    CK(cudaMalloc(&p, bytes));
    c->ws[id] = {p, bytes};
    *out = p;
    return TM_OK;
}

enum WsId {
    WS_B64 = 1, WS_X64, WS_R64, WS_AX64, WS_TE64, WS_MID64, WS_V64,
    WS_TE_S, WS_MID_S, WS_R_S, WS_P_S, WS_AP_S, WS_X_S,
    WS_STAGE_B, WS_STAGE_X, WS_STAGE_G, WS_APPLY_TE, WS_APPLY_MID, WS_STAGE_IO, WS_TUNE,
    WS_FCG_Z, WS_XDF,
    WS_MS_X = 100, WS_MS_P = 200, WS_MS_X64 = 300, WS_RAT = 400
};

// ---------------------------------------------------------------------------
// context
// ---------------------------------------------------------------------------
extern "C" tm_status tm_create(tm_ctx** out, const int dims[4], int device) {
    if (!out || !dims) return fail(TM_ERR_ARG, "tm_create: null argument");
    for (int k = 0; k < 4; ++k)
        if (dims[k] < 2 || dims[k] % 2) return fail(TM_ERR_ARG, "tm_create: extent %d = %d must be even and >= 2", k, dims[k]);
    if ((double)dims[0] * dims[1] * dims[2] * dims[3] >= 2147483648.0)
        return fail(TM_ERR_ARG, "tm_create: the volume must be below 2^31 sites");
    CK(cudaSetDevice(device));
    static std::atomic<unsigned long long> next_uid{1};
    tm_ctx* c = new tm_ctx();
    c->uid = next_uid.fetch_add(1);
    c->device = device;
    geom_init(c->g, dims[0], dims[1], dims[2], dims[3]);
    c->vh = c->g.vh;
    c->max_blocks = nblk(c->vh, MIN_BS);
    cudaError_t e = cudaSuccess;
    e = e ? e : cudaStreamCreateWithFlags(&c->sstream, cudaStreamNonBlocking);
    e = e ? e : cudaMalloc(&c->partial, sizeof(double) * c->max_blocks);
    e = e ? e : cudaMalloc(&c->counter, sizeof(unsigned int) * 4);
    e = e ? e : cudaMemset(c->counter, 0, sizeof(unsigned int) * 4);
    e = e ? e : cudaMalloc(&c->ctl, sizeof(SolverCtl));
    e = e ? e : cudaMemset(c->ctl, 0, sizeof(SolverCtl));
    e = e ? e : cudaMalloc(&c->ms, sizeof(MsCtl));
    e = e ? e : cudaMallocHost(&c->h_ctl, sizeof(SolverCtl));
    e = e ? e : cudaMallocHost(&c->h_ms, sizeof(MsCtl));
    e = e ? e : cudaMalloc(&c->d_scal, sizeof(double) * 16);
    e = e ? e : cudaMallocHost(&c->h_scal, sizeof(double) * 16);
    if (e != cudaSuccess) {
        tm_destroy(c);
        return fail(e == cudaErrorMemoryAllocation ? TM_ERR_OOM : TM_ERR_CUDA, "tm_create: %s", cudaGetErrorString(e));
    }
    *out = c;
    return TM_OK;
}

extern "C" tm_status tm_destroy(tm_ctx* c) {
    if (!c) return TM_OK;
    cudaSetDevice(c->device);
    if (c->sstream) cudaStreamSynchronize(c->sstream);
    for (int p = 0; p < 2; ++p) { cudaFree(c->gauge64[p]); cudaFree(c->clovA64[p]); }
    for (int q = 0; q < 4; ++q) {
        cudaFree(c->gaugeP[q][0]); cudaFree(c->gaugeP[q][1]);
        cudaFree(c->clovAP[q]); cudaFree(c->clovBP[q]); cudaFree(c->clovHP[q]); cudaFree(c->clovAeP[q]);
    }
    cudaFree(c->clovB64); cudaFree(c->clovH64);
    cudaFree(c->gaugeDF[0]); cudaFree(c->gaugeDF[1]);
    for (int k = 0; k < 3; ++k) cudaFree(c->clovDF[k]);
    cudaFree(c->partial); cudaFree(c->counter); cudaFree(c->ctl); cudaFree(c->ms); cudaFree(c->d_scal);
    cudaFreeHost(c->h_ctl); cudaFreeHost(c->h_ms); cudaFreeHost(c->h_scal);
    for (auto& kv : c->ws) cudaFree(kv.second.first);
    for (tm_ctx::IoRing* r : {&c->io_in, &c->io_out})
        for (int k = 0; k < tm_ctx::IoRing::N; ++k) {
            if (r->free[k]) {
                cudaEventSynchronize(r->free[k]);
                cudaEventDestroy(r->free[k]);
            }
            cudaFree(r->buf[k]);
        }
    if (c->sstream) cudaStreamDestroy(c->sstream);
    delete c;
    return TM_OK;
}

// ---------------------------------------------------------------------------
// gauge field and its derived objects (Sec. 3 state cascade)
// ---------------------------------------------------------------------------
extern "C" tm_status tm_gauge_load(tm_ctx* c, const double* links, double gauge_id, void* stream) {
    if (!c || !links) return fail(TM_ERR_ARG, "tm_gauge_load: null argument");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    const size_t canon = (size_t)2 * c->vh * 4 * 18 * sizeof(double);
    for (int p = 0; p < 2; ++p)
        if (!c->gauge64[p]) CK(cudaMalloc(&c->gauge64[p], link_bytes_parity(P64, c->vh)));
    const double* src = links;
    if (!is_device_ptr(links)) {
        void* stage = nullptr;
        CKS(ws_get(c, WS_STAGE_G, canon, &stage));
        CK(cudaMemcpyAsync(stage, links, canon, cudaMemcpyHostToDevice, st));
        src = reinterpret_cast<const double*>(stage);
    }
    CK(launch_gauge_import(c->gauge64[0], c->gauge64[1], src, c->g, st));
    if (src != links) {
        CK(cudaStreamSynchronize(st));
        auto it = c->ws.find(WS_STAGE_G);
        cudaFree(it->second.first);
        c->ws.erase(it);
    }
    c->gauge_id = gauge_id;
    c->gauge_gen += 1;   // every derived object is now stale
    return TM_OK;
}

extern "C" tm_status tm_gauge_id(const tm_ctx* c, double* id) {
    if (!c || !id) return fail(TM_ERR_ARG, "tm_gauge_id: null argument");
    *id = c->gauge_id;
    return TM_OK;
}

// parameters the clover term and its inverses depend on (rho does not enter them)
static bool same_params(const tm_params& a, const tm_params& b) {
    return a.kappa == b.kappa && a.csw == b.csw && a.mu == b.mu && a.mubar == b.mubar &&
           a.epsbar == b.epsbar && a.bc_t == b.bc_t;
}

extern "C" tm_status tm_clover_compute(tm_ctx* c, const tm_params* prm, void* stream) {
    if (!c || !prm) return fail(TM_ERR_ARG, "tm_clover_compute: null argument");
    if (c->gauge_gen == 0) return fail(TM_ERR_STALE, "tm_clover_compute: no gauge field loaded");
    if (prm->bc_t != 1 && prm->bc_t != -1) return fail(TM_ERR_ARG, "tm_clover_compute: bc_t must be +1 or -1");
    if (!(prm->kappa > 0.0)) return fail(TM_ERR_ARG, "tm_clover_compute: kappa must be positive");
    CK(cudaSetDevice(c->device));
    if (c->clover_gauge_gen == c->gauge_gen && same_params(c->params, *prm)) {
        c->params.rho = prm->rho;   // W_hat's rho leaves the clover inverse unchanged (Sec. 2)
        return TM_OK;
    }
    const cudaStream_t st = S(stream);
    const long vh = c->vh;
    const bool heavy = prm->mubar != 0.0 || prm->epsbar != 0.0;
    for (int p = 0; p < 2; ++p)
        if (!c->clovA64[p]) CK(cudaMalloc(&c->clovA64[p], sizeof(double) * CLOV_ODD_REALS * vh));
    if (!c->clovB64) CK(cudaMalloc(&c->clovB64, sizeof(double) * CLOV_EVEN_LIGHT_REALS * vh));
    if (heavy && !c->clovH64) CK(cudaMalloc(&c->clovH64, sizeof(double) * CLOV_EVEN_HEAVY_REALS * vh));
    const double k = prm->kappa;
    CK(launch_clover(c->g, c->gauge64[0], c->gauge64[1], 0, k, prm->csw, 2 * k * prm->mu, 2 * k * prm->mubar,
                     2 * k * prm->epsbar, c->clovA64[0], c->clovB64, heavy ? c->clovH64 : nullptr, st));
    CK(launch_clover(c->g, c->gauge64[0], c->gauge64[1], 1, k, prm->csw, 0.0, 0.0, 0.0, c->clovA64[1], nullptr,
                     nullptr, st));
    c->params = *prm;
    c->have_heavy = heavy;
    c->clover_gauge_gen = c->gauge_gen;
    c->clover_stamp += 1;
    return TM_OK;
}

extern "C" tm_status tm_clover_export(tm_ctx* c, int parity, double* out, void* stream) {
    if (!c || !out || (parity != 0 && parity != 1)) return fail(TM_ERR_ARG, "tm_clover_export: bad argument");
    if (c->clover_gauge_gen != c->gauge_gen) return fail(TM_ERR_STALE, "tm_clover_export: clover term is stale");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    const size_t bytes = sizeof(double) * 2 * 2 * 36 * c->vh;
    if (is_device_ptr(out)) {
        CK(launch_clover_unpack(out, c->clovA64[parity], c->vh, st));
    } else {
        void* tmp = nullptr;
        CK(cudaMalloc(&tmp, bytes));
        CK(launch_clover_unpack(reinterpret_cast<double*>(tmp), c->clovA64[parity], c->vh, st));
        CK(cudaMemcpyAsync(out, tmp, bytes, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        cudaFree(tmp);
    }
    return TM_OK;
}

// make sure the links and clover terms exist in storage precision P
static tm_status ensure_prec(tm_ctx* c, int P, cudaStream_t st) {
    if (c->clover_gauge_gen != c->gauge_gen || c->gauge_gen == 0)
        return fail(TM_ERR_STALE, "clover term is stale: call tm_clover_compute after tm_gauge_load");
    if (P == P64) return TM_OK;
    const long vh = c->vh;
    if (c->gaugeP_gen[P] != c->gauge_gen) {
        for (int p = 0; p < 2; ++p) {
            if (!c->gaugeP[P][p]) CK(cudaMalloc(&c->gaugeP[P][p], link_bytes_parity(P, vh)));
            cudaError_t e = P == P32 ? launch_links_from64<P32>(c->gaugeP[P][p], c->gauge64[p], vh, st)
                          : P == PB16 ? launch_links_from64<PB16>(c->gaugeP[P][p], c->gauge64[p], vh, st)
                                      : launch_links_from64<PF16>(c->gaugeP[P][p], c->gauge64[p], vh, st);
            CK(e);
        }
        c->gaugeP_gen[P] = c->gauge_gen;
    }
    if (c->clovP_stamp[P] != c->clover_stamp) {
        const size_t esz = prec_esz(P);
        auto conv = [&](void** dst, const double* src, int nreal) -> tm_status {
            if (!*dst) CK(cudaMalloc(dst, esz * nreal * vh));
            cudaError_t e = P == P32 ? launch_clover_from64<P32>(*dst, src, vh, nreal, st)
                          : P == PB16 ? launch_clover_from64<PB16>(*dst, src, vh, nreal, st)
                                      : launch_clover_from64<PF16>(*dst, src, vh, nreal, st);
            CK(e);
            return TM_OK;
        };
        CKS(conv(&c->clovAP[P], c->clovA64[1], CLOV_ODD_REALS));
        CKS(conv(&c->clovBP[P], c->clovB64, CLOV_EVEN_LIGHT_REALS));
        if (c->have_heavy) CKS(conv(&c->clovHP[P], c->clovH64, CLOV_EVEN_HEAVY_REALS));
        c->clovP_stamp[P] = c->clover_stamp;
    }
    return TM_OK;
}

// double-word copies of the FP64 links and clover arrays (made when stale)
static tm_status ensure_df(tm_ctx* c, cudaStream_t st) {
    CKS(ensure_prec(c, P64, st));
    const long vh = c->vh;
    if (c->gaugeDF_gen != c->gauge_gen) {
        for (int p = 0; p < 2; ++p) {
            if (!c->gaugeDF[p]) CK(cudaMalloc(&c->gaugeDF[p], link_bytes_parity(PDF, vh)));
            CK(launch_f64_to_df(c->gaugeDF[p], c->gauge64[p], 4 * 9 * vh, st));
        }
        c->gaugeDF_gen = c->gauge_gen;
    }
    if (c->clovDF_stamp != c->clover_stamp) {
        const double* src[3] = {c->clovA64[1], c->clovB64, c->clovH64};
        const int nreal[3] = {CLOV_ODD_REALS, CLOV_EVEN_LIGHT_REALS, CLOV_EVEN_HEAVY_REALS};
        for (int k = 0; k < 3; ++k) {
            if (k == 2 && !c->have_heavy) continue;
            if (!c->clovDF[k]) CK(cudaMalloc(&c->clovDF[k], (size_t)8 * nreal[k] * vh));
            CK(launch_f64_to_df(c->clovDF[k], src[k], (long)nreal[k] / 2 * vh, st));
        }
        c->clovDF_stamp = c->clover_stamp;
    }
    return TM_OK;
}

static const void* gauge_ptr(const tm_ctx* c, int P, int par) {
    return P == P64 ? c->gauge64[par] : P == PDF ? c->gaugeDF[par] : c->gaugeP[P][par];
}
static const void* clovA_ptr(const tm_ctx* c, int P) {
    return P == P64 ? (const void*)c->clovA64[1] : P == PDF ? c->clovDF[0] : c->clovAP[P];
}
static const void* clovB_ptr(const tm_ctx* c, int P) {
    return P == P64 ? (const void*)c->clovB64 : P == PDF ? c->clovDF[1] : c->clovBP[P];
}
static const void* clovH_ptr(const tm_ctx* c, int P) {
    return P == P64 ? (const void*)c->clovH64 : P == PDF ? c->clovDF[2] : c->clovHP[P];
}

// ---------------------------------------------------------------------------
// operator application
// ---------------------------------------------------------------------------
// blocks of a pass: one thread per site, except the direct two-flavour even pass
// (a thread per site and flavour)
static int pass_nblk(long vh, int nf, int kind, int staged) {
    return staged ? nblk(vh, STAGED_BS) : nblk(nf == 2 && kind == K1_EO_INV ? 2 * vh : vh, DSLASH_BS);
}

// launch one pass in the variant the context chose for (P, NF, KIND)
template <int P, int NF, int KIND, int NP>
static cudaError_t launch_pass(int variant, const OpBatch<NP>& b, int nb, cudaStream_t st) {
    if constexpr (P != P64 && P != PDF) {
        if (variant) return launch_dslash_staged<P, NF, KIND, NP>(b, nb, st);
    }
    return launch_dslash<P, NF, KIND, NP>(b, nb, st);
}

static OpProb make_prob(const tm_ctx* c, int P, int nf, int kind, int sign, void* out, const void* in,
                        const void* loc, SolverCtl* ctl, bool fuse, double rho = 0.0) {
    OpProb p{};
    p.g = c->g;
    // (the double-word passes run a thread per site and flavour)
    p.nblk = P == PDF ? nblk((long)nf * c->vh, DSLASH_BS) : pass_nblk(c->vh, nf, kind, c->variant[P][nf - 1][kind]);
    p.bc_t = (float)c->params.bc_t;
    p.gauge[0] = gauge_ptr(c, P, 0);
    p.gauge[1] = gauge_ptr(c, P, 1);
    p.clov = kind == K1_EO_INV ? (nf == 1 ? clovB_ptr(c, P) : clovH_ptr(c, P)) : clovA_ptr(c, P);
    p.in = in;
    p.loc = loc;
    p.out = out;
    const double k = c->params.kappa;
    p.kappa = k;
    p.tw = sign * 2.0 * k * (nf == 1 ? c->params.mu : c->params.mubar);
    p.eps = 2.0 * k * c->params.epsbar;
    p.rho = kind == K2_OE_LOCAL ? rho : 0.0;
    p.sign = sign;
    p.ctl = ctl;
    p.ms = c->ms;
    p.partial = fuse ? c->partial : nullptr;
    p.counter = c->counter;
    return p;
}

// out = Q_hat(sign) in (+ i rho in for W_hat), via the even temporary te.
// fin != FIN_NONE fuses ||out||^2.
template <int P, int NF>
static cudaError_t schur(const tm_ctx* c, int sign, void* out, const void* in, void* te, cudaStream_t st,
                         SolverCtl* ctl, int fin, double rho = 0.0) {
    OpBatch<1> b{};
    b.n = 1;
    b.fin = FIN_NONE;
    b.p[0] = make_prob(c, P, NF, K1_EO_INV, sign, te, in, nullptr, ctl, false);
    b.blk_start[0] = 0;
    b.blk_start[1] = b.p[0].nblk;
    const int v1 = P == PDF ? 0 : c->variant[P][NF - 1][K1_EO_INV];
    const int v2 = P == PDF ? 0 : c->variant[P][NF - 1][K2_OE_LOCAL];
    cudaError_t e = launch_pass<P, NF, K1_EO_INV, 1>(v1, b, b.p[0].nblk, st);
    if (e != cudaSuccess) return e;
    b.fin = fin;
    b.p[0] = make_prob(c, P, NF, K2_OE_LOCAL, sign, out, te, in, ctl, fin != FIN_NONE, rho);
    b.blk_start[1] = b.p[0].nblk;
    return launch_pass<P, NF, K2_OE_LOCAL, 1>(v2, b, b.p[0].nblk, st);
}

// signs of the two factors of a normal operator (first applied first)
static void normal_signs(tm_op op, int* s1, int* s2) {
    if (op == TM_MDAGM || op == TM_WHAT_SQ) { *s1 = +1; *s2 = -1; }   // Q- Q+, W- W+
    else if (op == TM_QPQM) { *s1 = -1; *s2 = +1; }    // Q+ Q-
    else { *s1 = -1; *s2 = +1; }                       // Qh Qh^+
}

// out = A in for a normal op, fin fused into the first factor (||Q in||^2 = <in, A in>)
template <int P, int NF>
static cudaError_t normal_op(const tm_ctx* c, tm_op op, void* out, const void* in, void* mid, void* te,
                             cudaStream_t st, SolverCtl* ctl, int fin) {
    int s1, s2;
    normal_signs(op, &s1, &s2);
    const double rt = is_what(op) ? 2.0 * c->params.kappa * c->params.rho : 0.0;
    cudaError_t e = schur<P, NF>(c, s1, mid, in, te, st, ctl, fin, s1 * rt);
    if (e != cudaSuccess) return e;
    return schur<P, NF>(c, s2, out, mid, te, st, ctl, FIN_NONE, s2 * rt);
}

template <int P, int NF>
static tm_status apply_t(tm_ctx* c, tm_op op, void* out, const void* in, cudaStream_t st) {
    void *te = nullptr, *mid = nullptr;
    CKS(ws_get(c, WS_APPLY_TE, spinor_bytes(P, 12 * NF, c->vh), &te));
    if (op == TM_QHAT_PLUS || op == TM_QH) {
        CK(schur<P, NF>(c, +1, out, in, te, st, nullptr, FIN_NONE));
    } else if (op == TM_QHAT_MINUS || op == TM_QH_DAG) {
        CK(schur<P, NF>(c, -1, out, in, te, st, nullptr, FIN_NONE));
    } else if (op == TM_WHAT_PLUS || op == TM_WHAT_MINUS) {
        const int sg = op == TM_WHAT_PLUS ? +1 : -1;
        CK(schur<P, NF>(c, sg, out, in, te, st, nullptr, FIN_NONE, sg * 2.0 * c->params.kappa * c->params.rho));
    } else {
        CKS(ws_get(c, WS_APPLY_MID, spinor_bytes(P, 12 * NF, c->vh), &mid));
        CK(normal_op<P, NF>(c, op, out, in, mid, te, st, nullptr, FIN_NONE));
    }
    return TM_OK;
}

// Reliable-update threshold when the caller gives none: about the square root of
// the sloppy storage's unit roundoff, so that the recursively updated residual is
// replaced by the FP64 one before its accumulated rounding (~eps relative to the
// residual at the last update) reaches ~sqrt(eps) of the current residual.
// Measured at 32^3x64 (mixed CG to 1e-10): FP16 0.02 -> 0.195 s (0.1: 0.226 s),
// FP32 0.002 -> 0.216 s (0.1: 0.279 s).
static double default_delta(int sloppy) {
    switch (sloppy) {
        case TM_F16: return 0.02;   // eps = 2^-11
        case TM_BF16: return 0.06;  // eps = 2^-8
        default: return 0.002;      // FP32
    }
}

static tm_status check_prec(int p) {
    if (p < TM_F64 || p > TM_F16) return fail(TM_ERR_ARG, "unknown precision %d", p);
    return TM_OK;
}

extern "C" tm_status tm_apply_Mhat(tm_ctx* c, tm_op op, tm_prec prec, void* out, const void* in, void* stream) {
    if (!c || !out || !in || out == in) return fail(TM_ERR_ARG, "tm_apply_Mhat: bad pointers");
    if (((uintptr_t)out | (uintptr_t)in) & 15) return fail(TM_ERR_ARG, "tm_apply_Mhat: fields must be 16-byte aligned");
    if (op < TM_QHAT_PLUS || op > TM_WHAT_SQ) return fail(TM_ERR_ARG, "tm_apply_Mhat: unknown op %d", (int)op);
    CKS(check_prec(prec));
    if (!device_fields(out, in)) return fail(TM_ERR_ARG, "tm_apply_Mhat: fields must be device pointers");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    CKS(ensure_prec(c, prec, st));
    if (nflav(op) == 2 && !c->have_heavy)
        return fail(TM_ERR_ARG, "tm_apply_Mhat: heavy operator needs mubar or epsbar in tm_clover_compute");
    const bool h = nflav(op) == 2;
    switch (prec) {
        case TM_F64: return h ? apply_t<P64, 2>(c, op, out, in, st) : apply_t<P64, 1>(c, op, out, in, st);
        case TM_F32: return h ? apply_t<P32, 2>(c, op, out, in, st) : apply_t<P32, 1>(c, op, out, in, st);
        case TM_BF16: return h ? apply_t<PB16, 2>(c, op, out, in, st) : apply_t<PB16, 1>(c, op, out, in, st);
        case TM_F16: return h ? apply_t<PF16, 2>(c, op, out, in, st) : apply_t<PF16, 1>(c, op, out, in, st);
    }
    return fail(TM_ERR_ARG, "tm_apply_Mhat: unknown precision");
}

// op(in) in double-word arithmetic on native FP64 fields (out doubles as the
// double-word result and is converted in place)
template <int NF>
static tm_status apply_dw_t(tm_ctx* c, tm_op op, void* out, const void* in, cudaStream_t st) {
    const long n16 = 12 * NF * c->vh;
    void* xdf = nullptr;
    CKS(ensure_df(c, st));
    CKS(ws_get(c, WS_XDF, spinor_bytes(PDF, 12 * NF, c->vh), &xdf));
    CK(launch_f64_to_df(xdf, in, n16, st));
    CKS(apply_t<PDF, NF>(c, op, out, xdf, st));
    CK(launch_df_to_f64(out, out, n16, st));
    return TM_OK;
}

extern "C" tm_status tm_apply_Mhat_dw(tm_ctx* c, tm_op op, void* out, const void* in, void* stream) {
    if (!c || !out || !in || out == in) return fail(TM_ERR_ARG, "tm_apply_Mhat_dw: bad pointers");
    if (((uintptr_t)out | (uintptr_t)in) & 15) return fail(TM_ERR_ARG, "tm_apply_Mhat_dw: fields must be 16-byte aligned");
    if (op < TM_QHAT_PLUS || op > TM_WHAT_SQ) return fail(TM_ERR_ARG, "tm_apply_Mhat_dw: unknown op %d", (int)op);
    if (!device_fields(out, in)) return fail(TM_ERR_ARG, "tm_apply_Mhat_dw: fields must be device pointers");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    CKS(ensure_prec(c, P64, st));
    if (nflav(op) == 2 && !c->have_heavy)
        return fail(TM_ERR_ARG, "tm_apply_Mhat_dw: heavy operator needs mubar or epsbar in tm_clover_compute");
    return nflav(op) == 2 ? apply_dw_t<2>(c, op, out, in, st) : apply_dw_t<1>(c, op, out, in, st);
}

// the even pass alone: out (even sites) = M_ee(sign)^-1 H_eo in (odd sites)
template <int P, int NF>
static cudaError_t even_t(const tm_ctx* c, int sign, void* out, const void* in, cudaStream_t st) {
    OpBatch<1> b{};
    b.n = 1;
    b.fin = FIN_NONE;
    b.p[0] = make_prob(c, P, NF, K1_EO_INV, sign, out, in, nullptr, nullptr, false);
    b.blk_start[0] = 0;
    b.blk_start[1] = b.p[0].nblk;
    return launch_pass<P, NF, K1_EO_INV, 1>(c->variant[P][NF - 1][K1_EO_INV], b, b.p[0].nblk, st);
}

extern "C" tm_status tm_apply_even(tm_ctx* c, tm_op op, tm_prec prec, void* out, const void* in, void* stream) {
    if (!c || !out || !in || out == in) return fail(TM_ERR_ARG, "tm_apply_even: bad pointers");
    if (((uintptr_t)out | (uintptr_t)in) & 15) return fail(TM_ERR_ARG, "tm_apply_even: fields must be 16-byte aligned");
    if (op != TM_QHAT_PLUS && op != TM_QHAT_MINUS && op != TM_QH && op != TM_QH_DAG)
        return fail(TM_ERR_ARG, "tm_apply_even: op must be a single Schur operator");
    CKS(check_prec(prec));
    if (!device_fields(out, in)) return fail(TM_ERR_ARG, "tm_apply_even: fields must be device pointers");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    CKS(ensure_prec(c, prec, st));
    const int nf = nflav(op);
    if (nf == 2 && !c->have_heavy)
        return fail(TM_ERR_ARG, "tm_apply_even: heavy operator needs mubar or epsbar in tm_clover_compute");
    const int sign = (op == TM_QHAT_PLUS || op == TM_QH) ? +1 : -1;
    const bool h = nf == 2;
    switch (prec) {
        case TM_F64: CK(h ? even_t<P64, 2>(c, sign, out, in, st) : even_t<P64, 1>(c, sign, out, in, st)); break;
        case TM_F32: CK(h ? even_t<P32, 2>(c, sign, out, in, st) : even_t<P32, 1>(c, sign, out, in, st)); break;
        case TM_BF16: CK(h ? even_t<PB16, 2>(c, sign, out, in, st) : even_t<PB16, 1>(c, sign, out, in, st)); break;
        case TM_F16: CK(h ? even_t<PF16, 2>(c, sign, out, in, st) : even_t<PF16, 1>(c, sign, out, in, st)); break;
    }
    return TM_OK;
}

// ---------------------------------------------------------------------------
// fields
// ---------------------------------------------------------------------------
extern "C" tm_status tm_field_bytes(const tm_ctx* c, tm_prec prec, int nf, size_t* bytes) {
    if (!c || !bytes || (nf != 1 && nf != 2)) return fail(TM_ERR_ARG, "tm_field_bytes: bad argument");
    CKS(check_prec(prec));
    *bytes = spinor_bytes(prec, 12 * nf, c->vh);
    return TM_OK;
}

template <int P>
static cudaError_t import_t(int nf, void* d, const double* s, long vh, cudaStream_t st) {
    return nf == 1 ? launch_import<P, 12>(d, s, vh, st) : launch_import<P, 24>(d, s, vh, st);
}
template <int P>
static cudaError_t export_t(int nf, double* d, const void* s, long vh, cudaStream_t st) {
    return nf == 1 ? launch_export<P, 12>(d, s, vh, st) : launch_export<P, 24>(d, s, vh, st);
}

static cudaError_t import_any(int prec, int nf, void* d, const double* s, long vh, cudaStream_t st) {
    switch (prec) {
        case P64: return import_t<P64>(nf, d, s, vh, st);
        case P32: return import_t<P32>(nf, d, s, vh, st);
        case PB16: return import_t<PB16>(nf, d, s, vh, st);
        default: return import_t<PF16>(nf, d, s, vh, st);
    }
}
static cudaError_t export_any(int prec, int nf, double* d, const void* s, long vh, cudaStream_t st) {
    switch (prec) {
        case P64: return export_t<P64>(nf, d, s, vh, st);
        case P32: return export_t<P32>(nf, d, s, vh, st);
        case PB16: return export_t<PB16>(nf, d, s, vh, st);
        default: return export_t<PF16>(nf, d, s, vh, st);
    }
}

extern "C" tm_status tm_field_import(tm_ctx* c, tm_prec prec, int nf, void* dst, const double* src, void* stream) {
    if (!c || !dst || !src || (nf != 1 && nf != 2)) return fail(TM_ERR_ARG, "tm_field_import: bad argument");
    if (((uintptr_t)dst | (uintptr_t)src) & 15) return fail(TM_ERR_ARG, "tm_field_import: pointers must be 16-byte aligned");
    CKS(check_prec(prec));
    if (!device_fields(dst)) return fail(TM_ERR_ARG, "tm_field_import: the native field must be a device pointer");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    if (is_device_ptr(src)) {
        CK(import_any(prec, nf, dst, src, c->vh, st));
        return TM_OK;
    }
    const size_t bytes = sizeof(double) * 24 * nf * c->vh;
    int k = 0;
    CKS(io_slot(c->io_in, bytes, st, &k));
    void* stage = c->io_in.buf[k];
    CK(cudaMemcpyAsync(stage, src, bytes, cudaMemcpyHostToDevice, st));
    CK(import_any(prec, nf, dst, reinterpret_cast<const double*>(stage), c->vh, st));
    CK(cudaEventRecord(c->io_in.free[k], st));
    if (!is_pinned_host(src)) CK(cudaStreamSynchronize(st));
    return TM_OK;
}

extern "C" tm_status tm_field_export(tm_ctx* c, tm_prec prec, int nf, double* dst, const void* src, void* stream) {
    if (!c || !dst || !src || (nf != 1 && nf != 2)) return fail(TM_ERR_ARG, "tm_field_export: bad argument");
    if (((uintptr_t)dst | (uintptr_t)src) & 15) return fail(TM_ERR_ARG, "tm_field_export: pointers must be 16-byte aligned");
    CKS(check_prec(prec));
    if (!device_fields(src)) return fail(TM_ERR_ARG, "tm_field_export: the native field must be a device pointer");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    if (is_device_ptr(dst)) {
        CK(export_any(prec, nf, dst, src, c->vh, st));
        return TM_OK;
    }
    const size_t bytes = sizeof(double) * 24 * nf * c->vh;
    int k = 0;
    CKS(io_slot(c->io_out, bytes, st, &k));
    void* stage = c->io_out.buf[k];
    CK(export_any(prec, nf, reinterpret_cast<double*>(stage), src, c->vh, st));
    CK(cudaMemcpyAsync(dst, stage, bytes, cudaMemcpyDeviceToHost, st));
    CK(cudaEventRecord(c->io_out.free[k], st));
    if (!is_pinned_host(dst)) CK(cudaStreamSynchronize(st));
    return TM_OK;
}

template <int P, int NF>
static tm_status kernel_times_t(tm_ctx* c, int sign, const void* in, int reps, double* ms, cudaStream_t st,
                                int v1, int v2) {
    void *te = nullptr, *out = nullptr;
    CKS(ws_get(c, WS_APPLY_TE, spinor_bytes(P, 12 * NF, c->vh), &te));
    CKS(ws_get(c, WS_APPLY_MID, spinor_bytes(P, 12 * NF, c->vh), &out));
    OpBatch<1> b{};
    b.n = 1;
    b.fin = FIN_NONE;
    b.blk_start[0] = 0;
    cudaEvent_t e0, e1, e2;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    CK(cudaEventCreate(&e2));
    b.p[0] = make_prob(c, P, NF, K1_EO_INV, sign, te, in, nullptr, nullptr, false);
    int nb = b.p[0].nblk = pass_nblk(c->vh, NF, K1_EO_INV, v1);
    b.blk_start[1] = nb;
    CK((launch_pass<P, NF, K1_EO_INV, 1>(v1, b, nb, st)));   // warm-up
    CK(cudaEventRecord(e0, st));
    for (int r = 0; r < reps; ++r) CK((launch_pass<P, NF, K1_EO_INV, 1>(v1, b, nb, st)));
    CK(cudaEventRecord(e1, st));
    b.p[0] = make_prob(c, P, NF, K2_OE_LOCAL, sign, out, te, in, nullptr, false);
    nb = b.p[0].nblk = pass_nblk(c->vh, NF, K2_OE_LOCAL, v2);
    b.blk_start[1] = nb;
    for (int r = 0; r < reps; ++r) CK((launch_pass<P, NF, K2_OE_LOCAL, 1>(v2, b, nb, st)));
    CK(cudaEventRecord(e2, st));
    CK(cudaEventSynchronize(e2));
    float t1 = 0, t2 = 0;
    CK(cudaEventElapsedTime(&t1, e0, e1));
    CK(cudaEventElapsedTime(&t2, e1, e2));
    ms[0] = t1 / reps;
    ms[1] = t2 / reps;
    cudaEventDestroy(e0); cudaEventDestroy(e1); cudaEventDestroy(e2);
    return TM_OK;
}

static tm_status kernel_times_any(tm_ctx* c, int prec, int nf, int sign, const void* in, int reps, double* ms,
                                  cudaStream_t st, int v1, int v2) {
    if (nf == 2) {
        switch (prec) {
            case TM_F64: return kernel_times_t<P64, 2>(c, sign, in, reps, ms, st, 0, 0);
            case TM_F32: return kernel_times_t<P32, 2>(c, sign, in, reps, ms, st, v1, v2);
            case TM_BF16: return kernel_times_t<PB16, 2>(c, sign, in, reps, ms, st, v1, v2);
            default: return kernel_times_t<PF16, 2>(c, sign, in, reps, ms, st, v1, v2);
        }
    }
    switch (prec) {
        case TM_F64: return kernel_times_t<P64, 1>(c, sign, in, reps, ms, st, 0, 0);
        case TM_F32: return kernel_times_t<P32, 1>(c, sign, in, reps, ms, st, v1, v2);
        case TM_BF16: return kernel_times_t<PB16, 1>(c, sign, in, reps, ms, st, v1, v2);
        default: return kernel_times_t<PF16, 1>(c, sign, in, reps, ms, st, v1, v2);
    }
}

extern "C" tm_status tm_kernel_times(tm_ctx* c, tm_op op, tm_prec prec, const void* in, int reps, double* ms,
                                     void* stream) {
    if (!c || !in || !ms || reps < 1) return fail(TM_ERR_ARG, "tm_kernel_times: bad argument");
    if (op != TM_QHAT_PLUS && op != TM_QHAT_MINUS && op != TM_QH && op != TM_QH_DAG)
        return fail(TM_ERR_ARG, "tm_kernel_times: op must be a single Schur operator");
    CKS(check_prec(prec));
    if (!device_fields(in)) return fail(TM_ERR_ARG, "tm_kernel_times: in must be a device pointer");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    CKS(ensure_prec(c, prec, st));
    const int sign = (op == TM_QHAT_PLUS || op == TM_QH) ? +1 : -1;
    const int nf = nflav(op);
    if (nf == 2 && !c->have_heavy) return fail(TM_ERR_ARG, "tm_kernel_times: no heavy clover term");
    return kernel_times_any(c, prec, nf, sign, in, reps, ms, st, c->variant[prec][nf - 1][0],
                            c->variant[prec][nf - 1][1]);
}

// ---------------------------------------------------------------------------
// force outer products of the hopping term (Sec. 4.3, rational-approximation force)
// ---------------------------------------------------------------------------
extern "C" tm_status tm_force_outer(tm_ctx* c, tm_prec prec, int nf, int n, const double* coeff,
                                    const void* const* x, const void* const* y, int gamma5_y, double* force,
                                    void* stream) {
    if (!c || !force) return fail(TM_ERR_ARG, "tm_force_outer: bad pointers");
    if (nf != 1 && nf != 2) return fail(TM_ERR_ARG, "tm_force_outer: nflavour must be 1 or 2");
    if (n < 0 || n > FORCE_MAXN) return fail(TM_ERR_ARG, "tm_force_outer: n = %d outside [0, %d]", n, FORCE_MAXN);
    if (prec != TM_F32 && prec != TM_BF16 && prec != TM_F16)
        return fail(TM_ERR_ARG, "tm_force_outer: fields must be TM_F32, TM_BF16 or TM_F16");
    if ((uintptr_t)force & 15) return fail(TM_ERR_ARG, "tm_force_outer: force must be 16-byte aligned");
    if (n > 0 && (!coeff || !x || !y)) return fail(TM_ERR_ARG, "tm_force_outer: bad pointers");
    CK(cudaSetDevice(c->device));
    if (!is_device_ptr(force)) return fail(TM_ERR_ARG, "tm_force_outer: force must be a device pointer");
    ForceArgs a{};
    a.g = c->g;
    a.n = n;
    for (int k = 0; k < n; ++k) {
        for (int p = 0; p < 2; ++p) {
            const void* xp = x[2 * k + p];
            const void* yp = y[2 * k + p];
            if (!xp || !yp || (((uintptr_t)xp | (uintptr_t)yp) & 15))
                return fail(TM_ERR_ARG, "tm_force_outer: field pair %d parity %d: null or misaligned", k, p);
            if (!is_device_ptr(xp) || !is_device_ptr(yp))
                return fail(TM_ERR_ARG, "tm_force_outer: field pair %d parity %d: not a device pointer", k, p);
            a.x[k][p] = xp;
            a.y[k][p] = yp;
        }
        a.c[k] = (float)coeff[k];
    }
    const cudaStream_t st = S(stream);
    CKS(ensure_prec(c, P32, st));   // FP32 links (and the boundary phase of tm_clover_compute)
    if (n == 0) return TM_OK;
    a.bc_t = (float)c->params.bc_t;
    a.gauge[0] = c->gaugeP[P32][0];
    a.gauge[1] = c->gaugeP[P32][1];
    a.force = force;
    a.g5y = gamma5_y ? 1 : 0;
    CK(launch_force_outer(prec, nf, a, st));
    return TM_OK;
}

// ---------------------------------------------------------------------------
// autotuner: per (lattice, precision, flavours) pick the faster stencil variant
// of each pass by timing both on this context's own fields; results are kept in
// the context and, if TM_TUNE_CACHE names a file, in a text cache keyed by
// "X Y Z T prec nflavour" so later processes skip the timing.
// ---------------------------------------------------------------------------
static bool tune_cache_lookup(const tm_ctx* c, int prec, int nf, tm_tuning* t) {
    const char* path = getenv("TM_TUNE_CACHE");
    if (!path || !*path) return false;
    FILE* f = fopen(path, "r");
    if (!f) return false;
    int X, Y, Z, T, p, n, a, b;
    bool found = false;
    while (fscanf(f, "%d %d %d %d %d %d %d %d", &X, &Y, &Z, &T, &p, &n, &a, &b) == 8) {
        if (X == c->g.X && Y == c->g.Y && Z == c->g.Z && T == c->g.T && p == prec && n == nf) {
            t->even_pass = a;
            t->odd_pass = b;
            found = true;
        }
    }
    fclose(f);
    return found;
}

static void tune_cache_store(const tm_ctx* c, int prec, int nf, const tm_tuning* t) {
    const char* path = getenv("TM_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%d %d %d %d %d %d %d %d\n", c->g.X, c->g.Y, c->g.Z, c->g.T, prec, nf, t->even_pass, t->odd_pass);
    fclose(f);
}

static tm_status check_tuning(int prec, int nf, const tm_tuning* t) {
    if (nf != 1 && nf != 2) return fail(TM_ERR_ARG, "tuning: nflavour must be 1 or 2");
    if ((t->even_pass != 0 && t->even_pass != 1) || (t->odd_pass != 0 && t->odd_pass != 1))
        return fail(TM_ERR_ARG, "tuning: variants are 0 (direct) or 1 (staged)");
    if (prec == TM_F64 && (t->even_pass || t->odd_pass))
        return fail(TM_ERR_UNSUPPORTED, "tuning: the staged variant has no FP64 form");
    return TM_OK;
}

extern "C" tm_status tm_set_tuning(tm_ctx* c, tm_prec prec, int nf, const tm_tuning* t) {
    if (!c || !t) return fail(TM_ERR_ARG, "tm_set_tuning: null argument");
    CKS(check_prec(prec));
    CKS(check_tuning(prec, nf, t));
    c->variant[prec][nf - 1][0] = t->even_pass;
    c->variant[prec][nf - 1][1] = t->odd_pass;
    return TM_OK;
}

extern "C" tm_status tm_get_tuning(const tm_ctx* c, tm_prec prec, int nf, tm_tuning* t) {
    if (!c || !t || (nf != 1 && nf != 2)) return fail(TM_ERR_ARG, "tm_get_tuning: bad argument");
    CKS(check_prec(prec));
    t->even_pass = c->variant[prec][nf - 1][0];
    t->odd_pass = c->variant[prec][nf - 1][1];
    return TM_OK;
}

extern "C" tm_status tm_autotune(tm_ctx* c, tm_prec prec, int nf, tm_tuning* chosen, void* stream) {
    if (!c || (nf != 1 && nf != 2)) return fail(TM_ERR_ARG, "tm_autotune: bad argument");
    CKS(check_prec(prec));
    CK(cudaSetDevice(c->device));
    tm_tuning t{0, 0};
    if (prec != TM_F64 && !tune_cache_lookup(c, prec, nf, &t)) {
        if (nf == 2 && !c->have_heavy) return fail(TM_ERR_ARG, "tm_autotune: no heavy clover term");
        const cudaStream_t st = S(stream);
        CKS(ensure_prec(c, prec, st));
        void* f = nullptr;
        CKS(ws_get(c, WS_TUNE, spinor_bytes(prec, 12 * nf, c->vh), &f));
        void* canon = nullptr;
        const size_t cb = sizeof(double) * 24 * nf * c->vh;
        CKS(ws_get(c, WS_STAGE_IO, cb, &canon));
        CK(cudaMemsetAsync(canon, 0, cb, st));
        CK(import_any(prec, nf, f, reinterpret_cast<const double*>(canon), c->vh, st));
        double direct[2], staged[2];
        const int reps = c->vh >= (1 << 18) ? 5 : 20;
        CKS(kernel_times_any(c, prec, nf, +1, f, reps, direct, st, 0, 0));
        CKS(kernel_times_any(c, prec, nf, +1, f, reps, staged, st, 1, 1));
        t.even_pass = staged[0] < direct[0] ? 1 : 0;
        t.odd_pass = staged[1] < direct[1] ? 1 : 0;
        tune_cache_store(c, prec, nf, &t);
    }
    c->variant[prec][nf - 1][0] = t.even_pass;
    c->variant[prec][nf - 1][1] = t.odd_pass;
    if (chosen) *chosen = t;
    return TM_OK;
}

// ---------------------------------------------------------------------------
// solver building blocks (single problem)
// ---------------------------------------------------------------------------
static VecBatch<1> vb1(const tm_ctx* c, void* v0, void* v1 = nullptr, void* v2 = nullptr, void* v3 = nullptr,
                       double* dst = nullptr) {
    VecBatch<1> b{};
    b.n = 1;
    const int nb = nblk(c->vh, BLAS_BS);
    b.blk_start[0] = 0;
    b.blk_start[1] = nb;
    VecProb& p = b.p[0];
    p.vh = c->vh;
    p.nblk = nb;
    p.v[0] = v0; p.v[1] = v1; p.v[2] = v2; p.v[3] = v3;
    p.ctl = c->ctl;
    p.ms = c->ms;
    p.partial = c->partial;
    p.counter = c->counter;
    p.dst = dst;
    return b;
}

template <int P>
static cudaError_t norm2_t(tm_ctx* c, int nf, const void* f, double* res, cudaStream_t st) {
    VecBatch<1> b = vb1(c, const_cast<void*>(f), nullptr, nullptr, nullptr, res);
    return nf == 1 ? launch_norm2<P, 12, 1>(b, nblk(c->vh, BLAS_BS), st)
                   : launch_norm2<P, 24, 1>(b, nblk(c->vh, BLAS_BS), st);
}

extern "C" tm_status tm_field_norm2(tm_ctx* c, tm_prec prec, int nf, const void* field, double* result,
                                    void* stream) {
    if (!c || !field || !result || (nf != 1 && nf != 2)) return fail(TM_ERR_ARG, "tm_field_norm2: bad argument");
    if (((uintptr_t)field & 15) || ((uintptr_t)result & 7))
        return fail(TM_ERR_ARG, "tm_field_norm2: misaligned pointer");
    CKS(check_prec(prec));
    if (!device_fields(field, result)) return fail(TM_ERR_ARG, "tm_field_norm2: field and result must be device pointers");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    switch (prec) {
        case TM_F64: CK(norm2_t<P64>(c, nf, field, result, st)); break;
        case TM_F32: CK(norm2_t<P32>(c, nf, field, result, st)); break;
        case TM_BF16: CK(norm2_t<PB16>(c, nf, field, result, st)); break;
        default: CK(norm2_t<PF16>(c, nf, field, result, st)); break;
    }
    return TM_OK;
}

static tm_status read_scalar(tm_ctx* c, double* dev, double* out, cudaStream_t st) {
    CK(cudaMemcpyAsync(c->h_scal, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    *out = c->h_scal[0];
    return TM_OK;
}

static tm_status put_ctl(tm_ctx* c, cudaStream_t st) {
    CK(cudaMemcpyAsync(c->ctl, c->h_ctl, sizeof(SolverCtl), cudaMemcpyHostToDevice, st));
    return TM_OK;
}
static tm_status get_ctl(tm_ctx* c, cudaStream_t st) {
    CK(cudaMemcpyAsync(c->h_ctl, c->ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return TM_OK;
}

// r = b - (A + shift) x and rr = ||r||^2 in FP64.  x_zero: x is known to be zero,
// so A x = 0 without applying the operator (a zero initial guess).  dw: A x in
// double-word arithmetic (x and the result rounded to a 48-bit significand on the
// way in and out; mid64, te64 and ax64 serve as double-word scratch), for the
// reliable updates inside a mixed-precision solve; otherwise native FP64.
template <int NF>
static tm_status true_residual(tm_ctx* c, tm_op op, double shift, void* x64, void* b64, void* r64, void* ax64,
                               void* mid64, void* te64, cudaStream_t st, double* rr, bool x_zero = false,
                               bool dw = false) {
    const long n16 = 12 * NF * c->vh;   // 16-byte elements of a field
    if (x_zero) {
        CK(cudaMemsetAsync(ax64, 0, spinor_bytes(P64, 12 * NF, c->vh), st));
    } else if (dw) {
        void* xdf = nullptr;
        CKS(ensure_df(c, st));
        CKS(ws_get(c, WS_XDF, spinor_bytes(PDF, 12 * NF, c->vh), &xdf));
        CK(launch_f64_to_df(xdf, x64, n16, st));
        CK((normal_op<PDF, NF>(c, op, ax64, xdf, mid64, te64, st, nullptr, FIN_NONE)));
        CK(launch_df_to_f64(ax64, ax64, n16, st));
    } else {
        CK((normal_op<P64, NF>(c, op, ax64, x64, mid64, te64, st, nullptr, FIN_NONE)));
    }
    c->h_ctl->shift = shift;
    CK(cudaMemcpyAsync(&c->ctl->shift, &c->h_ctl->shift, sizeof(double), cudaMemcpyHostToDevice, st));
    CK((launch_residual64<12 * NF, 1>(vb1(c, r64, b64, ax64, x64, c->d_scal), nblk(c->vh, BLAS_BS), st)));
    return read_scalar(c, c->d_scal, rr, st);
}

template <int P, int NC>
static tm_status norm2_dev(tm_ctx* c, const void* v, cudaStream_t st, double* out) {
    CK((launch_norm2<P, NC, 1>(vb1(c, const_cast<void*>(v), nullptr, nullptr, nullptr, c->d_scal),
                                nblk(c->vh, BLAS_BS), st)));
    return read_scalar(c, c->d_scal, out, st);
}

// whether a native FP64 field is exactly zero (||x||^2 == 0)
template <int NF>
static tm_status is_zero64(tm_ctx* c, const void* x64, cudaStream_t st, bool* zero) {
    double xx = 0.0;
    CKS((norm2_dev<P64, 12 * NF>(c, x64, st, &xx)));
    *zero = xx == 0.0;
    return TM_OK;
}

// One CG iteration in storage precision PS (x accumulated in PX):
//   p = r + beta p;  Ap (fused <p,Ap> -> alpha);  x += alpha p, r -= alpha Ap (fused rr -> beta, flag)
template <int PS, int NF>
static cudaError_t cg_iteration(tm_ctx* c, tm_op op, void* xs, void* p, void* r, void* ap, void* mid, void* te,
                                cudaStream_t st) {
    constexpr int PX = PS == P64 ? P64 : P32;
    const int nb = nblk(c->vh, BLAS_BS);
    cudaError_t e = launch_cg_pupdate<PS, 12 * NF, 1>(vb1(c, p, r), nb, st);
    if (e != cudaSuccess) return e;
    e = normal_op<PS, NF>(c, op, ap, p, mid, te, st, c->ctl, FIN_CG_ALPHA);
    if (e != cudaSuccess) return e;
    return launch_cg_update<PS, PX, 12 * NF, 1>(vb1(c, xs, p, r, ap), nb, st);
}

// Solve (A + shift) x = b in place on native FP64 x64, b64.
// PS == P64: plain FP64 CG.  Otherwise mixed precision with reliable updates:
// the iteration runs in PS storage / FP32 arithmetic with x accumulated in FP32;
// whenever ||r|| has dropped by delta since the last true residual, x is folded
// into the FP64 solution and r = b - A x is recomputed in double-word arithmetic
// (true_residual); a residual below the tolerance is confirmed in FP64.
template <int PS, int NF>
static tm_status solve_core(tm_ctx* c, tm_op op, double shift, const tm_solve_params* sp, void* x64, void* b64,
                            tm_solve_info* info, cudaStream_t st) {
    constexpr int NC = 12 * NF;
    const long vh = c->vh;
    const size_t b64sz = spinor_bytes(P64, NC, vh), bssz = spinor_bytes(PS, NC, vh);
    void *r64, *ax64, *te64, *mid64;
    CKS(ws_get(c, WS_R64, b64sz, &r64));
    CKS(ws_get(c, WS_AX64, b64sz, &ax64));
    CKS(ws_get(c, WS_TE64, b64sz, &te64));
    CKS(ws_get(c, WS_MID64, b64sz, &mid64));
    void *rs, *ps, *aps, *tes, *mids, *xs;
    if (PS == P64) {
        rs = r64; xs = x64; tes = te64; mids = mid64;
        CKS(ws_get(c, WS_P_S, bssz, &ps));
        CKS(ws_get(c, WS_AP_S, bssz, &aps));
    } else {
        CKS(ws_get(c, WS_R_S, bssz, &rs));
        CKS(ws_get(c, WS_P_S, bssz, &ps));
        CKS(ws_get(c, WS_AP_S, bssz, &aps));
        CKS(ws_get(c, WS_TE_S, bssz, &tes));
        CKS(ws_get(c, WS_MID_S, bssz, &mids));
        CKS(ws_get(c, WS_X_S, spinor_bytes(P32, NC, vh), &xs));
    }
    const double tol = sp->tol > 0 ? sp->tol : 1e-10;
    const int maxiter = sp->maxiter > 0 ? sp->maxiter : 100000;
    const double delta = PS == P64 ? 0.0 : (sp->delta > 0 ? sp->delta : default_delta(PS));
    const int chunk = sp->chunk > 0 ? sp->chunk : 16;
    const int nb = nblk(vh, BLAS_BS);

    double bb = 0;
    CKS((norm2_dev<P64, NC>(c, b64, st, &bb)));
    info->iters = 0;
    info->reliable_updates = 0;
    if (!std::isfinite(bb)) {
        info->true_rel_res = bb;
        info->status = TM_ERR_BREAKDOWN;
        return fail(TM_ERR_BREAKDOWN, "solve: right-hand side is not finite");
    }
    if (!(bb > 0)) {
        CK(cudaMemsetAsync(x64, 0, b64sz, st));
        info->true_rel_res = 0.0;
        info->status = TM_OK;
        return TM_OK;
    }
    double rr = 0;
    bool x0 = false;
    CKS(is_zero64<NF>(c, x64, st, &x0));
    const bool dw = PS != P64 && !sp->fp64_updates;   // double-word reliable updates
    CKS(true_residual<NF>(c, op, shift, x64, b64, r64, ax64, mid64, te64, st, &rr, x0, dw));
    const double target = tol * tol * bb;
    // an initial guess already within the tolerance is confirmed in FP64
    if (dw && !x0 && rr <= target)
        CKS(true_residual<NF>(c, op, shift, x64, b64, r64, ax64, mid64, te64, st, &rr));
    tm_status status = TM_OK;
    cudaGraphExec_t gexec = nullptr;
    if (rr > target) {
        if (PS != P64) {
            CK((launch_convert<PS, P64, NC, 1>(vb1(c, rs, r64), nb, st)));
            CK(cudaMemsetAsync(xs, 0, spinor_bytes(P32, NC, vh), st));
        }
        SolverCtl& h = *c->h_ctl;
        std::memset(&h, 0, sizeof(SolverCtl));
        h.rr = rr;
        h.rr_old = rr;
        h.beta = 0.0;
        h.shift = shift;
        h.maxiter = maxiter;
        h.stop_rr = std::max(target, delta * delta * rr);
        h.flag = CTL_RUN;
        CKS(put_ctl(c, st));
        if (sp->use_graph) {
            cudaGraph_t graph;
            CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
            for (int it = 0; it < chunk; ++it) {
                cudaError_t e = cg_iteration<PS, NF>(c, op, xs, ps, rs, aps, mids, tes, st);
                if (e != cudaSuccess) {
                    cudaStreamEndCapture(st, &graph);
                    return fail(TM_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
                }
            }
            CK(cudaStreamEndCapture(st, &graph));
            CK(cudaGraphInstantiate(&gexec, graph, 0));
            cudaGraphDestroy(graph);
        }
        for (;;) {
            if (gexec) {
                CK(cudaGraphLaunch(gexec, st));
            } else {
                for (int it = 0; it < chunk; ++it) CK((cg_iteration<PS, NF>(c, op, xs, ps, rs, aps, mids, tes, st)));
            }
            CKS(get_ctl(c, st));
            if (h.flag == CTL_RUN) continue;
            if (h.flag == CTL_BREAKDOWN) { status = TM_ERR_BREAKDOWN; break; }
            // reliable update / convergence check
            if (PS != P64) {
                CK((launch_add_to64<P32, NC, 1>(vb1(c, x64, xs), nb, st)));
                CK(cudaMemsetAsync(xs, 0, spinor_bytes(P32, NC, vh), st));
            }
            CKS(true_residual<NF>(c, op, shift, x64, b64, r64, ax64, mid64, te64, st, &rr, false, dw));
            info->reliable_updates += 1;
            // a double-word residual below the target is confirmed in FP64 (the
            // returned true residual is always an FP64 one)
            if (dw && rr <= target)
                CKS(true_residual<NF>(c, op, shift, x64, b64, r64, ax64, mid64, te64, st, &rr));
            if (rr <= target) break;
            if (h.flag == CTL_MAXITER || h.iter >= maxiter || !std::isfinite(rr)) {
                status = std::isfinite(rr) ? TM_ERR_NOT_CONVERGED : TM_ERR_BREAKDOWN;
                break;
            }
            if (PS != P64) CK((launch_convert<PS, P64, NC, 1>(vb1(c, rs, r64), nb, st)));
            h.beta = rr / h.rr_old;
            h.rr = rr;
            h.stop_rr = std::max(target, delta * delta * rr);
            h.flag = CTL_RUN;
            CKS(put_ctl(c, st));
        }
        info->iters = h.iter;
        if (gexec) cudaGraphExecDestroy(gexec);
    }
    info->true_rel_res = std::sqrt(rr / bb);
    info->status = status;
    if (status != TM_OK)
        fail(status, "solve: %s after %d iterations, true rel res %.3e",
             status == TM_ERR_BREAKDOWN ? "breakdown" : "not converged", info->iters, info->true_rel_res);
    return status;
}

template <int NF>
static tm_status solve_dispatch(tm_ctx* c, tm_op op, double shift, const tm_solve_params* sp, void* x64, void* b64,
                                tm_solve_info* info, cudaStream_t st) {
    switch (sp->sloppy) {
        case TM_F64: return solve_core<P64, NF>(c, op, shift, sp, x64, b64, info, st);
        case TM_F32: return solve_core<P32, NF>(c, op, shift, sp, x64, b64, info, st);
        case TM_BF16: return solve_core<PB16, NF>(c, op, shift, sp, x64, b64, info, st);
        case TM_F16: return solve_core<PF16, NF>(c, op, shift, sp, x64, b64, info, st);
    }
    return fail(TM_ERR_ARG, "unknown sloppy precision");
}

// canonical (host or device) <-> native FP64 working copies
static tm_status stage_in(tm_ctx* c, int nf, const double* canon, int stage_id, void* native64, cudaStream_t st) {
    const size_t bytes = sizeof(double) * 24 * nf * c->vh;
    const double* src = canon;
    if (!is_device_ptr(canon)) {
        void* s = nullptr;
        CKS(ws_get(c, stage_id, bytes, &s));
        CK(cudaMemcpyAsync(s, canon, bytes, cudaMemcpyHostToDevice, st));
        src = reinterpret_cast<const double*>(s);
    }
    CK(import_any(P64, nf, native64, src, c->vh, st));
    return TM_OK;
}
static tm_status stage_out(tm_ctx* c, int nf, double* canon, int stage_id, const void* native64, cudaStream_t st) {
    const size_t bytes = sizeof(double) * 24 * nf * c->vh;
    if (is_device_ptr(canon)) {
        CK(export_any(P64, nf, canon, native64, c->vh, st));
    } else {
        void* s = nullptr;
        CKS(ws_get(c, stage_id, bytes, &s));
        CK(export_any(P64, nf, reinterpret_cast<double*>(s), native64, c->vh, st));
        CK(cudaMemcpyAsync(canon, s, bytes, cudaMemcpyDeviceToHost, st));
    }
    return TM_OK;
}

static tm_status enter_solver(tm_ctx* c, void* stream) {
    // order the private solver stream after the caller's stream
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CK(cudaEventRecord(ev, S(stream)));
    CK(cudaStreamWaitEvent(c->sstream, ev, 0));
    cudaEventDestroy(ev);
    return TM_OK;
}

static tm_status check_solver_op(tm_ctx* c, tm_op op) {
    if (op != TM_MDAGM && op != TM_QPQM && op != TM_QH_SQ && op != TM_WHAT_SQ)
        return fail(TM_ERR_ARG, "solver op must be TM_MDAGM, TM_QPQM, TM_QH_SQ or TM_WHAT_SQ");
    if (op == TM_QH_SQ && !c->have_heavy)
        return fail(TM_ERR_ARG, "heavy operator needs mubar or epsbar in tm_clover_compute");
    return TM_OK;
}

extern "C" tm_status tm_solve_cg(tm_ctx* c, tm_op op, const tm_solve_params* sp, double* x, const double* b,
                                 tm_solve_info* info, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!c || !sp || !x || !b || !info) return fail(TM_ERR_ARG, "tm_solve_cg: null argument");
    CKS(check_prec(sp->sloppy));
    CK(cudaSetDevice(c->device));
    CKS(check_solver_op(c, op));
    const cudaStream_t st = c->sstream;
    CKS(enter_solver(c, stream));
    CKS(ensure_prec(c, P64, st));
    CKS(ensure_prec(c, sp->sloppy, st));
    const int nf = nflav(op);
    void *x64, *b64;
    CKS(ws_get(c, WS_X64, spinor_bytes(P64, 12 * nf, c->vh), &x64));
    CKS(ws_get(c, WS_B64, spinor_bytes(P64, 12 * nf, c->vh), &b64));
    CKS(stage_in(c, nf, b, WS_STAGE_B, b64, st));
    CKS(stage_in(c, nf, x, WS_STAGE_X, x64, st));
    tm_status s = nf == 1 ? solve_dispatch<1>(c, op, 0.0, sp, x64, b64, info, st)
                          : solve_dispatch<2>(c, op, 0.0, sp, x64, b64, info, st);
    CKS(stage_out(c, nf, x, WS_STAGE_X, x64, st));
    CK(cudaStreamSynchronize(st));
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    return s;
}

// ---------------------------------------------------------------------------
// multishift CG (Sec. 4.2) with shift-by-shift refinement
// ---------------------------------------------------------------------------
template <int PS, int NF>
static tm_status multishift_core(tm_ctx* c, tm_op op, int ns, const double* sh_sorted, void* b64,
                                 const tm_solve_params* sp, std::vector<void*>& xk64, int* iters,
                                 cudaStream_t st) {
    constexpr int NC = 12 * NF;
    constexpr int PX = PS == P64 ? P64 : P32;
    const long vh = c->vh;
    const size_t bs = spinor_bytes(PS, NC, vh), bx = spinor_bytes(PX, NC, vh);
    void *rs, *ps, *aps, *tes, *mids;
    CKS(ws_get(c, WS_R_S, bs, &rs));
    CKS(ws_get(c, WS_P_S, bs, &ps));
    CKS(ws_get(c, WS_AP_S, bs, &aps));
    CKS(ws_get(c, WS_TE_S, bs, &tes));
    CKS(ws_get(c, WS_MID_S, bs, &mids));
    MsVecs mv{};
    for (int k = 0; k < ns; ++k) {
        CKS(ws_get(c, WS_MS_P + k, bs, &mv.p[k]));
        if (PX == P64) {
            mv.x[k] = xk64[k];
        } else {
            CKS(ws_get(c, WS_MS_X + k, bx, &mv.x[k]));
        }
        CK(cudaMemsetAsync(mv.x[k], 0, bx, st));
    }
    const int nb = nblk(vh, BLAS_BS);
    double bb;
    CKS((norm2_dev<P64, NC>(c, b64, st, &bb)));
    if (!std::isfinite(bb) || !(bb > 0))
        return fail(std::isfinite(bb) ? TM_ERR_ARG : TM_ERR_BREAKDOWN,
                    "multishift: right-hand side must be finite and non-zero");
    CK((launch_convert<PS, P64, NC, 1>(vb1(c, rs, b64), nb, st)));
    // The sloppy multishift stops each shift when its recursively updated residual
    // falls below floor_tol; the shift-by-shift refinement takes it to sp->tol.
    // Swept on the heavy doublet at 24^3x48 (12 shifts, time of the whole solve
    // with refinement): FP32 1e-6 / 1e-7 / 1e-8 / 1e-9 / 1e-10 -> 0.721 / 0.631 /
    // 0.594 / 0.611 / 0.634 s; 16-bit 2e-4 / 5e-5 / 1e-5 / 1e-6 -> 0.972 / 0.936 /
    // 0.870 / 0.892 s.  Below the storage's own precision the sloppy solutions
    // still improve (the reductions are FP64), and a refinement iteration costs
    // about half a multishift one, until the extra multishift iterations stop
    // paying.
    const double floor_tol = PS == P64 ? 0.0 : (PS == P32 ? 1e-8 : 1e-5);
    const double ms_tol = std::max(sp->tol, floor_tol);
    MsCtl& m = *c->h_ms;
    std::memset(&m, 0, sizeof(MsCtl));
    for (int k = 0; k < ns; ++k) {
        m.zeta[k] = m.zeta_old[k] = 1.0;
        m.dshift[k] = sh_sorted[k] - sh_sorted[0];
        m.active[k] = 1;
    }
    m.alpha_old = 1.0;
    m.beta_old = 0.0;
    m.nshift = ns;
    m.n_active = ns;
    m.stop_rr = ms_tol * ms_tol * bb;
    CK(cudaMemcpyAsync(c->ms, &m, sizeof(MsCtl), cudaMemcpyHostToDevice, st));
    SolverCtl& h = *c->h_ctl;
    std::memset(&h, 0, sizeof(SolverCtl));
    h.rr = bb;
    h.rr_old = bb;
    h.shift = sh_sorted[0];
    h.maxiter = sp->maxiter > 0 ? sp->maxiter : 100000;
    h.stop_rr = 0.0;
    h.flag = CTL_RUN;
    CKS(put_ctl(c, st));
    auto iteration = [&](int first) -> cudaError_t {
        cudaError_t e = launch_ms_pupdate<PS, PX, NC>(vb1(c, rs, ps), mv, first, nb, st);
        if (e != cudaSuccess) return e;
        e = normal_op<PS, NF>(c, op, aps, ps, mids, tes, st, c->ctl, FIN_MS_ALPHA);
        if (e != cudaSuccess) return e;
        return launch_ms_update<PS, NC>(vb1(c, rs, ps, aps), nb, st);
    };
    CK(iteration(1));
    const int chunk = sp->chunk > 0 ? sp->chunk : 16;
    cudaGraphExec_t gexec = nullptr;
    if (sp->use_graph) {
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < chunk; ++it) {
            cudaError_t e = iteration(0);
            if (e != cudaSuccess) {
                cudaStreamEndCapture(st, &graph);
                return fail(TM_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
            }
        }
        CK(cudaStreamEndCapture(st, &graph));
        CK(cudaGraphInstantiate(&gexec, graph, 0));
        cudaGraphDestroy(graph);
    }
    tm_status status = TM_OK;
    for (;;) {
        CKS(get_ctl(c, st));
        if (h.flag != CTL_RUN) break;
        if (gexec) {
            CK(cudaGraphLaunch(gexec, st));
        } else {
            for (int it = 0; it < chunk; ++it) CK(iteration(0));
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    if (h.flag == CTL_BREAKDOWN) status = fail(TM_ERR_BREAKDOWN, "multishift: breakdown");
    CK((launch_ms_finish<PS, PX, NC>(vb1(c, rs, ps), mv, nb, st)));
    // hand the sloppy solutions to FP64
    if (PX != P64) {
        for (int k = 0; k < ns; ++k) {
            CK(cudaMemsetAsync(xk64[k], 0, spinor_bytes(P64, NC, vh), st));
            CK((launch_add_to64<P32, NC, 1>(vb1(c, xk64[k], mv.x[k]), nb, st)));
        }
    }
    *iters = h.iter;
    return status;
}

template <int NF>
static tm_status multishift_dispatch(tm_ctx* c, tm_op op, int ns, const double* sh, void* b64,
                                     const tm_solve_params* sp, std::vector<void*>& xk64, int* iters,
                                     cudaStream_t st) {
    switch (sp->sloppy) {
        case TM_F64: return multishift_core<P64, NF>(c, op, ns, sh, b64, sp, xk64, iters, st);
        case TM_F32: return multishift_core<P32, NF>(c, op, ns, sh, b64, sp, xk64, iters, st);
        case TM_BF16: return multishift_core<PB16, NF>(c, op, ns, sh, b64, sp, xk64, iters, st);
        case TM_F16: return multishift_core<PF16, NF>(c, op, ns, sh, b64, sp, xk64, iters, st);
    }
    return fail(TM_ERR_ARG, "unknown sloppy precision");
}

// Multishift CG in the sloppy precision plus shift-by-shift refinement (Sec. 4.2)
// on a native FP64 right-hand side b64 (not a WS_MS_X64 field); the refined
// solutions stay in the native FP64 workspace fields, xk[k] for shifts[k]
// (null when the multishift solve itself failed and shift k has no solution).
static tm_status ms_core(tm_ctx* c, tm_op op, int ns, const double* shifts, void* b64, const tm_solve_params* sp,
                         tm_solve_info* infos, cudaStream_t st, std::vector<void*>& xk) {
    const int nf = nflav(op);
    const size_t b64sz = spinor_bytes(P64, 12 * nf, c->vh);
    std::vector<int> order(ns);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int bq) { return shifts[a] < shifts[bq]; });
    std::vector<double> sh(ns);
    for (int k = 0; k < ns; ++k) sh[k] = shifts[order[k]];
    std::vector<void*> xk64(ns);
    for (int k = 0; k < ns; ++k) CKS(ws_get(c, WS_MS_X64 + k, b64sz, &xk64[k]));
    int ms_iters = 0;
    tm_status s = nf == 1 ? multishift_dispatch<1>(c, op, ns, sh.data(), b64, sp, xk64, &ms_iters, st)
                          : multishift_dispatch<2>(c, op, ns, sh.data(), b64, sp, xk64, &ms_iters, st);
    tm_status worst = s;
    // shift-by-shift refinement with mixed-precision CG, in its own storage
    // precision when sp->refine names one
    tm_solve_params rsp = *sp;
    if (sp->refine != TM_F64) rsp.sloppy = sp->refine;
    xk.assign(ns, nullptr);
    for (int k = 0; k < ns; ++k) {
        tm_solve_info& inf = infos[order[k]];
        std::memset(&inf, 0, sizeof(inf));
        if (s != TM_OK) { inf.status = s; continue; }
        xk[order[k]] = xk64[k];
        tm_status r = nf == 1 ? solve_dispatch<1>(c, op, sh[k], &rsp, xk64[k], b64, &inf, st)
                              : solve_dispatch<2>(c, op, sh[k], &rsp, xk64[k], b64, &inf, st);
        inf.iters += ms_iters;
        if (r != TM_OK && worst == TM_OK) worst = r;
    }
    return worst;
}

static tm_status ms_check(tm_ctx* c, tm_op op, int ns, const double* shifts, const tm_solve_params* sp,
                          const char* who) {
    if (ns < 1 || ns > MAX_SHIFTS) return fail(TM_ERR_ARG, "%s: 1 <= nshift <= %d", who, MAX_SHIFTS);
    for (int k = 0; k < ns; ++k)
        if (!(shifts[k] >= 0.0)) return fail(TM_ERR_ARG, "%s: shifts must be >= 0", who);
    if (op != TM_MDAGM && op != TM_QH_SQ && op != TM_QPQM) return fail(TM_ERR_ARG, "%s: bad op", who);
    CKS(check_prec(sp->sloppy));
    CKS(check_prec(sp->refine));
    CK(cudaSetDevice(c->device));
    return check_solver_op(c, op);
}

static tm_status ms_prepare(tm_ctx* c, const tm_solve_params* sp, cudaStream_t st) {
    CKS(ensure_prec(c, P64, st));
    CKS(ensure_prec(c, sp->sloppy, st));
    if (sp->refine != TM_F64) CKS(ensure_prec(c, sp->refine, st));
    return TM_OK;
}

extern "C" tm_status tm_solve_multishift(tm_ctx* c, tm_op op, int ns, const double* shifts, double** x,
                                         const double* b, const tm_solve_params* sp, tm_solve_info* infos,
                                         void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!c || !shifts || !x || !b || !sp || !infos) return fail(TM_ERR_ARG, "tm_solve_multishift: null argument");
    CKS(ms_check(c, op, ns, shifts, sp, "tm_solve_multishift"));
    for (int k = 0; k < ns; ++k)
        if (!x[k]) return fail(TM_ERR_ARG, "tm_solve_multishift: null solution buffer");
    const cudaStream_t st = c->sstream;
    CKS(enter_solver(c, stream));
    CKS(ms_prepare(c, sp, st));
    const int nf = nflav(op);
    void* b64;
    CKS(ws_get(c, WS_B64, spinor_bytes(P64, 12 * nf, c->vh), &b64));
    CKS(stage_in(c, nf, b, WS_STAGE_B, b64, st));
    std::vector<void*> xk;
    tm_status worst = ms_core(c, op, ns, shifts, b64, sp, infos, st, xk);
    for (int k = 0; k < ns; ++k) {
        if (!xk[k]) continue;
        CKS(stage_out(c, nf, x[k], WS_STAGE_X, xk[k], st));
        CK(cudaStreamSynchronize(st));
    }
    CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < ns; ++k) infos[k].seconds = secs;
    return worst;
}

// ---------------------------------------------------------------------------
// rational approximation of A^-1/2 (Sec. 4.2's rational monomials and their
// correction term, Fig. 4)
// ---------------------------------------------------------------------------
extern "C" tm_status tm_rational_inv_sqrt(int n, double lo, double hi, double* a0, double* a, double* sigma,
                                          double* delta) {
    if (!a0 || !a || !sigma || !delta || n < 1 || n > MAX_SHIFTS || !(lo > 0.0) || !(hi > lo))
        return fail(TM_ERR_ARG, "tm_rational_inv_sqrt: need 1 <= n <= %d, 0 < lo < hi", MAX_SHIFTS);
    if (!zolotarev_inv_sqrt(n, lo, hi, a0, a, sigma, delta)) return fail(TM_ERR_ARG, "tm_rational_inv_sqrt: failed");
    return TM_OK;
}

// y64 = a0 b64 + sum_k a_k (A + sigma_k)^-1 b64, native FP64 fields (y64 may be b64)
static tm_status rational_native(tm_ctx* c, tm_op op, int n, double a0, const double* a, const double* sigma,
                                 void* y64, void* b64, const tm_solve_params* sp, tm_solve_info* infos,
                                 cudaStream_t st, tm_status* worst) {
    std::vector<void*> xk;
    tm_status s = ms_core(c, op, n, sigma, b64, sp, infos, st, xk);
    if (s != TM_OK && *worst == TM_OK) *worst = s;
    for (int k = 0; k < n; ++k)
        if (!xk[k]) return fail(s, "rational approximation: the multishift solve failed");
    LinComb lc{};
    lc.n = n;
    lc.len = (long)c->vh * 12 * nflav(op);
    lc.a0 = a0;
    lc.b = reinterpret_cast<const double2*>(b64);
    for (int k = 0; k < n; ++k) {
        lc.x[k] = reinterpret_cast<const double2*>(xk[k]);
        lc.a[k] = a[k];
    }
    lc.y = reinterpret_cast<double2*>(y64);
    CK(launch_lincomb64(lc, st));
    return TM_OK;
}

static tm_status rational_args(tm_ctx* c, tm_op op, int n, const double* a, const double* sigma, void* y,
                               const void* b, const tm_solve_params* sp, tm_solve_info* infos, const char* who) {
    if (!c || !a || !sigma || !y || !b || !sp || !infos) return fail(TM_ERR_ARG, "%s: null argument", who);
    if ((((uintptr_t)y | (uintptr_t)b) & 15)) return fail(TM_ERR_ARG, "%s: fields must be 16-byte aligned", who);
    return ms_check(c, op, n, sigma, sp, who);
}

extern "C" tm_status tm_rational_apply(tm_ctx* c, tm_op op, int n, double a0, const double* a, const double* sigma,
                                       double* y, const double* b, const tm_solve_params* sp, tm_solve_info* infos,
                                       void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    CKS(rational_args(c, op, n, a, sigma, y, b, sp, infos, "tm_rational_apply"));
    const cudaStream_t st = c->sstream;
    CKS(enter_solver(c, stream));
    CKS(ms_prepare(c, sp, st));
    const int nf = nflav(op);
    const size_t sz = spinor_bytes(P64, 12 * nf, c->vh);
    void *b64, *y64;
    CKS(ws_get(c, WS_RAT + 0, sz, &b64));
    CKS(ws_get(c, WS_RAT + 1, sz, &y64));
    CKS(stage_in(c, nf, b, WS_STAGE_B, b64, st));
    tm_status worst = TM_OK;
    CKS(rational_native(c, op, n, a0, a, sigma, y64, b64, sp, infos, st, &worst));
    CKS(stage_out(c, nf, y, WS_STAGE_X, y64, st));
    CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < n; ++k) infos[k].seconds = secs;
    return worst;
}

template <int NF>
static tm_status correction_core(tm_ctx* c, tm_op op, int n, double a0, const double* a, const double* sigma,
                                 double p, double series_tol, int max_terms, void* y64, void* b64,
                                 const tm_solve_params* sp, tm_solve_info* infos, int* napply, cudaStream_t st,
                                 tm_status* worst) {
    constexpr int NC = 12 * NF;
    const size_t sz = spinor_bytes(P64, NC, c->vh);
    void *t64, *u64, *w64, *te, *mid;
    CKS(ws_get(c, WS_RAT + 2, sz, &t64));
    CKS(ws_get(c, WS_RAT + 3, sz, &u64));
    CKS(ws_get(c, WS_RAT + 4, sz, &w64));
    CKS(ws_get(c, WS_APPLY_TE, sz, &te));
    CKS(ws_get(c, WS_APPLY_MID, sz, &mid));
    const long len = (long)c->vh * NC;
    auto comb = [&](void* dst, double ca, const void* x, double cb, const void* v) -> tm_status {
        LinComb lc{};
        lc.n = 1;
        lc.len = len;
        lc.a0 = ca;
        lc.b = reinterpret_cast<const double2*>(x);
        lc.x[0] = reinterpret_cast<const double2*>(v);
        lc.a[0] = cb;
        lc.y = reinterpret_cast<double2*>(dst);
        CK(launch_lincomb64(lc, st));
        return TM_OK;
    };
    double bb = 0.0;
    CKS((norm2_dev<P64, NC>(c, b64, st, &bb)));
    CKS(comb(y64, 1.0, b64, 0.0, b64));
    CKS(comb(t64, 1.0, b64, 0.0, b64));
    double coef = 1.0;
    *napply = 0;
    for (int j = 1; j <= max_terms; ++j) {
        // t <- Z t = A r(A)^2 t - t; a failed multishift solve ends the series
        // (its residual would poison every later term), returning the terms so far
        CKS(rational_native(c, op, n, a0, a, sigma, u64, t64, sp, infos, st, worst));
        if (*worst != TM_OK) break;
        CKS(rational_native(c, op, n, a0, a, sigma, w64, u64, sp, infos, st, worst));
        if (*worst != TM_OK) break;
        CK((normal_op<P64, NF>(c, op, u64, w64, mid, te, st, nullptr, FIN_NONE)));
        CKS(comb(t64, 1.0, u64, -1.0, t64));
        ++*napply;
        coef *= (p - (j - 1)) / j;
        CKS(comb(y64, 1.0, y64, coef, t64));
        double tt = 0.0;
        CKS((norm2_dev<P64, NC>(c, t64, st, &tt)));
        if (coef * coef * tt <= series_tol * series_tol * bb) break;
    }
    return TM_OK;
}

extern "C" tm_status tm_rational_correction(tm_ctx* c, tm_op op, int n, double a0, const double* a,
                                            const double* sigma, double p, double series_tol, double* y,
                                            const double* b, const tm_solve_params* sp, tm_solve_info* infos,
                                            int* napply, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    CKS(rational_args(c, op, n, a, sigma, y, b, sp, infos, "tm_rational_correction"));
    if (!napply || !(series_tol > 0.0)) return fail(TM_ERR_ARG, "tm_rational_correction: bad argument");
    const cudaStream_t st = c->sstream;
    CKS(enter_solver(c, stream));
    CKS(ms_prepare(c, sp, st));
    const int nf = nflav(op);
    const size_t sz = spinor_bytes(P64, 12 * nf, c->vh);
    void *b64, *y64;
    CKS(ws_get(c, WS_RAT + 0, sz, &b64));
    CKS(ws_get(c, WS_RAT + 1, sz, &y64));
    CKS(stage_in(c, nf, b, WS_STAGE_B, b64, st));
    tm_status worst = TM_OK;
    const int max_terms = 40;
    CKS(nf == 1 ? correction_core<1>(c, op, n, a0, a, sigma, p, series_tol, max_terms, y64, b64, sp, infos,
                                     napply, st, &worst)
                : correction_core<2>(c, op, n, a0, a, sigma, p, series_tol, max_terms, y64, b64, sp, infos,
                                     napply, st, &worst));
    CKS(stage_out(c, nf, y, WS_STAGE_X, y64, st));
    CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int k = 0; k < n; ++k) infos[k].seconds = secs;
    return worst;
}

// ---------------------------------------------------------------------------
// power iteration
// ---------------------------------------------------------------------------
template <int NF>
static tm_status power_core(tm_ctx* c, tm_op op, int iters, double* lam, cudaStream_t st) {
    constexpr int NC = 12 * NF;
    const long vh = c->vh;
    const size_t sz = spinor_bytes(P64, NC, vh);
    void *v, *w, *te, *mid;
    CKS(ws_get(c, WS_V64, sz, &v));
    CKS(ws_get(c, WS_AX64, sz, &w));
    CKS(ws_get(c, WS_TE64, sz, &te));
    CKS(ws_get(c, WS_MID64, sz, &mid));
    // fixed start vector (splitmix64 of the component index), made on the host
    std::vector<double> h((size_t)2 * NC * vh);
    uint64_t s = 0x9e3779b97f4a7c15ull;
    for (size_t k = 0; k < h.size(); ++k) {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        h[k] = (double)(z >> 11) * (1.0 / 9007199254740992.0) - 0.5;
    }
    void* stage;
    CKS(ws_get(c, WS_STAGE_B, h.size() * sizeof(double), &stage));
    CK(cudaMemcpyAsync(stage, h.data(), h.size() * sizeof(double), cudaMemcpyHostToDevice, st));
    CK(import_any(P64, NF, v, reinterpret_cast<const double*>(stage), vh, st));
    CK(cudaStreamSynchronize(st));
    const int nb = nblk(vh, BLAS_BS);
    CK((launch_norm2<P64, NC, 1>(vb1(c, v, nullptr, nullptr, nullptr, c->d_scal), nb, st)));
    CK((launch_normalize64<NC>(vb1(c, v, nullptr, nullptr, nullptr, c->d_scal), nb, st)));
    std::memset(c->h_ctl, 0, sizeof(SolverCtl));
    CKS(put_ctl(c, st));
    for (int it = 0; it < iters; ++it) {
        // <v, A v> = ||Q v||^2 (fused, FIN_STORE -> ctl->result); w = A v; v = w / ||w||
        CK((normal_op<P64, NF>(c, op, w, v, mid, te, st, c->ctl, FIN_STORE)));
        CK((launch_norm2<P64, NC, 1>(vb1(c, w, nullptr, nullptr, nullptr, c->d_scal), nb, st)));
        CK((launch_normalize64<NC>(vb1(c, w, nullptr, nullptr, nullptr, c->d_scal), nb, st)));
        std::swap(v, w);
    }
    CKS(get_ctl(c, st));
    *lam = c->h_ctl->result;
    // keep the workspace map consistent with the swapped buffers
    c->ws[WS_V64].first = v;
    c->ws[WS_AX64].first = w;
    return TM_OK;
}

extern "C" tm_status tm_power_iteration(tm_ctx* c, tm_op op, int iters, double* lam, void* stream) {
    if (!c || !lam || iters < 1) return fail(TM_ERR_ARG, "tm_power_iteration: bad argument");
    CK(cudaSetDevice(c->device));
    CKS(check_solver_op(c, op));
    const cudaStream_t st = c->sstream;
    CKS(enter_solver(c, stream));
    CKS(ensure_prec(c, P64, st));
    return nflav(op) == 1 ? power_core<1>(c, op, iters, lam, st) : power_core<2>(c, op, iters, lam, st);
}

// ---------------------------------------------------------------------------
// batched solves: every step of every problem in one launch per kernel
// ---------------------------------------------------------------------------
struct BatchWs {
    void *x64, *b64, *rs, *ps, *aps, *tes, *mids, *xs;
};

template <int PS>
static tm_status batch_core(tm_ctx** cs, int n, tm_op op, const tm_solve_params* sp, std::vector<BatchWs>& w,
                            tm_solve_info* infos, cudaStream_t st) {
    constexpr int NC = 12;
    constexpr int PX = PS == P64 ? P64 : P32;
    const double tol = sp->tol > 0 ? sp->tol : 1e-10;
    const int maxiter = sp->maxiter > 0 ? sp->maxiter : 100000;
    const double delta = PS == P64 ? 0.0 : (sp->delta > 0 ? sp->delta : default_delta(PS));
    const int chunk = sp->chunk > 0 ? sp->chunk : 16;
    std::vector<double> bb(n), rr(n);
    std::vector<int> done(n, 0);
    // per-problem set-up: true residual, sloppy copies, control words
    for (int q = 0; q < n; ++q) {
        tm_ctx* c = cs[q];
        void *r64, *ax64, *te64, *mid64;
        const size_t sz = spinor_bytes(P64, NC, c->vh);
        CKS(ws_get(c, WS_R64, sz, &r64));
        CKS(ws_get(c, WS_AX64, sz, &ax64));
        CKS(ws_get(c, WS_TE64, sz, &te64));
        CKS(ws_get(c, WS_MID64, sz, &mid64));
        CKS((norm2_dev<P64, NC>(c, w[q].b64, st, &bb[q])));
        infos[q] = tm_solve_info{};
        if (!std::isfinite(bb[q])) { infos[q].status = TM_ERR_BREAKDOWN; done[q] = 1; continue; }
        if (!(bb[q] > 0)) { CK(cudaMemsetAsync(w[q].x64, 0, sz, st)); done[q] = 1; continue; }
        bool x0 = false;
        CKS(is_zero64<1>(c, w[q].x64, st, &x0));
        CKS(true_residual<1>(c, op, 0.0, w[q].x64, w[q].b64, r64, ax64, mid64, te64, st, &rr[q], x0));
        if (rr[q] <= tol * tol * bb[q]) { done[q] = 1; continue; }
        if (PS != P64) {
            CK((launch_convert<PS, P64, NC, 1>(vb1(c, w[q].rs, r64), nblk(c->vh, BLAS_BS), st)));
            CK(cudaMemsetAsync(w[q].xs, 0, spinor_bytes(P32, NC, c->vh), st));
        } else {
            w[q].rs = r64;
        }
        SolverCtl& h = *c->h_ctl;
        std::memset(&h, 0, sizeof(SolverCtl));
        h.rr = h.rr_old = rr[q];
        h.maxiter = maxiter;
        h.stop_rr = std::max(tol * tol * bb[q], delta * delta * rr[q]);
        h.flag = CTL_RUN;
        CKS(put_ctl(c, st));
    }
    // batched tables (problems that are already done keep flag != RUN and skip)
    OpBatch<MAXP> k1{}, k2a{}, k1b{}, k2b{};
    VecBatch<MAXP> pu{}, up{};
    int s1, s2;
    normal_signs(op, &s1, &s2);
    // Problem tables for a stencil variant per pass (0 direct, 1 staged).  The
    // variants are tuned on the batch itself: the batched passes of a mixed-size
    // batch behave unlike any one member's (the small lattices' blocks fill the
    // large one's tail), so both variants of both passes are timed on the
    // batch's own tables, with the passes that have no side effects on the solver
    // state (the even pass and the second odd pass).  The choice is kept per batch
    // composition and precision.
    int ob1 = 0, ob2 = 0, vbk = 0;
    auto build_tables = [&](int v1, int v2) -> tm_status {
        ob1 = ob2 = vbk = 0;
        for (int q = 0; q < n; ++q) {
            tm_ctx* c = cs[q];
            const int nb1 = nblk(c->vh, v1 ? STAGED_BS : DSLASH_BS), nb2 = nblk(c->vh, v2 ? STAGED_BS : DSLASH_BS);
            const int nbb = nblk(c->vh, BLAS_BS);
            SolverCtl* ctl = c->ctl;
            k1.blk_start[q] = k1b.blk_start[q] = ob1;
            k2a.blk_start[q] = k2b.blk_start[q] = ob2;
            pu.blk_start[q] = up.blk_start[q] = vbk;
            k1.p[q] = make_prob(c, PS, 1, K1_EO_INV, s1, w[q].tes, w[q].ps, nullptr, ctl, false);
            k2a.p[q] = make_prob(c, PS, 1, K2_OE_LOCAL, s1, w[q].mids, w[q].tes, w[q].ps, ctl, true);
            k1b.p[q] = make_prob(c, PS, 1, K1_EO_INV, s2, w[q].tes, w[q].mids, nullptr, ctl, false);
            k2b.p[q] = make_prob(c, PS, 1, K2_OE_LOCAL, s2, w[q].aps, w[q].tes, w[q].mids, ctl, false);
            k1.p[q].nblk = k1b.p[q].nblk = nb1;
            k2a.p[q].nblk = k2b.p[q].nblk = nb2;
            VecBatch<1> a = vb1(c, w[q].ps, w[q].rs);
            pu.p[q] = a.p[0];
            VecBatch<1> u = vb1(c, w[q].xs, w[q].ps, w[q].rs, w[q].aps);
            up.p[q] = u.p[0];
            ob1 += nb1;
            ob2 += nb2;
            vbk += nbb;
        }
        for (auto* t : {&k1, &k1b}) { t->n = n; t->blk_start[n] = ob1; t->fin = FIN_NONE; }
        for (auto* t : {&k2a, &k2b}) { t->n = n; t->blk_start[n] = ob2; t->fin = FIN_NONE; }
        k2a.fin = FIN_CG_ALPHA;
        pu.n = up.n = n;
        pu.blk_start[n] = up.blk_start[n] = vbk;
        return TM_OK;
    };
    for (int q = 0; q < n; ++q)
        if (done[q]) {   // done problems: a control word that stays stopped
            cs[q]->h_ctl->flag = CTL_STOP;
            CKS(put_ctl(cs[q], st));
        }
    int v1 = 0, v2 = 0;
    if (PS != P64) {
        std::string key = std::to_string(PS);
        for (int q = 0; q < n; ++q)
            key += " " + std::to_string(cs[q]->g.X) + "x" + std::to_string(cs[q]->g.Y) + "x" +
                   std::to_string(cs[q]->g.Z) + "x" + std::to_string(cs[q]->g.T);
        static std::mutex tune_mu;
        static std::map<std::string, std::pair<int, int>> tuned;
        std::lock_guard<std::mutex> lock(tune_mu);
        auto it = tuned.find(key);
        if (it != tuned.end()) {
            v1 = it->second.first;
            v2 = it->second.second;
        } else {
            cudaEvent_t e0, e1, e2;
            CK(cudaEventCreate(&e0));
            CK(cudaEventCreate(&e1));
            CK(cudaEventCreate(&e2));
            float best1 = 1e30f, best2 = 1e30f;
            for (int v = 0; v < 2; ++v) {
                CKS(build_tables(v, v));
                CK((launch_pass<PS, 1, K1_EO_INV, MAXP>(v, k1, ob1, st)));     // warm-up
                CK((launch_pass<PS, 1, K2_OE_LOCAL, MAXP>(v, k2b, ob2, st)));
                CK(cudaEventRecord(e0, st));
                for (int r = 0; r < 3; ++r) CK((launch_pass<PS, 1, K1_EO_INV, MAXP>(v, k1, ob1, st)));
                CK(cudaEventRecord(e1, st));
                for (int r = 0; r < 3; ++r) CK((launch_pass<PS, 1, K2_OE_LOCAL, MAXP>(v, k2b, ob2, st)));
                CK(cudaEventRecord(e2, st));
                CK(cudaEventSynchronize(e2));
                float t1 = 0.f, t2 = 0.f;
                CK(cudaEventElapsedTime(&t1, e0, e1));
                CK(cudaEventElapsedTime(&t2, e1, e2));
                if (t1 < best1) { best1 = t1; v1 = v; }
                if (t2 < best2) { best2 = t2; v2 = v; }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            cudaEventDestroy(e2);
            tuned[key] = {v1, v2};
        }
    }
    CKS(build_tables(v1, v2));
    auto iteration = [&]() -> cudaError_t {
        cudaError_t e = launch_cg_pupdate<PS, NC, MAXP>(pu, vbk, st);
        if (!e) e = launch_pass<PS, 1, K1_EO_INV, MAXP>(v1, k1, ob1, st);
        if (!e) e = launch_pass<PS, 1, K2_OE_LOCAL, MAXP>(v2, k2a, ob2, st);
        if (!e) e = launch_pass<PS, 1, K1_EO_INV, MAXP>(v1, k1b, ob1, st);
        if (!e) e = launch_pass<PS, 1, K2_OE_LOCAL, MAXP>(v2, k2b, ob2, st);
        if (!e) e = launch_cg_update<PS, PX, NC, MAXP>(up, vbk, st);
        return e;
    };
    cudaGraphExec_t gexec = nullptr;
    if (sp->use_graph) {
        cudaGraph_t graph;
        CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
        for (int it = 0; it < chunk; ++it) {
            cudaError_t e = iteration();
            if (e != cudaSuccess) {
                cudaStreamEndCapture(st, &graph);
                return fail(TM_ERR_CUDA, "capture: %s", cudaGetErrorString(e));
            }
        }
        CK(cudaStreamEndCapture(st, &graph));
        CK(cudaGraphInstantiate(&gexec, graph, 0));
        cudaGraphDestroy(graph);
    }
    tm_status worst = TM_OK;
    int remaining = 0;
    for (int q = 0; q < n; ++q) remaining += !done[q];
    while (remaining > 0) {
        if (gexec) CK(cudaGraphLaunch(gexec, st));
        else for (int it = 0; it < chunk; ++it) CK(iteration());
        // every running problem's control word in one synchronisation
        for (int q = 0; q < n; ++q)
            if (!done[q]) CK(cudaMemcpyAsync(cs[q]->h_ctl, cs[q]->ctl, sizeof(SolverCtl), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int q = 0; q < n; ++q) {
            if (done[q]) continue;
            tm_ctx* c = cs[q];
            SolverCtl& h = *c->h_ctl;
            if (h.flag == CTL_RUN) continue;
            infos[q].iters = h.iter;
            if (h.flag == CTL_BREAKDOWN) {
                infos[q].status = TM_ERR_BREAKDOWN; done[q] = 1; --remaining; worst = TM_ERR_BREAKDOWN;
                continue;
            }
            const int nbq = nblk(c->vh, BLAS_BS);
            if (PS != P64) {
                CK((launch_add_to64<P32, NC, 1>(vb1(c, w[q].x64, w[q].xs), nbq, st)));
                CK(cudaMemsetAsync(w[q].xs, 0, spinor_bytes(P32, NC, c->vh), st));
            }
            void *r64 = c->ws[WS_R64].first, *ax64 = c->ws[WS_AX64].first, *te64 = c->ws[WS_TE64].first,
                 *mid64 = c->ws[WS_MID64].first;
            const int saved_flag = h.flag;
            const double rr_old = h.rr_old;
            const int iters = h.iter;
            const bool dw = PS != P64 && !sp->fp64_updates;
            CKS(true_residual<1>(c, op, 0.0, w[q].x64, w[q].b64, r64, ax64, mid64, te64, st, &rr[q], false, dw));
            if (dw && rr[q] <= tol * tol * bb[q])   // confirmed in FP64
                CKS(true_residual<1>(c, op, 0.0, w[q].x64, w[q].b64, r64, ax64, mid64, te64, st, &rr[q]));
            infos[q].reliable_updates += 1;
            // true_residual overwrote h.shift only; restore the control word
            h.flag = saved_flag;
            if (rr[q] <= tol * tol * bb[q] || saved_flag == CTL_MAXITER || iters >= maxiter ||
                !std::isfinite(rr[q])) {
                infos[q].status = rr[q] <= tol * tol * bb[q] ? TM_OK
                                  : (std::isfinite(rr[q]) ? TM_ERR_NOT_CONVERGED : TM_ERR_BREAKDOWN);
                if (infos[q].status != TM_OK && worst == TM_OK) worst = (tm_status)infos[q].status;
                done[q] = 1;
                --remaining;
                h.flag = CTL_STOP;
                CKS(put_ctl(c, st));
                continue;
            }
            if (PS != P64) CK((launch_convert<PS, P64, NC, 1>(vb1(c, w[q].rs, r64), nbq, st)));
            h.beta = rr[q] / rr_old;
            h.rr = rr[q];
            h.iter = iters;
            h.shift = 0.0;
            h.stop_rr = std::max(tol * tol * bb[q], delta * delta * rr[q]);
            h.flag = CTL_RUN;
            CKS(put_ctl(c, st));
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    for (int q = 0; q < n; ++q) infos[q].true_rel_res = bb[q] > 0 ? std::sqrt(rr[q] / bb[q]) : 0.0;
    return worst;
}

extern "C" tm_status tm_solve_batch(tm_ctx** cs, int n, tm_op op, const tm_solve_params* sp, double** x,
                                    const double** b, tm_solve_info* infos, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!cs || !sp || !x || !b || !infos || n < 1 || n > MAXP) return fail(TM_ERR_ARG, "tm_solve_batch: bad argument");
    if (op != TM_MDAGM && op != TM_QPQM) return fail(TM_ERR_ARG, "tm_solve_batch: light normal operators only");
    CKS(check_prec(sp->sloppy));
    for (int q = 0; q < n; ++q) {
        if (!cs[q] || !x[q] || !b[q]) return fail(TM_ERR_ARG, "tm_solve_batch: null problem %d", q);
        if (cs[q]->device != cs[0]->device) return fail(TM_ERR_ARG, "tm_solve_batch: all contexts on one device");
    }
    CK(cudaSetDevice(cs[0]->device));
    const cudaStream_t st = cs[0]->sstream;
    CKS(enter_solver(cs[0], stream));
    std::vector<BatchWs> w(n);
    const int PS = sp->sloppy;
    for (int q = 0; q < n; ++q) {
        tm_ctx* c = cs[q];
        CKS(ensure_prec(c, P64, st));
        CKS(ensure_prec(c, PS, st));
        const size_t s64 = spinor_bytes(P64, 12, c->vh), ss = spinor_bytes(PS, 12, c->vh);
        CKS(ws_get(c, WS_X64, s64, &w[q].x64));
        CKS(ws_get(c, WS_B64, s64, &w[q].b64));
        CKS(ws_get(c, WS_P_S, ss, &w[q].ps));
        CKS(ws_get(c, WS_AP_S, ss, &w[q].aps));
        if (PS == P64) {
            CKS(ws_get(c, WS_TE64, s64, &w[q].tes));
            CKS(ws_get(c, WS_MID_S, ss, &w[q].mids));
            w[q].xs = w[q].x64;
            w[q].rs = nullptr;   // set to r64 in batch_core
        } else {
            CKS(ws_get(c, WS_TE_S, ss, &w[q].tes));
            CKS(ws_get(c, WS_MID_S, ss, &w[q].mids));
            CKS(ws_get(c, WS_R_S, ss, &w[q].rs));
            CKS(ws_get(c, WS_X_S, spinor_bytes(P32, 12, c->vh), &w[q].xs));
        }
        CKS(stage_in(c, 1, b[q], WS_STAGE_B, w[q].b64, st));
        CKS(stage_in(c, 1, x[q], WS_STAGE_X, w[q].x64, st));
    }
    tm_status s;
    switch (PS) {
        case P64: {
            // FP64 batch: the even temporary of the operator must not alias the residual's
            for (int q = 0; q < n; ++q) CKS(ws_get(cs[q], WS_TE_S, spinor_bytes(P64, 12, cs[q]->vh), &w[q].tes));
            s = batch_core<P64>(cs, n, op, sp, w, infos, st);
            break;
        }
        case P32: s = batch_core<P32>(cs, n, op, sp, w, infos, st); break;
        case PB16: s = batch_core<PB16>(cs, n, op, sp, w, infos, st); break;
        default: s = batch_core<PF16>(cs, n, op, sp, w, infos, st); break;
    }
    for (int q = 0; q < n; ++q) CKS(stage_out(cs[q], 1, x[q], WS_STAGE_X, w[q].x64, st));
    CK(cudaStreamSynchronize(st));
    const double secs = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    for (int q = 0; q < n; ++q) infos[q].seconds = secs;
    if (s != TM_OK) fail(s, "tm_solve_batch: at least one problem failed");
    return s;
}

// ---------------------------------------------------------------------------
// learned preconditioner: gauge-equivariant parallel-transport network
// ---------------------------------------------------------------------------
struct tm_ptc {
    int device = 0;
    int L = 0;
    int ch[9] = {};
    float2* W[8] = {};      // complex FP32 master weights [9][cout][cin][4][4]
    float2* m[8] = {};      // Adam first and second moments
    float2* v[8] = {};
    float2* G[8] = {};      // gradient accumulators
    void* wf[8] = {};       // BF16 real-embedded forward weights, 9 x 64 x 64
    void* wa[8] = {};       // BF16 real-embedded adjoint weights
    int step = 0;
    long V = 0;             // geometry of the activation buffers
    void* act[9] = {};      // activations per layer boundary, BF16 [ch][3][V] uint4
    void* del[2] = {};      // back-propagated deltas (8 channels)
    float* wpart = nullptr; // weight-gradient partials
    double* dpart = nullptr;
    double* dscal = nullptr;   // [0] ||e||^2, [1] loss sum, [2..] scratch
    double* hscal = nullptr;
    void* e32 = nullptr;       // training error vector (FP32 native odd)
    void* r32 = nullptr;       // training residual  (FP32 native odd)
    void* tmp32[2] = {};
    int nsm = 0;
    int* derr = nullptr;       // set by a layer kernel whose tensor-core wait ran out of its bound
    void* zmix = nullptr;      // per-path mixed fields of the layers with one output channel (9 channels)
    uint32_t* lp = nullptr;    // FP16 transport links [8][9][V] of context lp_uid at gauge generation lp_gen
    unsigned long long lp_uid = 0;
    long lp_gen = -1;
    double lp_bct = 0.0;
};

static size_t ptc_nw(const tm_ptc* n, int l) { return (size_t)9 * n->ch[l + 1] * n->ch[l] * 16; }

static tm_status ptc_embed_all(tm_ptc* n, cudaStream_t st) {
    for (int l = 0; l < n->L; ++l) CK(launch_ptc_embed_weights(n->W[l], n->ch[l], n->ch[l + 1], n->wf[l], n->wa[l], st));
    return TM_OK;
}

extern "C" tm_status tm_ptc_create(tm_ptc** out, int nlayers, const int* channels, int device) {
    if (!out || !channels || nlayers < 1 || nlayers > 8) return fail(TM_ERR_ARG, "tm_ptc_create: bad argument");
    if (channels[0] != 1 || channels[nlayers] != 1)
        return fail(TM_ERR_ARG, "tm_ptc_create: first and last channel counts must be 1");
    for (int l = 0; l <= nlayers; ++l) {
        const int c = channels[l];
        if (c != 1 && c != 2 && c != 4 && c != 8) return fail(TM_ERR_ARG, "tm_ptc_create: channels must be 1, 2, 4 or 8");
    }
    for (int l = 0; l < nlayers; ++l) {
        const int a = channels[l], b = channels[l + 1];
        const bool ok = (a == 1 && (b == 1 || b == 2 || b == 4 || b == 8)) || (b == 1 && (a == 2 || a == 4 || a == 8)) ||
                        (a == b);
        if (!ok) return fail(TM_ERR_UNSUPPORTED, "tm_ptc_create: layer %d (%d -> %d) has no kernel", l, a, b);
    }
    CK(cudaSetDevice(device));
    tm_ptc* n = new tm_ptc();
    n->device = device;
    n->L = nlayers;
    for (int l = 0; l <= nlayers; ++l) n->ch[l] = channels[l];
    cudaDeviceProp prop;
    CK(cudaGetDeviceProperties(&prop, device));
    n->nsm = prop.multiProcessorCount;
    for (int l = 0; l < nlayers; ++l) {
        const size_t b = sizeof(float2) * ptc_nw(n, l);
        CK(cudaMalloc(&n->W[l], b)); CK(cudaMemset(n->W[l], 0, b));
        CK(cudaMalloc(&n->m[l], b)); CK(cudaMemset(n->m[l], 0, b));
        CK(cudaMalloc(&n->v[l], b)); CK(cudaMemset(n->v[l], 0, b));
        CK(cudaMalloc(&n->G[l], b)); CK(cudaMemset(n->G[l], 0, b));
        CK(cudaMalloc(&n->wf[l], 2 * 9 * 64 * 64));
        CK(cudaMalloc(&n->wa[l], 2 * 9 * 64 * 64));
    }
    CK(cudaMalloc(&n->wpart, sizeof(float) * 9 * 4096 * n->nsm));
    CK(cudaMalloc(&n->dscal, sizeof(double) * 8));
    CK(cudaMallocHost(&n->hscal, sizeof(double) * 8));
    CK(cudaMalloc(&n->derr, sizeof(int)));
    CK(cudaMemset(n->derr, 0, sizeof(int)));
    CKS(ptc_embed_all(n, nullptr));
    CK(cudaDeviceSynchronize());
    *out = n;
    return TM_OK;
}

static void ptc_free_acts(tm_ptc* n) {
    for (auto& a : n->act) { cudaFree(a); a = nullptr; }
    for (auto& d : n->del) { cudaFree(d); d = nullptr; }
    cudaFree(n->dpart); n->dpart = nullptr;
    cudaFree(n->zmix); n->zmix = nullptr;
    cudaFree(n->lp); n->lp = nullptr;
    n->lp_uid = 0;
    n->lp_gen = -1;
    cudaFree(n->e32); cudaFree(n->r32); cudaFree(n->tmp32[0]); cudaFree(n->tmp32[1]);
    n->e32 = n->r32 = n->tmp32[0] = n->tmp32[1] = nullptr;
    n->V = 0;
}

extern "C" tm_status tm_ptc_destroy(tm_ptc* n) {
    if (!n) return TM_OK;
    cudaSetDevice(n->device);
    cudaDeviceSynchronize();
    for (int l = 0; l < n->L; ++l) {
        cudaFree(n->W[l]); cudaFree(n->m[l]); cudaFree(n->v[l]); cudaFree(n->G[l]);
        cudaFree(n->wf[l]); cudaFree(n->wa[l]);
    }
    ptc_free_acts(n);
    cudaFree(n->wpart);
    cudaFree(n->dscal);
    cudaFreeHost(n->hscal);
    cudaFree(n->derr);
    delete n;
    return TM_OK;
}

static tm_status ptc_buffers(tm_ptc* n, const tm_ctx* c) {
    const long V = 2 * c->vh;
    if (n->V == V) return TM_OK;
    ptc_free_acts(n);
    for (int l = 0; l <= n->L; ++l) CK(cudaMalloc(&n->act[l], (size_t)n->ch[l] * 3 * 16 * V));
    for (auto& d : n->del) CK(cudaMalloc(&d, (size_t)PTC_MAXC * 3 * 16 * V));
    CK(cudaMalloc(&n->dpart, sizeof(double) * ((V + 255) / 256)));
    CK(cudaMalloc(&n->zmix, (size_t)9 * 3 * 16 * V));
    CK(cudaMalloc(&n->lp, (size_t)8 * 9 * 4 * V));
    const size_t s32 = spinor_bytes(P32, 12, c->vh);
    CK(cudaMalloc(&n->e32, s32));
    CK(cudaMalloc(&n->r32, s32));
    CK(cudaMalloc(&n->tmp32[0], s32));
    CK(cudaMalloc(&n->tmp32[1], s32));
    n->V = V;
    return TM_OK;
}

static PtcGeom ptc_geom(const tm_ctx* c) {
    PtcGeom g{};
    g.X = c->g.X; g.Y = c->g.Y; g.Z = c->g.Z; g.T = c->g.T;
    g.vh = c->vh;
    g.V = 2 * c->vh;
    g.bc_t = (float)c->params.bc_t;
    g.gauge[0] = c->gaugeP[PF16][0];
    g.gauge[1] = c->gaugeP[PF16][1];
    g.lp = nullptr;
    return g;
}

// weights canonical: complex FP64 [layer][path 9][cout][cin][4][4], host pointer
extern "C" tm_status tm_ptc_set_weights(tm_ptc* n, const double* w) {
    if (!n || !w) return fail(TM_ERR_ARG, "tm_ptc_set_weights: null argument");
    CK(cudaSetDevice(n->device));
    size_t off = 0;
    for (int l = 0; l < n->L; ++l) {
        const size_t cnt = ptc_nw(n, l);
        std::vector<float2> h(cnt);
        for (size_t k = 0; k < cnt; ++k) h[k] = make_float2((float)w[2 * (off + k)], (float)w[2 * (off + k) + 1]);
        CK(cudaMemcpy(n->W[l], h.data(), sizeof(float2) * cnt, cudaMemcpyHostToDevice));
        off += cnt;
    }
    CKS(ptc_embed_all(n, nullptr));
    CK(cudaDeviceSynchronize());
    return TM_OK;
}

extern "C" tm_status tm_ptc_get_weights(const tm_ptc* n, double* w) {
    if (!n || !w) return fail(TM_ERR_ARG, "tm_ptc_get_weights: null argument");
    CK(cudaSetDevice(n->device));
    size_t off = 0;
    for (int l = 0; l < n->L; ++l) {
        const size_t cnt = ptc_nw(n, l);
        std::vector<float2> h(cnt);
        CK(cudaMemcpy(h.data(), n->W[l], sizeof(float2) * cnt, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < cnt; ++k) { w[2 * (off + k)] = h[k].x; w[2 * (off + k) + 1] = h[k].y; }
        off += cnt;
    }
    return TM_OK;
}

extern "C" tm_status tm_ptc_num_weights(const tm_ptc* n, size_t* count) {
    if (!n || !count) return fail(TM_ERR_ARG, "tm_ptc_num_weights: null argument");
    size_t s = 0;
    for (int l = 0; l < n->L; ++l) s += ptc_nw(n, l);
    *count = s;
    return TM_OK;
}

// Initial weights: the identity path carries scale * 1 between equal channel
// indices (a product of L layers then maps r to scale^L r), every other weight is
// uniform noise in [-noise, noise] (re and im) from splitmix64 seeded by `seed`.
extern "C" tm_status tm_ptc_init(tm_ptc* n, double scale, double noise, unsigned long long seed) {
    if (!n) return fail(TM_ERR_ARG, "tm_ptc_init: null argument");
    size_t total = 0;
    for (int l = 0; l < n->L; ++l) total += ptc_nw(n, l);
    std::vector<double> w(2 * total);
    uint64_t s = seed * 0x9e3779b97f4a7c15ull + 1;
    auto uni = [&]() {
        uint64_t z = (s += 0x9e3779b97f4a7c15ull);
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0) * 2.0 - 1.0;
    };
    size_t off = 0;
    for (int l = 0; l < n->L; ++l) {
        const int ci = n->ch[l], co = n->ch[l + 1];
        for (int p = 0; p < 9; ++p)
            for (int a = 0; a < co; ++a)
                for (int b = 0; b < ci; ++b)
                    for (int si = 0; si < 4; ++si)
                        for (int t = 0; t < 4; ++t) {
                            const size_t k = off + ((((size_t)p * co + a) * ci + b) * 4 + si) * 4 + t;
                            w[2 * k] = noise * uni();
                            w[2 * k + 1] = noise * uni();
                            if (p == 0 && a == b && si == t) w[2 * k] += scale;
                        }
        off += ptc_nw(n, l);
    }
    n->step = 0;
    for (int l = 0; l < n->L; ++l) {
        CK(cudaMemset(n->m[l], 0, sizeof(float2) * ptc_nw(n, l)));
        CK(cudaMemset(n->v[l], 0, sizeof(float2) * ptc_nw(n, l)));
    }
    return tm_ptc_set_weights(n, w.data());
}

// geometry of c with the network's transport-link field, rebuilt when the
// context (by its unique id), its gauge field or its time boundary phase changed
static tm_status ptc_geom_links(tm_ptc* n, tm_ctx* c, cudaStream_t st, PtcGeom* out) {
    PtcGeom g = ptc_geom(c);
    if (n->lp_uid != c->uid || n->lp_gen != c->gauge_gen || n->lp_bct != c->params.bc_t) {
        CK(launch_ptc_links(g, n->lp, st));
        n->lp_uid = c->uid;
        n->lp_gen = c->gauge_gen;
        n->lp_bct = c->params.bc_t;
    }
    g.lp = n->lp;
    *out = g;
    return TM_OK;
}

// z (FP32 native odd) = N(r) (FP32 native odd); activations kept in n->act
static tm_status ptc_forward(tm_ptc* n, tm_ctx* c, void* z, const void* r, cudaStream_t st) {
    PtcGeom g;
    CKS(ptc_geom_links(n, c, st, &g));
    CK(launch_ptc_embed_odd(P32, r, n->act[0], g, st));
    for (int l = 0; l < n->L; ++l)
        CK(launch_ptc_layer(n->ch[l], n->ch[l + 1], g, n->act[l], n->act[l + 1], n->wf[l], n->nsm, n->derr, n->zmix,
                            st));
    if (z) CK(launch_ptc_extract_odd(P32, n->act[n->L], z, g, st));
    return TM_OK;
}

// loss of (r, e) with activations from ptc_forward(r); gradients accumulate into G (scaled)
static tm_status ptc_backward(tm_ptc* n, tm_ctx* c, const void* e, float scale, cudaStream_t st) {
    PtcGeom g;
    CKS(ptc_geom_links(n, c, st, &g));
    CK(launch_ptc_loss_delta(n->act[n->L], e, n->del[0], g, n->dscal + 0, n->dpart, n->dscal + 1, st));
    int cur = 0;
    for (int l = n->L - 1; l >= 0; --l) {
        CK(launch_ptc_wgrad(n->ch[l], n->ch[l + 1], g, n->act[l], n->del[cur], n->wpart, n->nsm, n->G[l], scale,
                            n->derr, st));
        if (l > 0) {
            CK(launch_ptc_layer(n->ch[l + 1], n->ch[l], g, n->del[cur], n->del[1 - cur], n->wa[l], n->nsm, n->derr,
                                n->zmix, st));
            cur = 1 - cur;
        }
    }
    return TM_OK;
}

static tm_status ptc_prepare(tm_ptc* n, tm_ctx* c, cudaStream_t st) {
    if (c->device != n->device) return fail(TM_ERR_ARG, "network and context on different devices");
    CKS(ensure_prec(c, PF16, st));
    CKS(ensure_prec(c, P32, st));
    return ptc_buffers(n, c);
}

// after a synchronisation: report (and clear) a layer wait that ran out of its bound
static tm_status ptc_check_flag(tm_ptc* n) {
    int h = 0;
    CK(cudaMemcpy(&h, n->derr, sizeof(int), cudaMemcpyDeviceToHost));
    if (h != 0) {
        CK(cudaMemset(n->derr, 0, sizeof(int)));
        return fail(TM_ERR_TIMEOUT, "PTC layer: a wait on the tensor cores ran out of its bound");
    }
    return TM_OK;
}

extern "C" tm_status tm_ptc_sync(tm_ptc* n, void* stream) {
    if (!n) return fail(TM_ERR_ARG, "tm_ptc_sync: null argument");
    CK(cudaSetDevice(n->device));
    CK(cudaStreamSynchronize(S(stream)));
    return ptc_check_flag(n);
}

extern "C" tm_status tm_wait_selftest(int device, double seconds, int* timed_out) {
    if (!timed_out || !(seconds > 0) || seconds > 10) return fail(TM_ERR_ARG, "tm_wait_selftest: bad argument");
    CK(cudaSetDevice(device));
    int* d = nullptr;
    CK(cudaMalloc(&d, sizeof(int)));
    tm_status s = TM_OK;
    int h = -1;
    if (launch_ptc_wait_selftest((long long)(seconds * 1e9), d, nullptr) != cudaSuccess ||
        cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        s = fail(TM_ERR_CUDA, "tm_wait_selftest: %s", cudaGetErrorString(cudaGetLastError()));
    cudaFree(d);
    *timed_out = h;
    return s;
}

extern "C" tm_status tm_ptc_apply(tm_ptc* n, tm_ctx* c, void* out, const void* in, void* stream) {
    if (!n || !c || !out || !in || out == in) return fail(TM_ERR_ARG, "tm_ptc_apply: bad argument");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    CKS(ptc_prepare(n, c, st));
    return ptc_forward(n, c, out, in, st);
}

// loss and gradient of one pair (canonical FP64 r, e, host or device); grad host, same layout as weights
extern "C" tm_status tm_ptc_grad(tm_ptc* n, tm_ctx* c, const double* r, const double* e, double* loss, double* grad,
                                 void* stream) {
    if (!n || !c || !r || !e || !loss || !grad) return fail(TM_ERR_ARG, "tm_ptc_grad: null argument");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = S(stream);
    CKS(ptc_prepare(n, c, st));
    void* b64;
    CKS(ws_get(c, WS_B64, spinor_bytes(P64, 12, c->vh), &b64));
    CKS(stage_in(c, 1, r, WS_STAGE_B, b64, st));
    CK((launch_convert<P32, P64, 12, 1>(vb1(c, n->r32, b64), nblk(c->vh, BLAS_BS), st)));
    CKS(stage_in(c, 1, e, WS_STAGE_B, b64, st));
    CK((launch_convert<P32, P64, 12, 1>(vb1(c, n->e32, b64), nblk(c->vh, BLAS_BS), st)));
    CK((launch_norm2<P32, 12, 1>(vb1(c, n->e32, nullptr, nullptr, nullptr, n->dscal + 0), nblk(c->vh, BLAS_BS), st)));
    for (int l = 0; l < n->L; ++l) CK(cudaMemsetAsync(n->G[l], 0, sizeof(float2) * ptc_nw(n, l), st));
    CKS(ptc_forward(n, c, nullptr, n->r32, st));
    CKS(ptc_backward(n, c, n->e32, 1.0f, st));
    CK(cudaMemcpyAsync(n->hscal, n->dscal, sizeof(double) * 2, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CKS(ptc_check_flag(n));
    *loss = n->hscal[1] / n->hscal[0];
    size_t off = 0;
    for (int l = 0; l < n->L; ++l) {
        const size_t cnt = ptc_nw(n, l);
        std::vector<float2> h(cnt);
        CK(cudaMemcpy(h.data(), n->G[l], sizeof(float2) * cnt, cudaMemcpyDeviceToHost));
        for (size_t k = 0; k < cnt; ++k) { grad[2 * (off + k)] = h[k].x; grad[2 * (off + k) + 1] = h[k].y; }
        off += cnt;
    }
    return TM_OK;
}

// Training on solver-generated pairs: e ~ complex Gaussian (Philox4x32-10 keyed by
// seed, stream = pair index), r = A e with the FP32 operator of the pair's context
// (pairs cycle through the contexts), loss ||N(r) - e||^2/||e||^2, Adam every
// `batch` pairs on the mean gradient.  losses (host, npairs) receives every loss.
extern "C" tm_status tm_ptc_train(tm_ptc* n, tm_ctx** cs, int nctx, tm_op op, int npairs, int batch, double lr,
                                  unsigned long long seed, double* losses, void* stream) {
    if (!n || !cs || nctx < 1 || npairs < 1 || batch < 1 || !(lr > 0)) return fail(TM_ERR_ARG, "tm_ptc_train: bad argument");
    if (op != TM_MDAGM && op != TM_QPQM) return fail(TM_ERR_ARG, "tm_ptc_train: light normal operator only");
    for (int q = 0; q < nctx; ++q)
        if (!cs[q] || cs[q]->vh != cs[0]->vh || cs[q]->device != n->device)
            return fail(TM_ERR_ARG, "tm_ptc_train: contexts must share device and volume");
    CK(cudaSetDevice(n->device));
    const cudaStream_t st = S(stream);
    for (int q = 0; q < nctx; ++q) CKS(ptc_prepare(n, cs[q], st));
    double* dloss = nullptr;
    CK(cudaMalloc(&dloss, sizeof(double) * 2 * npairs));
    std::memset(cs[0]->h_ctl, 0, sizeof(SolverCtl));
    for (int q = 0; q < nctx; ++q) {
        std::memset(cs[q]->h_ctl, 0, sizeof(SolverCtl));
        CKS(put_ctl(cs[q], st));
    }
    tm_status status = TM_OK;
    for (int k = 0; k < npairs && status == TM_OK; ++k) {
        tm_ctx* c = cs[k % nctx];
        void *te, *mid;
        CKS(ws_get(c, WS_TE_S, spinor_bytes(P32, 12, c->vh), &te));
        CKS(ws_get(c, WS_MID_S, spinor_bytes(P32, 12, c->vh), &mid));
        CK(launch_ptc_gauss_odd(n->e32, c->vh, seed, (unsigned long long)k, st));
        CK((normal_op<P32, 1>(c, op, n->r32, n->e32, mid, te, st, nullptr, FIN_NONE)));
        CK((launch_norm2<P32, 12, 1>(vb1(c, n->e32, nullptr, nullptr, nullptr, n->dscal + 0), nblk(c->vh, BLAS_BS), st)));
        CKS(ptc_forward(n, c, nullptr, n->r32, st));
        CKS(ptc_backward(n, c, n->e32, 1.0f / batch, st));
        CK(cudaMemcpyAsync(dloss + 2 * k, n->dscal, sizeof(double) * 2, cudaMemcpyDeviceToDevice, st));
        if ((k + 1) % batch == 0 || k + 1 == npairs) {
            n->step += 1;
            for (int l = 0; l < n->L; ++l)
                CK(launch_ptc_adam(n->W[l], n->m[l], n->v[l], n->G[l], (int)ptc_nw(n, l), (float)lr, 0.9f, 0.999f,
                                   1e-8f, n->step, st));
            CKS(ptc_embed_all(n, st));
        }
    }
    std::vector<double> h(2 * (size_t)npairs);
    CK(cudaMemcpyAsync(h.data(), dloss, sizeof(double) * 2 * npairs, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    cudaFree(dloss);
    CKS(ptc_check_flag(n));
    if (losses)
        for (int k = 0; k < npairs; ++k) losses[k] = h[2 * k + 1] / h[2 * k];
    return status;
}

extern "C" tm_status tm_ptc_save(const tm_ptc* n, const char* path) {
    if (!n || !path) return fail(TM_ERR_ARG, "tm_ptc_save: null argument");
    CK(cudaSetDevice(n->device));
    FILE* f = fopen(path, "wb");
    if (!f) return fail(TM_ERR_ARG, "tm_ptc_save: cannot open %s", path);
    const char magic[8] = {'T', 'M', 'P', 'T', 'C', '1', 0, 0};
    fwrite(magic, 1, 8, f);
    fwrite(&n->L, sizeof(int), 1, f);
    fwrite(n->ch, sizeof(int), n->L + 1, f);
    fwrite(&n->step, sizeof(int), 1, f);
    for (int l = 0; l < n->L; ++l) {
        const size_t cnt = ptc_nw(n, l);
        std::vector<float2> h(cnt);
        for (float2* src : {n->W[l], n->m[l], n->v[l]}) {
            if (cudaMemcpy(h.data(), src, sizeof(float2) * cnt, cudaMemcpyDeviceToHost) != cudaSuccess) {
                fclose(f);
                return fail(TM_ERR_CUDA, "tm_ptc_save: copy failed");
            }
            fwrite(h.data(), sizeof(float2), cnt, f);
        }
    }
    fclose(f);
    return TM_OK;
}

extern "C" tm_status tm_ptc_load(tm_ptc* n, const char* path) {
    if (!n || !path) return fail(TM_ERR_ARG, "tm_ptc_load: null argument");
    CK(cudaSetDevice(n->device));
    FILE* f = fopen(path, "rb");
    if (!f) return fail(TM_ERR_ARG, "tm_ptc_load: cannot open %s", path);
    char magic[8];
    int L = 0, ch[9] = {}, step = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "TMPTC1", 6) == 0 && fread(&L, sizeof(int), 1, f) == 1 &&
              L == n->L && fread(ch, sizeof(int), L + 1, f) == (size_t)(L + 1) && fread(&step, sizeof(int), 1, f) == 1;
    for (int l = 0; ok && l <= L; ++l) ok = ch[l] == n->ch[l];
    for (int l = 0; ok && l < n->L; ++l) {
        const size_t cnt = ptc_nw(n, l);
        std::vector<float2> h(cnt);
        for (float2* dst : {n->W[l], n->m[l], n->v[l]}) {
            ok = ok && fread(h.data(), sizeof(float2), cnt, f) == cnt;
            if (ok) ok = cudaMemcpy(dst, h.data(), sizeof(float2) * cnt, cudaMemcpyHostToDevice) == cudaSuccess;
        }
    }
    fclose(f);
    if (!ok) return fail(TM_ERR_ARG, "tm_ptc_load: %s does not hold a network of this shape", path);
    n->step = step;
    CKS(ptc_embed_all(n, nullptr));
    CK(cudaDeviceSynchronize());
    return TM_OK;
}

// ---------------------------------------------------------------------------
// flexible CG with the network as preconditioner (Notay's FCG, truncation 1):
//   z_k = N(r_k);  p_k = z_k - (<q_{k-1}, z_k> / <p_{k-1}, q_{k-1}>) p_{k-1};  q_k = A p_k;
//   alpha = <p_k, r_k> / <p_k, q_k>;  x += alpha p_k;  r -= alpha q_k.
// Vectors FP32, operator FP32, network BF16; every time the iterated residual has
// dropped by `delta` the solution is folded into FP64 and r = b - A x is
// recomputed in double-word arithmetic (reliable update; FP64 once it is below
// the tolerance), restarting the recursion.
// ---------------------------------------------------------------------------
extern "C" tm_status tm_solve_fcg(tm_ctx* c, tm_op op, tm_ptc* n, const tm_solve_params* sp, double* x,
                                  const double* b, tm_solve_info* info, void* stream) {
    const auto t0 = std::chrono::steady_clock::now();
    if (!c || !n || !sp || !x || !b || !info) return fail(TM_ERR_ARG, "tm_solve_fcg: null argument");
    if (op != TM_MDAGM && op != TM_QPQM) return fail(TM_ERR_ARG, "tm_solve_fcg: light normal operator only");
    CK(cudaSetDevice(c->device));
    const cudaStream_t st = c->sstream;
    CKS(enter_solver(c, stream));
    CKS(ensure_prec(c, P64, st));
    CKS(ptc_prepare(n, c, st));
    const long vh = c->vh;
    const int nb = nblk(vh, BLAS_BS);
    const size_t s64 = spinor_bytes(P64, 12, vh), s32 = spinor_bytes(P32, 12, vh);
    void *x64, *b64, *r64, *ax64, *te64, *mid64, *xs, *rs, *z, *p, *q, *te, *mid;
    CKS(ws_get(c, WS_X64, s64, &x64));
    CKS(ws_get(c, WS_B64, s64, &b64));
    CKS(ws_get(c, WS_R64, s64, &r64));
    CKS(ws_get(c, WS_AX64, s64, &ax64));
    CKS(ws_get(c, WS_TE64, s64, &te64));
    CKS(ws_get(c, WS_MID64, s64, &mid64));
    CKS(ws_get(c, WS_X_S, s32, &xs));
    CKS(ws_get(c, WS_R_S, s32, &rs));
    CKS(ws_get(c, WS_P_S, s32, &p));
    CKS(ws_get(c, WS_AP_S, s32, &q));
    CKS(ws_get(c, WS_TE_S, s32, &te));
    CKS(ws_get(c, WS_MID_S, s32, &mid));
    CKS(ws_get(c, WS_FCG_Z, s32, &z));
    CKS(stage_in(c, 1, b, WS_STAGE_B, b64, st));
    CKS(stage_in(c, 1, x, WS_STAGE_X, x64, st));
    const double tol = sp->tol > 0 ? sp->tol : 1e-10;
    const int maxiter = sp->maxiter > 0 ? sp->maxiter : 10000;
    const double delta = sp->delta > 0 ? sp->delta : default_delta(P32);   // FP32 vectors
    double bb;
    CKS((norm2_dev<P64, 12>(c, b64, st, &bb)));
    info->iters = 0;
    info->reliable_updates = 0;
    if (!std::isfinite(bb)) return fail(TM_ERR_BREAKDOWN, "tm_solve_fcg: right-hand side is not finite");
    double rr;
    bool x0 = false;
    CKS(is_zero64<1>(c, x64, st, &x0));
    CKS(true_residual<1>(c, op, 0.0, x64, b64, r64, ax64, mid64, te64, st, &rr, x0));
    const double target = tol * tol * bb;
    std::memset(c->h_ctl, 0, sizeof(SolverCtl));
    CKS(put_ctl(c, st));
    double* d2 = c->d_scal + 2;
    auto cdot = [&](const void* a, const void* bq, double* re, double* im) -> tm_status {
        CK(launch_cdot32(a, bq, vh, c->partial, c->counter, d2, st));
        CK(cudaMemcpyAsync(c->h_scal, d2, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        *re = c->h_scal[0];
        *im = c->h_scal[1];
        return TM_OK;
    };
    tm_status status = TM_OK;
    int its = 0;
    while (rr > target && bb > 0) {
        // (re)start from the recomputed residual
        CK((launch_convert<P32, P64, 12, 1>(vb1(c, rs, r64), nb, st)));
        CK(cudaMemsetAsync(xs, 0, s32, st));
        const double rr_start = rr;
        double pq_old = 0.0;
        bool first = true;
        double rr_it = rr;
        while (rr_it > std::max(target, delta * delta * rr_start) && its < maxiter) {
            CKS(ptc_forward(n, c, z, rs, st));
            if (first) {
                CK(cudaMemcpyAsync(p, z, s32, cudaMemcpyDeviceToDevice, st));
            } else {
                // p = z + beta p_old in place, beta = -<q_old, z> / <p_old, q_old>; p and q
                // still hold the previous direction and its image here
                double qr, qi;
                CKS(cdot(q, z, &qr, &qi));
                CK(launch_cxpay32(p, z, -qr / pq_old, -qi / pq_old, vh, st));
            }
            // q = A p with <p, q> = ||Q p||^2 fused
            CK((normal_op<P32, 1>(c, op, q, p, mid, te, st, c->ctl, FIN_STORE)));
            CK(cudaMemcpyAsync(c->h_scal + 4, &c->ctl->result, sizeof(double), cudaMemcpyDeviceToHost, st));
            double pr, pi;
            CKS(cdot(p, rs, &pr, &pi));
            const double pq = c->h_scal[4];
            if (!(pq > 0) || !std::isfinite(pq)) { status = TM_ERR_BREAKDOWN; break; }
            const double ar = pr / pq, ai = pi / pq;
            CK(launch_caxpy32(xs, p, ar, ai, vh, st));
            CK(launch_caxpy32(rs, q, -ar, -ai, vh, st));
            pq_old = pq;
            first = false;
            ++its;
            CKS((norm2_dev<P32, 12>(c, rs, st, &rr_it)));
            if (!std::isfinite(rr_it)) { status = TM_ERR_BREAKDOWN; break; }
        }
        if (status != TM_OK) break;
        CK((launch_add_to64<P32, 12, 1>(vb1(c, x64, xs), nb, st)));
        const bool dw = !sp->fp64_updates;
        CKS(true_residual<1>(c, op, 0.0, x64, b64, r64, ax64, mid64, te64, st, &rr, false, dw));
        if (dw && rr <= target)   // confirmed in FP64
            CKS(true_residual<1>(c, op, 0.0, x64, b64, r64, ax64, mid64, te64, st, &rr));
        info->reliable_updates += 1;
        if (its >= maxiter && rr > target) { status = TM_ERR_NOT_CONVERGED; break; }
    }
    info->iters = its;
    info->true_rel_res = bb > 0 ? std::sqrt(rr / bb) : 0.0;
    info->status = status;
    CKS(stage_out(c, 1, x, WS_STAGE_X, x64, st));
    CK(cudaStreamSynchronize(st));
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    CKS(ptc_check_flag(n));
    if (status != TM_OK) return fail(status, "tm_solve_fcg: %s", status == TM_ERR_BREAKDOWN ? "breakdown" : "not converged");
    return TM_OK;
}

namespace tmk {
// record an error message for tm_last_error from another translation unit
tm_status tmk_fail_msg(tm_status s, const char* msg) { return fail(s, "%s", msg); }

// for the other translation units (multigrid): error messages, precision copies
// of the links and clover terms, context workspace
tm_status tmk_failf(tm_status s, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return s;
}
tm_status tmk_ensure_prec(tm_ctx* c, int P, cudaStream_t st) { return ensure_prec(c, P, st); }
tm_status tmk_ws_get(tm_ctx* c, int id, size_t bytes, void** out) { return ws_get(c, id, bytes, out); }
}  // namespace tmk
