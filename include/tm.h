/*
 * tm.h -- C ABI of the GB300 (sm_103a) even-odd twisted-mass clover solver library.
 *
 * Paper: "Twisted mass ensemble generation on GPU machines" (arXiv 2212.06635).
 * The library applies the asymmetric even-odd preconditioned operators of Sec. 2
 * (eq:hQpm for the light doublet, eq:hQh for the non-degenerate heavy doublet)
 * and solves with them by CG, mixed-precision CG with reliable updates (Sec. 4.1,
 * "MP-CG") and multishift CG with shift-by-shift refinement (Sec. 4.2).
 *
 * Conventions (fixed here; the paper leaves them open):
 *   dims          {X, Y, Z, T}, each even and >= 2; lex = ((t*Z+z)*Y+y)*X+x;
 *                 parity = (x+y+z+t) mod 2.  Solves live on ODD sites
 *                 (ODD_ODD_ASYMMETRIC, Sec. 2); odd site k has lex/2 == k.
 *   operator      hopping normalisation
 *                   M = A + i 2 kappa mu g5 - kappa H,
 *                   H psi(x) = sum_mu (1-g_mu) U_mu(x) psi(x+mu) + (1+g_mu) U_mu(x-mu)^+ psi(x-mu)
 *                   A = 1 - kappa csw sum_{mu<nu} g_mu g_nu F_munu (clover leaf, traceless),
 *                 chiral gamma basis with g5 = diag(1,1,-1,-1).  Heavy doublet:
 *                   M_h = M(mu=0) x 1_f + i 2 kappa mubar g5 tau3 - 2 kappa epsbar tau1.
 *                 kappa, csw, mu, mubar, epsbar are the bare (mass-normalised) values.
 *   boundary      periodic in space; bc_t (+1 or -1) multiplies hops across t = T-1 <-> 0.
 *   canonical     host/device FP64, C order, interleaved complex (re, im):
 *     gauge       [t][z][y][x][mu 4][row 3][col 3]        mu = 0:x 1:y 2:z 3:t
 *     odd field   [site_o][spin 4][colour 3]              (light, 24 doubles per site)
 *                 [site_o][flavour 2][spin 4][colour 3]   (heavy, 48 doubles per site)
 *   native        the library's own device layout of a field in a storage precision
 *                 (structure of arrays over sites; 16-bit fields carry one FP32 scale
 *                 per site).  Obtain sizes with tm_field_bytes and convert with
 *                 tm_field_import / tm_field_export.
 *
 * Ownership: every pointer argument stays owned by the caller; the library copies
 * what it keeps (gauge field, clover terms) into memory owned by the tm_ctx.
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Operator and field calls are stream-ordered and do not synchronise;
 * tm_solve_* and tm_power_iteration synchronise `stream` before returning so that
 * the info records are filled.
 * Errors: every call returns a tm_status; tm_last_error() returns a message for
 * the calling thread's most recent failure.  No call aborts the process, and no
 * kernel traps: device-side failures are reported through status words.
 */
#ifndef TM_H
#define TM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tm_ctx tm_ctx;

typedef enum {
    TM_OK = 0,
    TM_ERR_ARG = 1,            /* invalid argument (null pointer, bad size, misaligned) */
    TM_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    TM_ERR_OOM = 3,            /* device allocation failed */
    TM_ERR_STALE = 4,          /* clover term older than the gauge field (call tm_clover_compute) */
    TM_ERR_NOT_CONVERGED = 5,  /* maxiter reached before the tolerance */
    TM_ERR_BREAKDOWN = 6,      /* <p, A p> <= 0 or not finite */
    TM_ERR_TIMEOUT = 7,
    TM_ERR_UNSUPPORTED = 8
} tm_status;

typedef enum { TM_F64 = 0, TM_F32 = 1, TM_BF16 = 2, TM_F16 = 3 } tm_prec;

typedef enum {
    TM_QHAT_PLUS = 0,    /* Q_hat_+  (eq:hQpm, + sign)                          light */
    TM_QHAT_MINUS = 1,   /* Q_hat_-  = Q_hat_+^dagger                           light */
    TM_MDAGM = 2,        /* M_hat^dagger M_hat = Q_hat_- Q_hat_+  (HPD)         light */
    TM_QPQM = 3,         /* Q_hat_+ Q_hat_-  (HMC ordering, HPD)               light */
    TM_QH = 4,           /* Q_hat_h  (eq:hQh)                                   heavy */
    TM_QH_DAG = 5,       /* Q_hat_h^dagger = tau1 Q_hat_h tau1 (mubar -> -mubar) heavy */
    TM_QH_SQ = 6,        /* Q_hat_h Q_hat_h^dagger  (HPD)                       heavy */
    TM_WHAT_PLUS = 7,    /* W_hat_+(rho) = Q_hat_+ + i rho (eq:hWpm)            light */
    TM_WHAT_MINUS = 8,   /* W_hat_-(rho) = Q_hat_- - i rho = W_hat_+^dagger     light */
    TM_WHAT_SQ = 9       /* W_hat_- W_hat_+ = W_hat_+^dagger W_hat_+  (HPD)     light */
} tm_op;

typedef struct {
    double kappa, csw;
    double mu;          /* light twisted mass (eq:hQpm) */
    double mubar;       /* heavy doublet mu_sigma (eq:hQh) */
    double epsbar;      /* heavy doublet mu_delta (eq:hQh) */
    int bc_t;           /* +1 periodic, -1 antiperiodic in time */
    double rho;         /* mass-preconditioning mass of W_hat (eq:hWpm); enters as
                           i 2 kappa rho on odd sites and leaves the clover inverse
                           rho-independent, as Sec. 2 notes */
} tm_params;

typedef struct {
    double tol;          /* target FP64 true relative residual ||b - A x|| / ||b|| */
    int maxiter;         /* bound on Krylov iterations (all restarts together) */
    tm_prec sloppy;      /* storage precision of the inner iteration; TM_F64 = plain FP64 CG */
    double delta;        /* reliable-update trigger: ||r_sloppy|| < delta * ||r_true_last||;
                            <= 0 selects a default of about sqrt(unit roundoff) of the
                            sloppy storage: FP16 0.02, BF16 0.06, FP32 0.002 */
    int chunk;           /* iterations enqueued between two host checks (0 = default 16) */
    int use_graph;       /* capture the chunk in a CUDA graph and replay it */
    tm_prec refine;      /* tm_solve_multishift only: storage precision of the
                            shift-by-shift refinement CG; TM_F64 (0) = same as
                            sloppy.  TM_F16 after an FP32 multishift is Sec. 4.2's
                            "single precision MS-CG with double-half shift-by-shift
                            refinement" */
    int fp64_updates;    /* mixed solvers: 1 recomputes every reliable-update residual
                            with the native FP64 operator; 0 (default) uses the
                            double-word operator (tm_apply_Mhat_dw) and FP64 only to
                            confirm a residual below tol */
} tm_solve_params;

typedef struct {
    int iters;            /* Krylov iterations */
    int reliable_updates; /* true-residual recomputations (double-word arithmetic
                             in the mixed solvers, FP64 in plain FP64 CG) */
    int status;           /* tm_status of this solve */
    double true_rel_res;  /* FP64 ||b - A x|| / ||b|| of the returned x */
    double seconds;       /* wall time of the call */
} tm_solve_info;

/* Context: one lattice on one device.  dims as above; device = CUDA ordinal.
 * Fails with TM_ERR_ARG for odd or < 2 extents, or a volume of 2^31 sites or
 * more (site indices are 32-bit). */
tm_status tm_create(tm_ctx** ctx, const int dims[4], int device);
tm_status tm_destroy(tm_ctx* ctx);

/* Copy a canonical FP64 gauge field (host or device pointer, detected) into the
 * context and record gauge_id (the position along a trajectory, Sec. 3,
 * tm_GaugeState_t).  Marks every derived object (low-precision links, clover
 * terms) stale, as Sec. 3's update_tm_gauge_id cascade does. */
tm_status tm_gauge_load(tm_ctx* ctx, const double* links, double gauge_id, void* stream);
tm_status tm_gauge_id(const tm_ctx* ctx, double* gauge_id);

/* Build the clover term A (odd sites) and the even-site inverses
 * (A_ee +- i 2 kappa mu g5)^-1 and, when mubar or epsbar is non-zero, the heavy
 * block inverse of eq:hQh, in FP64, and store them in every storage precision
 * that is later requested.  A no-op when gauge_id and params are unchanged. */
tm_status tm_clover_compute(tm_ctx* ctx, const tm_params* params, void* stream);

/* Debug/test export of the FP64 clover blocks of all sites of one parity,
 * layout [site_cb][chirality 2][6][6] complex (chirality 0 = spins 0,1). */
tm_status tm_clover_export(tm_ctx* ctx, int parity, double* out, void* stream);

/* Bytes of one native odd-site field: nflavour 1 (light) or 2 (heavy). */
tm_status tm_field_bytes(const tm_ctx* ctx, tm_prec prec, int nflavour, size_t* bytes);
/* canonical FP64 <-> native (device).  The canonical pointer may be a host
 * pointer or a device pointer.  16-byte aligned.  A host pointer is copied
 * through one of three library-owned device staging buffers per direction:
 *   - pageable host memory: the call synchronises `stream` before returning;
 *   - pinned host memory (cudaMallocHost / cudaHostRegister): the call is
 *     stream-ordered like the device case; the caller keeps the source unchanged
 *     (import) or leaves the destination unread (export) until `stream` has
 *     passed the call, so imports and exports on different streams can overlap
 *     an operator running on a third. */
tm_status tm_field_import(tm_ctx* ctx, tm_prec prec, int nflavour, void* dst_native,
                          const double* src_canonical, void* stream);
tm_status tm_field_export(tm_ctx* ctx, tm_prec prec, int nflavour, double* dst_canonical,
                          const void* src_native, void* stream);

/* *result (device pointer, FP64) = ||field||^2 of a native field: per-thread sums
 * in the arithmetic precision, FP64 across threads and blocks, block partials
 * summed in a fixed order by the last block (deterministic for a given size).
 * Stream-ordered; uses the context's reduction scratch. */
tm_status tm_field_norm2(tm_ctx* ctx, tm_prec prec, int nflavour, const void* field, double* result,
                         void* stream);

/* Allocation-free variant of tm_field_norm2, for callers that cannot allocate
 * device memory when they need a norm: a host framework that has reserved the
 * whole device memory budget for its own pool (a side cudaMalloc would fail or
 * take memory already promised elsewhere), or a latency-critical loop that must
 * never reach the device allocator (cudaMalloc / cudaFree can synchronise the
 * device).  The paper has no counterpart: this is a library service, not part of
 * the method.  Same arguments, result and reduction order as tm_field_norm2, but
 * the block partials live in a fixed array in the library's device memory (about
 * 512 KB, held by every GPU that loads the library until exit) instead of the
 * context's scratch.  Limit: at most 16,777,216 sites per parity (TM_ERR_ARG
 * beyond).  field and result must be device pointers (TM_ERR_ARG otherwise,
 * before any launch).  The first call on a device looks up that array's device
 * address, so make the first call before any stream capture.  All calls share
 * the array, which keeps the last call's partial sums (each call overwrites the
 * ones it reads and zeroes the counter first): calls whose executions overlap on
 * the GPU (different streams, or different contexts on one device) race and give
 * wrong results.  Calls no cudaMalloc, cudaFree or allocating library routine. */
tm_status tm_field_norm2_noalloc(const tm_ctx* ctx, tm_prec prec, int nflavour, const void* field,
                                 double* result, void* stream);

/* out = op(in), native fields of precision prec on the device (eq:hQpm / eq:hQh).
 * Light ops take nflavour-1 fields, heavy ops nflavour-2 fields.  out != in.
 * Returns TM_ERR_STALE if the clover term predates the gauge field, TM_ERR_ARG
 * for a field that is not device memory (checked before any launch, as in
 * every call that takes a native field).  Operator
 * calls on one context share its intermediate fields: issue them on one stream
 * (field imports and exports may run on others). */
tm_status tm_apply_Mhat(tm_ctx* ctx, tm_op op, tm_prec prec, void* out, const void* in,
                        void* stream);

/* out = op(in) on native FP64 fields (the layout of tm_apply_Mhat with TM_F64),
 * evaluated in double-word arithmetic: each real is carried as an unevaluated sum
 * of two FP32 numbers (a 48-bit significand), in and out are rounded to that on
 * the way in and out, and links and clover blocks come from double-word copies
 * made from the FP64 ones when stale.  This is how the mixed-precision solvers
 * recompute their true residuals between reliable updates (Sec. 4.1's reliable
 * updates): on this GPU the FP32 units outrun the FP64 ones by ~70x.  A solver
 * confirms a residual below its tolerance with the native FP64 operator.
 * Errors as tm_apply_Mhat. */
tm_status tm_apply_Mhat_dw(tm_ctx* ctx, tm_op op, void* out, const void* in, void* stream);

/* The even pass of one Schur operator alone: out = M_ee(s)^-1 H_eo in, the even
 * sites' reconstruction term of eq:hQpm / eq:hQh (x_e = M_ee^-1 (b_e + kappa H_eo x_o)
 * for the full system).  op = TM_QHAT_PLUS / TM_QH (s = +) or TM_QHAT_MINUS /
 * TM_QH_DAG (s = -); in: native odd-site field, out: native field of the same
 * precision and flavour count holding the even sites (site k has lex/2 == k).
 * Stream-ordered; the errors of tm_apply_Mhat. */
tm_status tm_apply_even(tm_ctx* ctx, tm_op op, tm_prec prec, void* out, const void* in, void* stream);

/* Solve A x = b, A = TM_MDAGM, TM_QPQM, TM_QH_SQ or TM_WHAT_SQ, by CG (sloppy = TM_F64) or by
 * mixed-precision CG with reliable updates (Sec. 4.1; the true residuals between
 * updates in double-word arithmetic, see tm_apply_Mhat_dw, a residual below
 * the tolerance confirmed in FP64).  x, b canonical FP64, host or device
 * pointers; x is the initial guess on entry (zero it for none). */
tm_status tm_solve_cg(tm_ctx* ctx, tm_op op, const tm_solve_params* sp, double* x,
                      const double* b, tm_solve_info* info, void* stream);

/* Solve (A + shifts[k]) x[k] = b for nshift shifts (A = TM_MDAGM or TM_QH_SQ) with
 * one multishift CG in the sloppy precision (Sec. 4.2), then refine each shift
 * by mixed-precision CG to sp->tol ("shift-by-shift refinement").  x[k] canonical
 * FP64 output buffers (host or device); infos has nshift records. */
tm_status tm_solve_multishift(tm_ctx* ctx, tm_op op, int nshift, const double* shifts,
                              double** x, const double* b, const tm_solve_params* sp,
                              tm_solve_info* infos, void* stream);

/* Rational approximation of x^-1/2 on [lo, hi] with n poles (1 <= n <= 16), the
 * form Sec. 4.2's rational monomials of the heavy doublet apply with one
 * multishift solve: r(x) = a0 + sum_k a[k] / (x + sigma[k]), Zolotarev's best
 * approximation in the relative sense; *delta = max |sqrt(x) r(x) - 1| on
 * [lo, hi].  Host computation only (no context, no device). */
tm_status tm_rational_inv_sqrt(int n, double lo, double hi, double* a0, double* a, double* sigma,
                               double* delta);

/* y = r(A) b = a0 b + sum_k a[k] (A + sigma[k])^-1 b for A = TM_MDAGM, TM_QPQM or
 * TM_QH_SQ: one tm_solve_multishift (sloppy multishift CG, shift-by-shift
 * refinement to sp->tol, Sec. 4.2) and one FP64 combination on the device.
 * y, b: canonical FP64 (host or device); infos: n records of the solves.
 * Synchronises like the solvers. */
tm_status tm_rational_apply(tm_ctx* ctx, tm_op op, int n, double a0, const double* a, const double* sigma,
                            double* y, const double* b, const tm_solve_params* sp, tm_solve_info* infos,
                            void* stream);

/* The correction term of the rational approximation (Fig. 4's heatbath and
 * acceptance): y = (1 + Z)^p b with Z = A r(A)^2 - 1, r the rational function of
 * (a0, a, sigma), summed as the binomial series sum_j binom(p, j) Z^j b until a
 * term's norm is below series_tol ||b|| (at most 40 terms).  Each Z costs two
 * rational applications and one FP64 A.  p = -1/4 gives the heatbath field
 * phi = (1 + Z)^-1/4 eta, p = 1/2 the acceptance factor ((1 + Z)^1/2 phi, whose
 * inner product with phi is the correction's energy).  *napply = number of Z
 * applications; infos: the records of the last multishift solve. */
tm_status tm_rational_correction(tm_ctx* ctx, tm_op op, int n, double a0, const double* a,
                                 const double* sigma, double p, double series_tol, double* y,
                                 const double* b, const tm_solve_params* sp, tm_solve_info* infos,
                                 int* napply, void* stream);

/* n independent solves A_i x_i = b_i on contexts of possibly different volumes, all
 * advanced together by batched kernels (one launch per step covers every
 * problem).  n <= 32.  The stencil variants are those chosen (tm_autotune /
 * tm_set_tuning) for the context with the most sites. */
tm_status tm_solve_batch(tm_ctx** ctxs, int n, tm_op op, const tm_solve_params* sp,
                         double** x, const double** b, tm_solve_info* infos, void* stream);

/* Largest eigenvalue of the HPD op (TM_MDAGM, TM_QPQM, TM_QH_SQ) by `iters` power
 * iterations from a fixed seeded start vector, FP64. */
tm_status tm_power_iteration(tm_ctx* ctx, tm_op op, int iters, double* lambda_max, void* stream);

/* Average device time per launch of the two passes of one Schur operator in
 * storage precision prec (op = TM_QHAT_PLUS / TM_QHAT_MINUS / TM_QH / TM_QH_DAG):
 * ms[0] = even pass (hop + inverse blocks, eq:hQpm's (M_ee)^-1 M_eo),
 * ms[1] = odd pass (hop + clover + twist + g5).  Each pass is launched `reps`
 * times back to back between CUDA events recorded on `stream`; `in` is a native
 * field of precision prec, outputs go to library-owned scratch. */
tm_status tm_kernel_times(tm_ctx* ctx, tm_op op, tm_prec prec, const void* in, int reps, double* ms,
                          void* stream);

/* Fermion-force outer products of the hopping term on every link (the force of
 * the rational-approximation monomials, whose outer products of several
 * two-flavour spinors Sec. 4.3 "Efficiency" reports as left on the CPU):
 *
 *   force_mu(x) += T_A[ U_mu(x) W_mu(x) ],
 *   W_mu(x) = ph_mu(x) sum_k coeff[k] sum_flavour
 *               [ X_k(x+mu) (x) ((1 - g_mu) Y_k(x))^*  +  ((1 + g_mu) Y_k(x+mu)) (x) X_k(x)^* ],
 *
 * with (a (x) b^*)_ij = a_i conj(b_j) over colour (spin summed), ph_mu(x) = bc_t
 * of the last tm_clover_compute on the time links crossing t = T-1 -> 0 (1
 * elsewhere), and T_A[Z] = (Z - Z^+)/2 - tr(Z - Z^+)/6 the traceless
 * anti-hermitian part.  force_mu(x) is then the derivative of
 * S = sum_k coeff[k] Re <Y_k, H X_k> along U_mu(x) -> exp(t w) U_mu(x), w in su(3):
 * dS/dt = Re tr(w force_mu(x)).  The clover term's own link dependence is not
 * included.
 *   prec      storage precision of the fields: TM_F32, TM_BF16 or TM_F16 (the
 *             products are formed in FP32; TM_F64 fields are rejected)
 *   nflavour  1 or 2
 *   n         field pairs, 0 <= n <= TM_FORCE_MAXN (n = 0: nothing to do)
 *   coeff     host array of n weights
 *   x, y      host arrays of 2n device pointers: x[2k + p] is the native field
 *             X_k (tm_field_bytes of prec, nflavour) on the sites of parity p
 *             (p = 0 even, 1 odd; tm_field_import converts either parity's
 *             canonical half-lattice array, site k having lex/2 == k), 16-byte aligned
 *   gamma5_y  non-zero: every Y_k enters as g5 Y_k
 *   force     device, canonical FP64 gauge layout [t][z][y][x][mu][3][3] (re, im),
 *             16-byte aligned; accumulated into
 * Needs a loaded gauge field and a current clover term (TM_ERR_STALE otherwise).
 * Stream-ordered, one launch.
 *
 * Schur operators.  For odd fields a, b, the derivative of Re <a, Q_hat_s b>
 * through the two hops of Q_hat_s = g5 [M_oo - kappa^2 H_oe M_ee(s)^-1 H_eo]
 * (clover term held fixed) is the force of the single pair
 *   X = (R_s b on even sites, b on odd sites),  Y = (R_-s a, a),  gamma5_y = 1,
 * with weight -kappa^2, where R_s = M_ee(s)^-1 H_eo comes from tm_apply_even
 * (s = + for TM_QHAT_PLUS / TM_QH, - for TM_QHAT_MINUS / TM_QH_DAG).  For a
 * rational force, pass one such pair per shift, weighted by -kappa^2 times the
 * shift's coefficient. */
#define TM_FORCE_MAXN 32
tm_status tm_force_outer(tm_ctx* ctx, tm_prec prec, int nflavour, int n, const double* coeff,
                         const void* const* x, const void* const* y, int gamma5_y, double* force,
                         void* stream);

/* ---------------------------------------------------------------------------
 * Learned preconditioner: gauge-equivariant parallel-transport network (PTC).
 * Not in the paper, which preconditions its hardest solves by multigrid
 * (Sec. 4.1); the network stands in for it inside flexible CG.  Layer l maps
 * channels[l] -> channels[l+1] spinor fields on the full lattice:
 *   out^a(x) = sum_{p} sum_b W_p^{ab} (T_p in^b)(x),  p in {1, +x,+y,+z,+t, -x,-y,-z,-t},
 *   (T_{+mu} f)(x) = U_mu(x) f(x+mu),  (T_{-mu} f)(x) = U_mu(x-mu)^+ f(x-mu),
 * W_p^{ab} a complex 4x4 spin matrix; no activation (the preconditioner is a
 * linear map).  The input is the odd-site residual embedded with zeros on even
 * sites; the output is the odd sites of the last layer.  Channel mixing runs on
 * the tensor cores in BF16 with FP32 accumulation; activations are BF16.
 * Canonical weights: complex FP64 [layer][path 9][c_out][c_in][4][4], host memory.
 * ------------------------------------------------------------------------- */
typedef struct tm_ptc tm_ptc;

/* channels has nlayers+1 entries, first and last 1, each 1, 2, 4 or 8 (the
 * layer shapes 1->c, c->c, c->1).  Weights start at zero. */
tm_status tm_ptc_create(tm_ptc** net, int nlayers, const int* channels, int device);
tm_status tm_ptc_destroy(tm_ptc* net);
tm_status tm_ptc_num_weights(const tm_ptc* net, size_t* complex_count);
tm_status tm_ptc_set_weights(tm_ptc* net, const double* weights);
/* Start near the identity: path 1 carries scale * 1 between equal channel
 * indices, every other weight is uniform noise in [-noise, noise] (re, im) from
 * a seeded splitmix64 stream; resets the Adam state. */
tm_status tm_ptc_init(tm_ptc* net, double scale, double noise, unsigned long long seed);
tm_status tm_ptc_get_weights(const tm_ptc* net, double* weights);
/* out = N(in): native FP32 light odd fields of ctx's lattice (device), stream-ordered. */
tm_status tm_ptc_apply(tm_ptc* net, tm_ctx* ctx, void* out, const void* in, void* stream);
/* Check of the bounded waits used by the PTC kernels (the paper has no
 * counterpart): one GPU thread waits on an mbarrier that nothing arrives on,
 * bounded by `seconds` (0 < seconds <= 10).  *timed_out = 1 when the bound ran
 * out as designed (0: the phase completed, 2: the wait ended otherwise); the
 * context stays usable.  Synchronous. */
tm_status tm_wait_selftest(int device, double seconds, int* timed_out);
/* Wait for the network's work queued on stream and report a layer kernel whose
 * bounded wait on the tensor cores ran out (TM_ERR_TIMEOUT; its output is then
 * incomplete).  tm_ptc_grad, tm_ptc_train and tm_solve_fcg check the same flag
 * before they return. */
tm_status tm_ptc_sync(tm_ptc* net, void* stream);
/* Loss L = ||N(r) - e||^2 / ||e||^2 of one pair (canonical FP64 r, e; host or
 * device) and its Wirtinger gradient dL/dconj(W) (host, canonical weight layout). */
tm_status tm_ptc_grad(tm_ptc* net, tm_ctx* ctx, const double* r, const double* e, double* loss,
                      double* grad, void* stream);
/* Train on npairs solver-generated pairs: e ~ complex Gaussian (Philox4x32-10
 * keyed by seed, one stream per pair), r = A e with the FP32 operator op
 * (TM_MDAGM or TM_QPQM) of ctxs[k % nctx] (same volume), Adam (lr, 0.9, 0.999)
 * on the mean gradient of every `batch` pairs.  losses: host array of npairs or NULL. */
tm_status tm_ptc_train(tm_ptc* net, tm_ctx** ctxs, int nctx, tm_op op, int npairs, int batch, double lr,
                       unsigned long long seed, double* losses, void* stream);
/* Checkpoint: weights and Adam state to / from a binary file. */
tm_status tm_ptc_save(const tm_ptc* net, const char* path);
tm_status tm_ptc_load(tm_ptc* net, const char* path);

/* Flexible CG (truncation 1) on A = TM_MDAGM or TM_QPQM, preconditioned by net;
 * FP32 vectors and operator, BF16 network; reliable updates (sp->delta) in
 * double-word arithmetic (tm_apply_Mhat_dw) restart the recursion; stops at
 * FP64 true relative residual sp->tol (a residual below it is confirmed with the
 * FP64 operator).
 * x, b canonical FP64 (host or device); sp->sloppy is ignored. */
tm_status tm_solve_fcg(tm_ctx* ctx, tm_op op, tm_ptc* net, const tm_solve_params* sp, double* x,
                       const double* b, tm_solve_info* info, void* stream);

/* ---------------------------------------------------------------------------
 * Two-level multigrid on the full operator (Sec. 4.1: the light sector's most
 * poorly conditioned solves run an outer GCR preconditioned by multigrid, about a
 * hundred times faster than mixed-precision CG at the physical mass; the paper
 * gives no detail of the method).  The library builds the textbook
 * aggregation-based Galerkin form for Wilson-type operators:
 *   aggregates   the lattice cut into blocks of block[0..3] sites, each block split
 *                by chirality (spins 0,1 / spins 2,3): aggregate a = 2 k + h, k the
 *                block's lexicographic index on the block lattice
 *                ((kt*nz + kz)*ny + ky)*nx + kx;
 *   near-null    nvec fields given by the caller (random fields), each smoothed by
 *                setup_steps minimal-residual steps on M v = 0 and normalised;
 *   prolongator  per aggregate, the Gram-Schmidt orthonormalisation (R with a
 *                positive real diagonal) of the vectors' restrictions; P^+ P = 1;
 *   coarse op.   M_c = P^+ M P, nearest neighbour on the block lattice;
 *   precond.     z = P M_c^-1 P^+ r, the coarse system solved by restarted GCR to
 *                relative residual coarse_tol (the exact coarse solve is the limit
 *                coarse_tol -> 0), then smooth_steps minimal-residual steps on
 *                M z = r starting from that z.
 * Canonical full field: FP64 [t][z][y][x][spin 4][colour 3] (re, im), every
 * lattice site, device memory, 16-byte aligned.  Coarse vector: complex FP64
 * [a][j], a = 2 k + h, j < nvec (tm_mg_coarse_size complex entries).
 * The multigrid keeps the gauge generation and clover stamp of its setup; calls
 * after tm_gauge_load or a new tm_clover_compute return TM_ERR_STALE until the
 * next tm_mg_setup.
 * ------------------------------------------------------------------------- */
typedef struct tm_mg tm_mg;

typedef struct {
    int block[4];        /* aggregate block extents (X, Y, Z, T), each dividing the lattice extent */
    int nvec;            /* near-null vectors: 1 .. 16 and at most 6 x block volume */
    int setup_steps;     /* minimal-residual steps per near-null vector */
    int smooth_steps;    /* minimal-residual post-smoothing steps of the preconditioner */
    int sign;            /* +1: M(+mu), -1: M(-mu) */
    tm_prec prec;        /* TM_F64 or TM_F32: storage and arithmetic of the setup, the
                            prolongator, the coarse operator and the preconditioner;
                            reductions are FP64 either way */
    double coarse_tol;   /* relative residual of the coarse GCR solve (> 0) */
    int coarse_maxiter;  /* bound on coarse GCR iterations per preconditioner application */
    int coarse_restart;  /* coarse GCR restart length, 1 .. 16 */
} tm_mg_params;

/* out = M(sign) in, the full (unpreconditioned) operator of the conventions above
 * on canonical full fields (device), in storage and arithmetic prec (TM_F64 or
 * TM_F32).  Stream-ordered.  TM_ERR_STALE without a current clover term. */
tm_status tm_apply_full(tm_ctx* ctx, int sign, tm_prec prec, double* out, const double* in, void* stream);
/* Allocates the hierarchy's device memory for ctx's lattice (prolongator
 * 12 V nvec complex, coarse operator 36 nvec^2 complex per block, the near-null
 * fields and the coarse solver's vectors).  The context must outlive it. */
tm_status tm_mg_create(tm_mg** mg, tm_ctx* ctx, const tm_mg_params* params);
tm_status tm_mg_destroy(tm_mg* mg);
tm_status tm_mg_coarse_size(const tm_mg* mg, size_t* n_complex);
/* Setup from nvec canonical full fields stored back to back at init (device):
 * smoothing, prolongator, coarse operator.  Synchronous. */
tm_status tm_mg_setup(tm_mg* mg, const double* init, void* stream);
/* The smoothed, normalised near-null vectors: nvec canonical full fields back to back (device). */
tm_status tm_mg_vectors(tm_mg* mg, double* out, void* stream);
/* fine = P coarse;  coarse = P^+ fine;  out = M_c in.  Device vectors, stream-ordered. */
tm_status tm_mg_prolong(tm_mg* mg, double* fine, const double* coarse, void* stream);
tm_status tm_mg_restrict(tm_mg* mg, double* coarse, const double* fine, void* stream);
tm_status tm_mg_coarse_apply(tm_mg* mg, double* out, const double* in, void* stream);
/* z = the preconditioner applied to r (canonical full fields, device); the coarse
 * GCR iterations it took go to *coarse_iters (may be NULL).  Synchronous. */
tm_status tm_mg_precondition(tm_mg* mg, double* z, const double* r, int* coarse_iters, void* stream);
/* Solve M(sign) x = b (canonical full fields, device; x in: initial guess, out:
 * solution) to FP64 true relative residual sp->tol.  The outer loop recomputes
 * r = b - M x with the FP64 operator; until converged, a restarted flexible GCR
 * (restart sp->chunk, 0 = 8, at most 16) in the multigrid's precision, or in
 * sp->sloppy (TM_F64 / TM_F32) without one, preconditioned by mg (NULL: none),
 * solves M e = r / ||r|| to relative residual sp->delta (<= 0: 1e-5; FP64 inner
 * solves aim at the outer target directly) and x += ||r|| e.  info->iters counts
 * GCR iterations, info->reliable_updates the outer corrections.  mg must belong to
 * ctx and the same sign.  Synchronous. */
tm_status tm_solve_gcr(tm_ctx* ctx, int sign, tm_mg* mg, const tm_solve_params* sp, double* x,
                       const double* b, tm_solve_info* info, void* stream);

/* Stencil kernel variant of each pass of the Schur operator for one storage
 * precision and flavour count: 0 = direct (operands loaded into registers),
 * 1 = shared-memory staged (asynchronous copies of the neighbour spinors, links
 * and site-local blocks, two directions ahead; FP32 and 16-bit only). */
typedef struct {
    int even_pass;   /* hop + inverse blocks   */
    int odd_pass;    /* hop + clover + g5      */
} tm_tuning;

/* Autotuner: time both variants of both passes on this context's lattice and
 * keep the faster of each (used by every later operator, solver and batch
 * call).  If the environment variable TM_TUNE_CACHE names a file, choices are
 * read from / appended to it, keyed by "X Y Z T prec nflavour".  FP64 always
 * uses the direct kernel.  `chosen` may be NULL. */
tm_status tm_autotune(tm_ctx* ctx, tm_prec prec, int nflavour, tm_tuning* chosen, void* stream);
tm_status tm_set_tuning(tm_ctx* ctx, tm_prec prec, int nflavour, const tm_tuning* tuning);
tm_status tm_get_tuning(const tm_ctx* ctx, tm_prec prec, int nflavour, tm_tuning* tuning);

/* Measured fused multiply-add rate of the CUDA cores in FP64 or FP32 (flops per
 * second, 2 per FMA): register-resident chains on every SM, CUDA-event timed.
 * The roofline denominator of passes bound by arithmetic instead of memory; the
 * paper has no counterpart.  Synchronous; allocates a few bytes. */
tm_status tm_fma_rate(int device, tm_prec prec, double* flops_per_s);

/* Message of the calling thread's last failure ("" if none). */
const char* tm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* TM_H */
