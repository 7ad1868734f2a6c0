/*
 * rsign.h -- C ABI of the GB300 shifted matrix-sign reflector library.
 *
 * Problem (Sec. 2.1, Prop. 2.1): H is a real symmetric d x d matrix with
 * ordered eigenvalues lam_1 <= ... <= lam_d and eigenvectors q_i; for a target
 * index k in {1, ..., d-1} the prescribed-index reflector is
 *     R_k = I - 2 P_k,   P_k = sum_{i<=k} q_i q_i^T          (Eq. Pk, Eq. Rk_intro)
 * and for every shift s in (lam_k, lam_{k+1})
 *     R_k = sign(H - s I).                                   (Prop. 2.1)
 * The library computes sign(H - sI) with the scaled Newton-Schulz iteration
 *     X_0 = alpha (H - s I),  X_{m+1} = 1/2 X_m (3 I - X_m^2)  (Eq. NS)
 * with alpha <= 1/rho(H - sI) (Cor. 3.5), and certifies the result through
 * trace(R) = d - 2k (the sign pattern of Prop. 2.1 / Lemma 3.4).
 *
 * Conventions for every call:
 *   - matrices are dense, row-major, leading dimension d, IEEE binary64;
 *   - a matrix pointer may address device memory or host memory (pageable
 *     or pinned); host buffers are copied in and out on `stream` inside the
 *     call.  The caller owns every buffer; the library never frees them;
 *   - only the symmetric part 1/2 (H + H^T) of H is used; H is read-only;
 *   - workspace is allocated inside the call (stream-ordered, from a
 *     library-owned pool) and released before it returns; the pool keeps the
 *     memory mapped for later calls until rsign_trim_workspace();
 *   - state that outlives a call, shared by every host thread of the
 *     process: that pool (one per device, created under a lock); the tile
 *     width the batched call's autotuner chose per batch shape (a map under
 *     a lock: the first call of a shape times both widths, later calls reuse
 *     the choice); one-time kernel attributes and the tensor-map encoder
 *     entry point; the static array of rsign_reflector_noalloc; and the
 *     process-wide settings of the rsign_dbg_* entry points (not
 *     thread-safe, for tests).  Nothing else is kept between calls, and
 *     calls on different streams share no buffers except the pool's
 *     allocator (rsign_reflector_noalloc excepted, see there);
 *   - calls are blocking: they return once `info` (if given) is filled, since
 *     the certificate is part of the result;
 *   - errors are reported through the return value only: the library never
 *     prints, never aborts, and leaves no sticky CUDA error behind for
 *     argument errors; RSIGN_ERR_CUDA reports a failed CUDA call;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 */
#ifndef RSIGN_H
#define RSIGN_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RSIGN_OK = 0,
  RSIGN_ERR_ARG = 1,         /* invalid argument: d < 2, k outside [1, d-1], NULL, tol <= 0,
                                non-finite entry in H, bad policy or option              */
  RSIGN_ERR_NOCONV = 2,      /* step budget exhausted before the tolerance was met        */
  RSIGN_ERR_CERT = 3,        /* trace certificate failed: |trace R - (d - 2k)| >= 1/2,
                                i.e. the shift is not in (lam_k, lam_{k+1}) or alpha*rho
                                exceeded sqrt(3); R holds the iterate for diagnosis      */
  RSIGN_ERR_GAP = 4,         /* automatic shift: target gap not resolved                  */
  RSIGN_ERR_CUDA = 5,        /* a CUDA runtime call failed                                */
  RSIGN_ERR_TIMEOUT = 6,     /* a bounded device-side wait gave up                        */
  RSIGN_ERR_UNSUPPORTED = 7  /* device is not sm_103 or the size exceeds a limit
                                (d > 16384; d > 512 for rsign_reflector_noalloc)          */
} rsign_status;

/* Precision policy of the Newton-Schulz steps. */
typedef enum {
  RSIGN_FP64 = 0,         /* every step in FP64 (native FP64 pipe)                       */
  RSIGN_FP16 = 1,         /* FP16 operands, FP32 tensor accumulation, no FP64 stage:
                             accuracy floor ~ u_fp16 ||H|| / gap                         */
  RSIGN_BF16 = 2,         /* BF16 operands, FP32 tensor accumulation, no FP64 stage      */
  RSIGN_FP16_POLISH = 3,  /* FP16 steps followed by `polish_steps` FP64 NS steps          */
  RSIGN_BF16_POLISH = 4,  /* BF16 steps followed by `polish_steps` FP64 NS steps          */
  RSIGN_FP16_REFINE = 5,  /* FP16 steps, then commutator refinement sweeps with
                             FP64-grade products until the error estimate (with
                             refine_stop = RSIGN_STOP_BOUND: the bound) is <= tol       */
  RSIGN_BF16_REFINE = 6,  /* BF16 steps, then the same refinement                        */
  RSIGN_FP32 = 7          /* FP32-class steps: iterates carried as FP16 hi/lo pairs (22-bit
                             significands, the fused pair products hi*hi + hi*lo + lo*hi
                             with FP32 accumulation), no FP64 stage: accuracy floor
                             ~ u_fp32 ||H|| / gap                                        */
} rsign_policy;

/* Scaling rule for alpha (Sec. 4.3 scaling discussion). */
typedef enum {
  RSIGN_ALPHA_INF = 0,    /* alpha = 1/||H - sI||_inf (Gershgorin bound on rho)          */
  RSIGN_ALPHA_POWER = 1   /* alpha = 1/(1.02 rho_est), rho_est from power steps on H - sI
                             (closer to 1/rho than the Gershgorin bound, so a larger scaled
                             margin and fewer steps); sign preservation needs alpha rho <
                             sqrt(3), i.e. rho_est > 0.57 rho: if the trace certificate
                             fails, rsign_reflector_ex repeats the call with RSIGN_ALPHA_INF */
} rsign_alpha_mode;

/* Per-call report, filled on the host when `info` is not NULL. */
typedef struct {
  int32_t steps_low;       /* Newton-Schulz steps in FP16/BF16                         */
  int32_t steps_fp64;      /* Newton-Schulz steps in FP64 or FP64-grade arithmetic     */
  int32_t sweeps_refine;   /* commutator refinement sweeps                             */
  int32_t cert_ok;         /* 1 iff |trace - (d-2k)| < 1/2 and resid_fro <= tol_fro    */
  double alpha;            /* scaling used, X_0 = alpha (H - sI)                       */
  double shift;            /* shift s used                                             */
  double gamma_est;        /* alpha * estimated margin min |lam_i - s| (auto shift) or
                              NaN when the margin is not known                         */
  double resid_fro;        /* ||R^2 - I||_F of the returned R; REFINE policies: of the
                              iterate before the final update-form polish step (the
                              returned R is one quadratically convergent step further) */
  double trace;            /* trace(R)                                                 */
  double correction_fro;   /* ||last refinement correction||_F (REFINE policies)       */
  double commutator_norm;  /* estimate of ||R A - A R||_2, A = H - sI, at the last
                              a-posteriori check (REFINE): 8 power steps on the
                              antisymmetric C, v -> R A v - A R v, with FP64-class
                              (double-float, ~2^-46 per term) products; NaN otherwise  */
  double err_est;          /* a-posteriori estimate of ||R - sign(H - sI)||_2 (REFINE):
                              2.5 max(1.5 kappa alpha ||G||_2, ||C||_2 / g) (the factor
                              2.5 covers the largest underestimate measured, 2.1x;
                              it is an estimate, not a bound): G = 1/2 R C,
                              C = R A - A R, kappa the gain of the last tangent solve,
                              g the eigenvalue gap of the 2 x 2 Rayleigh-Ritz projection
                              of A on the dominant plane of C (at least 2 mu when a
                              margin mu is known); NaN for other policies              */
  double tol_fro;          /* the residual threshold applied: max(tol, 16 d u_64)      */
  double ms_total;         /* device time of the call, ms (CUDA events on `stream`)    */
  double ms_low;           /* device time of the low-precision stage, ms               */
  double ms_fp64;          /* device time of the FP64 / FP64-grade stages, ms          */
  double flops_low;        /* algorithmic flops of the low-precision stage (2 d^3 per
                              NS step: SYRK X^2 plus the symmetric product)           */
  int64_t launches;        /* kernel launches this call issued, counting the ones
                              enqueued after the device-side stop (they return at once) */
  int64_t workspace_bytes; /* device workspace the call allocated                      */
  /* automatic shift (s = NaN), Sec. 4.3 / Prop. 4.1-4.2; NaN / 0 otherwise:          */
  double lam_k_est;        /* Lanczos estimate of lam_k                                */
  double lam_k1_est;       /* Lanczos estimate of lam_{k+1}                            */
  double shift_eps;        /* endpoint error bound eps (largest Ritz residual bound plus a
                              rounding allowance 16 sqrt(d) u ||T||, u = 2^-46 the unit
                              of the double-float products A v)                         */
  double margin_lb;        /* guaranteed margin m_hat - eps of the chosen shift        */
  int32_t lanczos_iters;   /* Lanczos steps taken                                      */
  int32_t steps_pred;      /* NS steps the scalar recurrence predicts for eps_m(gamma) <= tol,
                              gamma = alpha * margin_lb (Prop. 3.6); -1 when unknown     */
  /* batched calls (rsign_reflector_batched[_ex]); 0 for single calls:                */
  int32_t batch_grouped;   /* 1: the matrix went through the grouped launches          */
  int32_t batch_tile;      /* tile width of the grouped tensor-core launches (128 or
                              256; 64 = FP64 tiles only); the ms_* fields of a grouped
                              matrix are those of the whole batch                      */
  int32_t ns_scaled_steps; /* leading steps run with the scaled step (rsign_options
                              ns_scaling); 0 = the plain iteration throughout           */
  int32_t refine_levels;   /* REFINE: 5-bit digit levels of the first sweep's FP64-grade
                              R A product (5..7, from the truncation model: the error it
                              leaves after the sweep ~ 2^(-5L) s_A s_R sqrt(d) / mu <=
                              tol/2, s the largest row scales of the digit splits, mu the
                              margin or a lower bound from the stage-1 step count)     */
  double err_bound;        /* REFINE with a known margin mu (rsign_options.margin or the
                              certified margin of the automatic shift): bound of
                              ||R - sign(H - sI)||_2 from the last check, 1 - sqrt(1 - 2c),
                              c = ||R A - A R||_2 / (2 mu) + ||R^2 - I||_2 / 2 (inf if
                              2c >= 1); with rsign_options.refine_stop = RSIGN_STOP_BOUND
                              the refinement stops on err_bound <= tol instead of err_est
                              <= tol.  Both 2-norms are power-step estimates
                              (commutator_norm and the check's power steps on R^2 - I,
                              which converge from below).  NaN otherwise                */
} rsign_info;

/* Optional knobs; rsign_options_default() fills the defaults. */
typedef struct {
  int32_t max_steps;        /* NS step budget per stage (default 100)                   */
  int32_t polish_steps;     /* FP64 polish steps for *_POLISH policies (default 2)      */
  int32_t max_sweeps;       /* refinement sweep budget (default 4)                      */
  int32_t alpha_mode;       /* rsign_alpha_mode (default RSIGN_ALPHA_INF)               */
  int32_t power_steps;      /* power steps for RSIGN_ALPHA_POWER (default 20)           */
  int32_t timing;           /* 1: fill ms_* fields with CUDA events (default 1)        */
  int32_t low_split;        /* REFINE policies: 1 carries the low-precision iterates as
                               hi/lo pairs (three fused pair products per step, about
                               twice the mantissa bits, one refinement sweep usually
                               suffices); 0 plain operands (default 1)                */
  int32_t lanczos_max;      /* automatic shift: Lanczos step budget (default 600)      */
  int32_t batch_graphs;     /* batched calls: 1 replays each chunk of grouped NS steps
                               as one CUDA graph (default 1); 0 launches eagerly       */
  int32_t batch_tile;       /* batched calls: tile width of the grouped tensor-core
                               launches, 128 or 256; 0 lets the autotuner time both
                               widths (and two tile orders) on the batch's first step
                               and cache the choice per batch shape (default 0)        */
  int32_t ns_scaling;       /* 1: scaled Newton-Schulz steps X <- 1/2 a X (3I - a^2 X^2)
                               (the stable step scalings cited in Sec. 3.5) while a
                               margin bound is known: a = sqrt(3/(1 + l + l^2)) for the
                               spectral interval [l, 1], l <- 1/2 a l (3 - a^2 l^2), then
                               plain steps; l_0 = alpha * margin.  Same limit, about
                               half the steps for small l.  0: the plain iteration
                               (default 0)                                              */
  double margin;            /* lower bound of min_i |lam_i - s| for ns_scaling (the
                               half-gap for a midpoint shift), NaN = unknown (default);
                               the automatic shift supplies its certified margin       */
  int32_t refine_stop;      /* REFINE stop test: RSIGN_STOP_ESTIMATE (default) stops on
                               err_est <= tol; RSIGN_STOP_BOUND stops on err_bound <= tol
                               and needs a margin (rsign_options.margin or the automatic
                               shift), else RSIGN_ERR_ARG.  The bound divides the
                               commutator by the whole gap 2 mu, so broadband rounding
                               noise in R (large eigenvalue differences) inflates it:
                               it can stay above tol at errors far below tol           */
  int32_t engine;           /* rsign_engine (default RSIGN_ENGINE_NS3)                   */
} rsign_options;

/* Polynomial sign engines (rsign_options.engine), Sec. 3.4 / Sec. 5.4 on higher-degree odd
 * filters.  Both are fixed points of sign with X_0 = alpha (H - sI), alpha <= 1/rho. */
typedef enum {
  RSIGN_ENGINE_NS3 = 0,   /* Eq. NS: X <- 1/2 X (3I - X^2), two products per step (and the
                             scaled variant of rsign_options.ns_scaling)                   */
  RSIGN_ENGINE_NS5 = 1    /* the quintic X <- 1/8 X (15I - 10X^2 + 3X^4), in update form
                             X + 1/2 X W with E = I - X^2, W = E + 3/4 E^2: three products
                             per step, cubic convergence near +-1, growth 15/8 near 0.
                             FP64, FP16, BF16, FP32 and *_POLISH policies (the polish steps
                             stay Eq. NS; no scaled variant); REFINE policies and batched
                             calls: RSIGN_ERR_ARG; rsign_reflector_backward differentiates
                             the NS3 map                                                    */
} rsign_engine;

/* Stop tests of the refinement sweeps (rsign_options.refine_stop). */
typedef enum {
  RSIGN_STOP_ESTIMATE = 0,
  RSIGN_STOP_BOUND = 1
} rsign_refine_stop;

void rsign_options_default(rsign_options* opt);

/*
 * rsign_reflector -- R = sign(H - sI) = I - 2 P_k  (Prop. 2.1, Eq. NS).
 *   H      d x d, symmetric part used; device or host memory.
 *   d      matrix order, 2 <= d <= 16384.
 *   k      target index, 1 <= k <= d-1 (Sec. 2.1); used by the trace certificate.
 *   s      shift, expected in (lam_k, lam_{k+1}); the midpoint (Prop. 4.1) is the
 *          recommended choice.  NaN requests an automatic midpoint shift from
 *          Lanczos estimates of lam_k, lam_{k+1} (Sec. 4.3, Prop. 4.2).
 *   tol    target: FP64 policy stops when ||X^2 - I||_F < max(tol, 16 d u_64);
 *          REFINE policies stop when the a-posteriori error estimate err_est
 *          (or, with refine_stop = RSIGN_STOP_BOUND, the bound err_bound) of
 *          ||R - sign(H - sI)||_2 is at most tol.
 *   policy rsign_policy.
 *   R      d x d output (device or host), fully written on RSIGN_OK and
 *          RSIGN_ERR_CERT / RSIGN_ERR_NOCONV (last iterate).
 *   info   optional report.
 * Returns RSIGN_OK when the trace certificate holds and the tolerance was met.
 */
rsign_status rsign_reflector(const double* H, int64_t d, int32_t k, double s, double tol,
                             rsign_policy policy, double* R, rsign_info* info, void* stream);

/* Same as rsign_reflector with explicit options (NULL = defaults). */
rsign_status rsign_reflector_ex(const double* H, int64_t d, int32_t k, double s, double tol,
                                rsign_policy policy, const rsign_options* opt, double* R,
                                rsign_info* info, void* stream);

/*
 * rsign_apply -- out = R V, the reflected directions d = -R g of Eq. discrete_step
 * are -rsign_apply(R, g).  Prop. 3.3 bounds ||R~ g - R g|| by ||R~ - R||_2 ||g||.
 *   R   d x d (row-major), V d x nv (row-major, ld nv), out d x nv (row-major).
 *   FP64 arithmetic.  Device or host pointers.
 */
rsign_status rsign_apply(const double* R, int64_t d, const double* V, int64_t nv, double* out,
                         void* stream);

/*
 * rsign_reflector_batched -- n independent reflectors R_i = sign(H_i - s_i I)
 * (the batched regime of Sec. 4.5).  Arrays H, d, k, s, R, infos have n
 * entries; H[i] and R[i] are d[i] x d[i] (device or host memory, each on its
 * own).  Returns the first non-OK status in index order (all are attempted);
 * infos[i] holds each matrix's own status-relevant report.  n = 0 returns
 * RSIGN_OK at once (no device work; the pointers may be NULL); n < 0 is
 * RSIGN_ERR_ARG.
 *   Grouped path: every matrix with d[i] <= 1024, a finite s[i] and a
 *   policy among FP64, FP16, BF16, FP16_POLISH, BF16_POLISH is placed in a
 *   Dmax x Dmax slot of one slab and the whole group advances together: each
 *   Newton-Schulz step is one grouped tensor-core (or FP64) launch for the
 *   squares of all unconverged matrices, one stop-test launch and one
 *   grouped launch for the updates; a matrix whose residual stops
 *   decreasing (its own stop test, the same as rsign_reflector's) retires
 *   and its tiles are skipped from then on.  Chunks of eight steps are
 *   replayed as one CUDA graph.  alpha_i is the Gershgorin bound of each
 *   matrix (Sec. 4.3).  Each matrix gets the same result as its own
 *   rsign_reflector call with the same policy and RSIGN_ALPHA_INF.
 *   Other matrices (s[i] = NaN for the automatic shift, REFINE policies and
 *   FP32, d[i] > 1024) are computed with rsign_reflector_ex calls that up
 *   to 16 library-owned host threads run concurrently, each on a stream of
 *   its own that first waits for `stream`; each result equals that
 *   matrix's lone rsign_reflector_ex call bit for bit.  The call returns
 *   once every matrix is done.
 */
rsign_status rsign_reflector_batched(int32_t n, const double* const* H, const int64_t* d,
                                     const int32_t* k, const double* s, double tol,
                                     rsign_policy policy, double* const* R, rsign_info* infos,
                                     void* stream);

/* Same as rsign_reflector_batched with explicit options (NULL = defaults);
 * alpha_mode is ignored by the grouped path (Gershgorin alpha). */
rsign_status rsign_reflector_batched_ex(int32_t n, const double* const* H, const int64_t* d,
                                        const int32_t* k, const double* s, double tol,
                                        rsign_policy policy, const rsign_options* opt,
                                        double* const* R, rsign_info* infos, void* stream);

/*
 * rsign_reflector_backward -- adjoint of R = p_m(alpha (H - sI)) (Eq. NS
 * unrolled) with s and alpha held fixed: given Rbar = dL/dR (d x d),
 * returns Hbar = dL/dH (symmetrised, d x d).  The recurrence is run backward
 * over checkpoints of the forward iterates taken every `ckpt_every` steps.
 * The policy selects the arithmetic of the forward and backward steps:
 * FP64 (checkpointed FP64 recomputation); FP16/BF16 and *_REFINE (the
 * stage-1 trajectory kept whole, tangent products in the operand type);
 * *_POLISH (the same, preceded by the FP64 adjoint of the two FP64 polish
 * steps of the default forward).  Device or host pointers; blocking.
 */
rsign_status rsign_reflector_backward(const double* H, int64_t d, int32_t k, double s,
                                      rsign_policy policy, const double* Rbar, double* Hbar,
                                      int32_t ckpt_every, void* stream);

/* ---------------------------------------------------------------------------
 * Shift policies along a sequence of slowly varying matrices H_0, H_1, ...
 * (Sec. 4.4: Prop. 4.2 and the shift policies of Algorithm 1).
 * ------------------------------------------------------------------------- */
typedef enum {
  RSIGN_SHIFT_MIDPOINT = 0,       /* refresh at every matrix: s = midpoint of the estimates    */
  RSIGN_SHIFT_REUSE_REFRESH = 1,  /* keep s while its certified margin minus the drift bound
                                     stays above `threshold`; otherwise refresh (Prop. 4.2)   */
  RSIGN_SHIFT_DAMPED = 2          /* refresh at every matrix: blend of the previous shift and
                                     the new midpoint, clipped into the certified interval    */
} rsign_shift_policy;

/* State carried from one matrix of the sequence to the next (host memory). */
typedef struct {
  double shift;        /* shift in use; NaN before the first refresh                       */
  double lam_k_est;    /* Lanczos estimates of lam_k, lam_{k+1} at the last refresh         */
  double lam_k1_est;
  double eps;          /* their error bound (largest Ritz residual)                        */
  double margin_cert;  /* certified margin of `shift` at the current matrix: the estimated
                          margin minus eps at the refresh, minus every drift bound since    */
  double drift_sum;    /* sum of the drift bounds since the last refresh                    */
  int32_t refreshes;   /* endpoint estimations so far                                       */
  int32_t reuses;      /* matrices that kept the previous shift                              */
} rsign_shift_state;

/* Report of one rsign_shift_update call. */
typedef struct {
  int32_t refreshed;     /* 1: new endpoint estimates were computed                          */
  int32_t lanczos_iters; /* Lanczos steps of the refresh (0 when reused)                     */
  double drift_ub;       /* the drift bound used (Weyl bound on the endpoint drift): the
                            caller's drift_bound, else min(||D||_F, (||D||_1 + ||D||_inf)/2)
                            for D = H_new - H_old; NaN without either                       */
  double drift_est;      /* power-step estimate of ||sym(D)||_2 (a lower bound) when H_old is
                            given, for comparison; NaN otherwise                             */
  double margin_cert;    /* certified margin of the returned shift at H_new                  */
} rsign_shift_report;

/* Sets shift, estimates and margin to NaN and the counters to zero. */
void rsign_shift_state_init(rsign_shift_state* state);

/* Host-only rule of Prop. 4.2: 1 when the state's shift stays admissible at a
 * matrix whose distance from the current one is at most drift_ub in the
 * 2-norm, with certified margin margin_cert - drift_ub > max(0, threshold). */
int32_t rsign_shift_can_reuse(const rsign_shift_state* state, double drift_ub, double threshold);

/* Host-only damped midpoint: damping * s_prev + (1 - damping) * midpoint,
 * clipped into (lam_k_est + eps, lam_k1_est - eps) shrunk by a quarter of its
 * half-width on each side; the midpoint when s_prev is NaN or the interval empty. */
double rsign_shift_damped(double s_prev, double lam_k_est, double lam_k1_est, double eps, double damping);

/*
 * rsign_shift_update -- the shift for H_new given the state left by H_old.
 *   H_new, H_old  d x d (device or host); H_old = NULL at the first matrix.
 *   drift_bound   a caller-certified bound on ||H_new - H_old||_2 (for
 *                 instance a Hessian Lipschitz constant times the step
 *                 length), or NaN: then the GPU computes the rigorous bound
 *                 min(||D||_F, (||D||_1 + ||D||_inf)/2) from H_old, which is
 *                 tight for low-rank changes and up to sqrt(d) loose for
 *                 spread-out ones.
 *   REUSE_REFRESH: if rsign_shift_can_reuse holds for the drift bound, keeps
 *   state->shift and lowers state->margin_cert by it; otherwise refreshes.
 *   MIDPOINT and DAMPED always refresh.  A refresh runs
 *   the GPU Lanczos of the automatic shift on H_new, sets the (damped)
 *   midpoint and certifies it by m_hat > eps (Prop. 4.2); when that fails the
 *   state's shift becomes NaN and RSIGN_ERR_GAP is returned.
 *   threshold >= 0; damping in [0, 1] (DAMPED only).  The state is updated in
 *   place; `report` is optional.  Blocking.
 */
rsign_status rsign_shift_update(const double* H_new, const double* H_old, int64_t d, int32_t k,
                                rsign_shift_policy policy, double threshold, double damping,
                                double drift_bound, rsign_shift_state* state, rsign_shift_report* report,
                                void* stream);

/*
 * rsign_reflector_noalloc -- the FP64-policy reflector (same result as
 * rsign_reflector with RSIGN_FP64) for callers that cannot allocate device
 * memory during their work: code whose device memory is planned once at
 * start-up, embedders with a fixed memory budget, or threads that must not
 * wait on the allocator.  The paper has no counterpart of this entry point;
 * it exists for deployment only.
 *   - No device memory is allocated or freed: the workspace is one static
 *     device array inside librsign (about 8.2 MiB), which every GPU that loads
 *     the library holds until the process exits.
 *   - Limit: 2 <= d <= 512; larger d returns RSIGN_ERR_UNSUPPORTED.
 *   - H and R must be device pointers (host buffers would need staging
 *     memory): host pointers return RSIGN_ERR_ARG.  tol and k as for
 *     rsign_reflector; at most 100 Newton-Schulz steps.
 *   - All calls share the static array: calls that overlap on the GPU (on
 *     several streams or from several host threads) race and must be
 *     serialised by the caller.  Each call clears the part it needs zeroed.
 *   - Set-up: the first call on each device looks up the array's device
 *     address (cudaGetSymbolAddress, with that device current).  That first
 *     call should come before any stream capture begins.
 *   - Blocking like rsign_reflector; info->workspace_bytes is 0.
 */
rsign_status rsign_reflector_noalloc(const double* H, int64_t d, int32_t k, double s, double tol,
                                     double* R, rsign_info* info, void* stream);

/* Human-readable name of a status code (static string). */
const char* rsign_status_str(rsign_status st);

/* Library version string, e.g. "rsign 0.1 sm_103a". */
const char* rsign_version(void);

/*
 * rsign_trim_workspace -- return the workspace memory cached by earlier calls
 * to the driver.  Calls take their workspace from a library-owned
 * stream-ordered pool per device that keeps freed memory for the next call
 * (re-mapping tens of GB per call would cost tens of milliseconds); this
 * releases it.  Call it when no rsign call is in flight.  The paper has no
 * counterpart; it is resource management only.
 */
rsign_status rsign_trim_workspace(void);

#ifdef __cplusplus
}
#endif

#endif /* RSIGN_H */
