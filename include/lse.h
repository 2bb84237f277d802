/*
 * lse.h -- C ABI of the GB300 superfast line-spectral-estimation library.
 *
 * The method is the block-coordinate-descent estimator of Hansen, Fleury and
 * Rao, "Superfast Line Spectral Estimation" (IEEE TSP 2018), complete-data
 * case (Sec. III, Phi = I, M = N): given y in C^N it estimates the model order
 * K and, per component, the frequency theta_k in [0,1), the coefficient
 * alpha_k and the variance gamma_k, plus the noise variance beta
 * (Sec. II, eqs. model, estModel, obj).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * - Complex arrays are interleaved (re, im).  y is complex64; frequencies,
 *   variances and coefficients are double.
 * - Index n runs 0..N-1: [psi(theta)]_n = exp(j 2 pi n theta) (the paper's
 *   n-1 for n = 1..N, eq. model).
 * - The caller owns every buffer it passes.  Host-pointer entry points copy in
 *   and out; the *_d entry points take device pointers and a cudaStream_t
 *   (passed as void*), enqueue their work on that stream and return without
 *   synchronising unless stated.
 * - Errors are reported only through lse_status; nothing is thrown across
 *   the ABI.  A context is not thread-safe: use one context per host thread.
 */
#ifndef LSE_H
#define LSE_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LSE_API __attribute__((visibility("default")))
#else
#define LSE_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct lse_ctx lse_ctx;

typedef enum lse_status {
  LSE_OK = 0,
  LSE_EINVAL = 1,    /* an argument is out of range (message via lse_last_error) */
  LSE_ENOMEM = 2,    /* a device allocation failed */
  LSE_EBUDGET = 3,   /* the request needs more device memory than hbm_budget_bytes */
  LSE_ENUMERIC = 4,  /* the Levinson recursion met a pivot <= 0 or a non-finite value */
  LSE_ENOTCONV = 5,  /* max_outer iterations reached; the current estimate is returned */
  LSE_ETIMEOUT = 6,  /* a bounded device-side wait expired */
  LSE_ECUDA = 7,     /* a CUDA runtime call failed */
  LSE_ECAPACITY = 8  /* more components than the caller's capacity; K is set, arrays untouched */
} lse_status;

/* Arithmetic of the hot path.
 * LSE_PREC_FP64: every step in FP64 (the plain path).
 * LSE_PREC_MIXED: first column, Levinson recursion, Gohberg-Semencul apply,
 *   objective, off-grid Newton sums, beta and gamma updates in FP64; grid
 *   FFTs and the grid combine/search in FP32 (complex64); every grid
 *   decision (argmin, approximate-activation candidates) is re-scored in
 *   FP64 before it is taken.  (FP32 Newton sums were measured to break the
 *   line search, so they stay FP64.)
 * LSE_PREC_MIXED_DF: as LSE_PREC_MIXED, but the first column, the Levinson
 *   recursion, the Gohberg-Semencul transforms and the off-grid Newton sums
 *   run in double-float arithmetic (pairs of FP32 numbers, 48-bit
 *   significand) on the FP32 pipes, which on GB300 are ~64x faster than its
 *   FP64 pipe; the objective, beta and gamma updates stay FP64.  Grid
 *   decisions are re-scored with the double-float off-grid sums. */
enum { LSE_PREC_FP64 = 0, LSE_PREC_MIXED = 1, LSE_PREC_MIXED_DF = 2 };

/* element type of grid outputs */
enum { LSE_F32 = 0, LSE_F64 = 1 };

typedef struct lse_config {
  int32_t device;                  /* CUDA device ordinal */
  int32_t precision;               /* LSE_PREC_FP64, LSE_PREC_MIXED or LSE_PREC_MIXED_DF */
  uint64_t hbm_budget_bytes;       /* cap on the context's device workspace; 0 = no cap */
  int32_t grid_size;               /* L for lse_fit*: 0 = 8N rounded to the nearest power of two
                                      (Sec. II-C5 footnote); > 0: that L (a power of two >= 2N) */
  double tau;                      /* threshold adjustment of eq. (activate_criterion); paper: 5 */
  int32_t max_outer;               /* outer-iteration cap (paper silent); default 200 */
  int32_t max_inner;               /* (theta,gamma) updates per outer iteration (Sec. II-D): 5 */
  int32_t approx_activation_iters; /* outer iterations that may use the approximate activation
                                      of Sec. II-E; default 10; 0 disables it */
  uint64_t flags;                  /* LSE_FLAG_* bits; other bits must be 0 */
} lse_config;

/* Disable the grid-FFT autotuner.  By default the first grid evaluation of a
 * context for a new (element type, L) times every on-chip FFT schedule on that
 * batch (this synchronises the stream once) and keeps the fastest; with the
 * environment variable LSE_AUTOTUNE_CACHE naming a file, choices are loaded
 * at lse_create and saved after tuning.  Tune (or load the cache) before
 * capturing grid evaluations into a CUDA graph. */
#define LSE_FLAG_NO_AUTOTUNE 1u

/* Run every fit and eval-grid factorisation in one block per instance.  By
 * default a launch whose batch leaves a spare SM per instance runs as
 * two-block thread-block clusters: on every precision path when all its
 * instances take the superfast recursion (N >= 64), and on the double-float
 * path (LSE_PREC_MIXED_DF) also with Levinson instances.  For an instance on
 * the superfast recursion the second block takes half of every pass of the
 * recursion's FFT stages kept in global memory, of its refinement step and
 * of the Gohberg-Semencul applies (and, in lse_eval_grid, of the omega_s
 * transforms); the results equal the one-block launch's bit for bit.  For an
 * instance on the Levinson recursion (double-float path) the second
 * block takes half of every order when the recursion fits in shared memory
 * (N <= about 6000); when a batch with Levinson instances has a larger N and
 * the launch leaves eight SMs per instance, the clusters have eight blocks
 * sharing the recursion's vectors in global memory (instances small enough
 * for shared memory, and superfast ones, then run in one block).  The
 * Levinson results agree with the one-block launch to rounding (the inner
 * products are summed in a different order). */
#define LSE_FLAG_NO_CLUSTER 2u

/* Run the O(N^2) Levinson-Durbin recursion for every N.  By default the
 * Gohberg-Semencul generator of an instance with N >= 64 comes from a
 * divide-and-conquer ("superfast") Schur recursion, O(N log^2 N): runs of
 * orders combined as 2x2 polynomial matrices by FFT products (the faster
 * route for large N the paper names, Sec. III intro), in one thread block per
 * instance.  Both give the same generator, ln|C| and pivots to rounding; the
 * superfast path loses about a decimal digit more to rounding at large
 * kappa(C). */
#define LSE_FLAG_LEVINSON 4u

/* Compute the off-grid sums of Sec. III-B/C (q, r, u at the active
 * frequencies and the generator sums behind s, t, v, x; also the sums that
 * re-score grid candidates) directly, O(N) per frequency, for every K.  By
 * default a set of at least 32 frequencies (N >= 64) goes through a type-2
 * non-uniform FFT instead (the route of the Sec. III-B footnote): the
 * sequences divided by the transform of a Kaiser-Bessel kernel of width 16,
 * one batched FFT of M >= 2N points, and a 16-point interpolation per
 * frequency, O(N log N + 16 K); its error is near the FFT's own rounding
 * (about 1e-14 of sum |f_n|). */
#define LSE_FLAG_DIRECT_SUMS 8u

/* Take step 4a of the estimator (the (theta, gamma) update, Sec. II-D) as one
 * L-BFGS update, the paper's own choice (Sec. II-C1, J = 10 saved pairs),
 * instead of the default per-component diagonal Newton step: the initial
 * inverse Hessian of every update is the diagonal of eqs. (derivative2) with
 * its replacements ((50N)^2, gamma^-2), the direction comes from the two-loop
 * recursion over the pairs kept (s.y > 0), the memory is emptied at the start
 * of step 4 of every outer iteration and whenever a component is removed, and
 * the stopping decrement is g.H g.  With no pair saved the step is the Newton
 * one.  Applies to the complete-data fits (single and multiple measurement
 * vectors); the incomplete-data fits use the Newton step. */
#define LSE_FLAG_LBFGS 16u

/* Fill cfg with the paper's defaults (device 0, FP64, tau = 5, ...). */
LSE_API void lse_config_default(lse_config* cfg);

/* Result of one fit.  K_cap, theta, alpha and gamma are set by the caller;
 * everything else is written by the library.  Components are sorted by
 * frequency.  alpha_k = gamma_k q_k is the posterior mean of eq. (bmu)
 * (footnote to eq. bmu). */
typedef struct lse_result {
  int32_t K;          /* out: number of active components */
  int32_t K_cap;      /* in: capacity of theta, gamma (K_cap) and alpha (2*K_cap) */
  double* theta;      /* out [K_cap]: frequencies in [0,1), ascending */
  double* alpha;      /* out [2*K_cap]: complex coefficients, interleaved */
  double* gamma;      /* out [K_cap]: component variances > 0 */
  double beta;        /* out: noise variance */
  double objective;   /* out: eq. (obj) at the returned state, without the constant */
  int32_t iters;      /* out: outer iterations run */
  int32_t n_evals;    /* out: model evaluations (factorisations of C) */
  int32_t n_grid;     /* out: grid evaluations (activation searches, Sec. II-C5) */
} lse_result;

/* Device-resident results of a batched fit.  Instance b owns the slice
 * [off_b, off_b + N_b) of theta, gamma and alpha (complex, interleaved) where
 * off_b is the instance's offset in the y batch: K <= N always (K_max = N,
 * footnote in Sec. II-A), so the slice always fits.  All arrays are device
 * memory owned by the caller. */
typedef struct lse_batch_out {
  double* theta;      /* [sum N_b] */
  double* gamma;      /* [sum N_b] */
  double* alpha;      /* [2 * sum N_b] */
  int32_t* K;         /* [B] */
  double* beta;       /* [B] */
  double* objective;  /* [B] */
  int32_t* iters;     /* [B] */
  int32_t* n_evals;   /* [B] */
  int32_t* n_grid;    /* [B] */
  int32_t* status;    /* [B] lse_status per instance */
} lse_batch_out;

/* Create a context on cfg->device (cfg may be NULL for defaults).  The
 * context owns its device workspace, twiddle tables and stream. */
LSE_API lse_status lse_create(const lse_config* cfg, lse_ctx** out);

/* Release everything the context owns.  NULL is accepted. */
LSE_API void lse_destroy(lse_ctx* ctx);

/* Static description of a status code. */
LSE_API const char* lse_strerror(lse_status s);

/* Detail of the last failing call on this context (empty if none). */
LSE_API const char* lse_last_error(const lse_ctx* ctx);

/* Fit one instance (Sec. II algorithm; superfast evaluations of Sec. III).
 * y: host, complex64 [2*N floats]; 2 <= N <= 131072.  On LSE_ECAPACITY out->K holds
 * the number of components and the arrays are not written.  Blocks until the
 * result is in out. */
LSE_API lse_status lse_fit(lse_ctx* ctx, const float* y, int32_t N, lse_result* out);

/* Fit B independent instances of possibly different N in one launch.
 * y: host complex64, instance b = y[offsets[b] .. offsets[b+1]) (complex
 * elements); offsets has B+1 entries, offsets[0] = 0.  outs[b] and
 * per_instance[b] receive instance b's result and status; the return value
 * is LSE_OK if the launch ran (instances fail independently) or the first
 * launch-level error.  Blocks until done. */
LSE_API lse_status lse_fit_batch(lse_ctx* ctx, const float* y, const int64_t* offsets, int32_t B,
                         lse_result* outs, lse_status* per_instance);

/* Device-pointer batched fit.  y_d: device complex64 batch; offsets: HOST
 * array [B+1] as in lse_fit_batch; out: device arrays (lse_batch_out).
 * stream: cudaStream_t (NULL = the context's stream).  Asynchronous: the
 * results are valid once the stream has reached this point.  The call does
 * not wait for the device, except when the context must grow its device
 * memory or twiddle tables (a larger shape than any before).  Launch
 * descriptors are uploaded only when they differ from the previous call's.
 * The call may be stream-captured once a call with the same offsets has run
 * outside capture (nothing is then allocated or uploaded); otherwise it
 * returns LSE_EINVAL during capture.  While capturing, ordering against the
 * context's own stream is left to the caller. */
LSE_API lse_status lse_fit_batch_d(lse_ctx* ctx, const float* y_d, const int64_t* offsets, int32_t B,
                           const lse_batch_out* out, void* stream);

/* ---- Multiple measurement vectors (Sec. V) ---------------------------------
 * G snapshots y^(1), ..., y^(G) of one instance share the frequencies, the
 * variances gamma, the noise variance and the activation probability, hence
 * one covariance C (eq. py); each snapshot has its own coefficients.  The fit
 * minimises G ln|C| + sum_g y_g^H C^{-1} y_g minus the prior term (eq. L_MMV):
 * one factorisation of C per evaluation serves every snapshot, while the
 * Gohberg-Semencul apply, the q, r, u sums and the q grid run per snapshot.
 * The derivatives are sums over snapshots (Sec. V); activation and
 * deactivation use Q = sum_g |q_g|^2 in eq. (singlecomp-mmv): gamma-hat =
 * (Q/G - s)/s^2, Delta L = G ln(1 + gb s) + ln((1-zeta)/zeta) - gb Q/(1 + gb s),
 * the activation test Q/(G s) > (1 + 1/(gb s)) (ln(1 + gb s) + ln((1-zeta)/zeta)/G)
 * + tau, and the removal test gamma Q~/(1 + gamma s~) - G ln(1 + gamma s~) <
 * ln((1-zeta)/zeta); beta averages the residual term over snapshots; the
 * initial beta, eps_beta and the termination and Newton-decrement thresholds
 * scale with G N.  With G = 1 every rule is the single-snapshot one and the
 * results equal lse_fit's bit for bit. */

/* Fit one instance of G snapshots.  y: host complex64, G x N snapshot-major
 * (snapshot g at y[2 g N .. 2 (g+1) N)); 2 <= N <= 131072, 1 <= G <= 1024.
 * out->alpha holds K_cap x G complex values: snapshot g's coefficient of
 * component k at alpha[2 (g K_cap + k)] (eq. bmu with y replaced by y^(g));
 * theta and gamma as for lse_fit.  Blocks until the result is in out. */
LSE_API lse_status lse_fit_mmv(lse_ctx* ctx, const float* y, int32_t N, int32_t G, lse_result* out);

/* Batched device-pointer fit of B instances of G snapshots each (G the same
 * for the whole batch, N ragged).  offsets: HOST [B+1] in samples per
 * snapshot, as for lse_fit_batch_d; instance b's snapshot g starts at complex
 * element G offsets[b] + g N_b of y_d.  out: as lse_batch_out, except that
 * alpha holds 2 G sum N_b doubles: instance b's snapshot g's coefficient of
 * its k-th component at complex element G offsets[b] + g N_b + k.  The
 * asynchrony and stream-capture rules of lse_fit_batch_d apply. */
LSE_API lse_status lse_fit_mmv_batch_d(lse_ctx* ctx, const float* y_d, const int64_t* offsets, int32_t B,
                                       int32_t G, const lse_batch_out* out, void* stream);

/* ---- Planned batches and CUDA graphs ----------------------------------
 * A plan fixes the shape of a batched fit (offsets, B) and owns its device
 * workspace, so that a launch enqueues device work only (a counter reset and
 * one persistent fit kernel that pulls instances, largest N first) and can be
 * captured into a CUDA graph. */
typedef struct lse_plan lse_plan;

/* Prepare fits of B instances laid out as `offsets` (HOST, B+1 entries, as for
 * lse_fit_batch) with the context's configuration.  Allocates the plan's
 * workspace (counted against hbm_budget_bytes) and uploads the descriptors. */
LSE_API lse_status lse_plan_fit(lse_ctx* ctx, const int64_t* offsets, int32_t B, lse_plan** out);

/* Enqueue one batched fit of the planned shape on `stream` (cudaStream_t; NULL
 * = legacy default stream): device pointers as for lse_fit_batch_d.  No host
 * synchronisation and no allocation, so the call may be stream-captured.  One
 * launch of a plan at a time: launches of the same plan share its workspace. */
LSE_API lse_status lse_plan_launch(lse_plan* plan, const float* y_d, const lse_batch_out* out, void* stream);

/* As lse_plan_launch, through a CUDA graph: the first call (and any call with
 * different y_d / out pointers) captures the launch into a graph on the
 * context's stream and instantiates it; every call then replays it on
 * `stream` with one cudaGraphLaunch. */
LSE_API lse_status lse_plan_graph_launch(lse_plan* plan, const float* y_d, const lse_batch_out* out, void* stream);

/* Wait for the device, release the plan's graph and workspace.  NULL is accepted. */
LSE_API void lse_plan_destroy(lse_plan* plan);

/* ---- Serving: continuous batching ---------------------------------------
 * A server owns `streams` slots (each a stream, a context and device
 * buffers).  lse_serve_submit queues a request; lse_serve_poll (never
 * blocks on the GPU) hands back finished results, then lets every idle slot
 * take the oldest pending requests (at most max_group, and only as many as
 * the remaining device-memory budget cfg->hbm_budget_bytes allows; 0 = no
 * cap) and launch one batched fit over them.  Requests that arrive while
 * other groups run start on free slots, so their work overlaps on the
 * device.  Each instance is fitted with the arithmetic of a lone lse_fit, so
 * its result does not depend on the batch it ran in: bit for bit when the
 * group and the lone fit run in the same unit mode (one block, or a cluster;
 * see LSE_FLAG_NO_CLUSTER), to rounding otherwise.
 * Not thread-safe: one server per host thread. */
typedef struct lse_server lse_server;

typedef struct lse_serve_result {
  int64_t request_id;  /* out: the id given to lse_serve_submit */
  int32_t status;      /* out: lse_status of this request */
  int32_t N;           /* out */
  int32_t K;           /* out: number of components (written even if K > K_cap) */
  int32_t K_cap;       /* in: capacity of theta, gamma (K_cap) and alpha (2*K_cap) */
  double* theta;       /* in: caller array (may be NULL) */
  double* gamma;       /* in: caller array (may be NULL) */
  double* alpha;       /* in: caller array, complex interleaved (may be NULL) */
  double beta;         /* out */
  double objective;    /* out */
  int32_t iters;       /* out */
  int32_t n_evals;     /* out */
} lse_serve_result;

/* cfg: fit configuration and total device-memory budget (NULL = defaults). */
LSE_API lse_status lse_serve_create(const lse_config* cfg, int32_t streams, int32_t max_group, lse_server** out);

/* Queue a request: y HOST complex64 [2N], copied; 2 <= N <= 131072.
 * LSE_EBUDGET if the request alone needs more device memory than the budget. */
LSE_API lse_status lse_serve_submit(lse_server* s, const float* y, int32_t N, int64_t request_id);

/* Harvest finished groups, admit pending requests, and write up to `cap`
 * finished results into `results` (their K_cap/theta/gamma/alpha set by the
 * caller; a result whose K exceeds K_cap gets status LSE_ECAPACITY).  Returns
 * the number written (results may be NULL to discard), -1 on a NULL server. */
LSE_API int32_t lse_serve_poll(lse_server* s, lse_serve_result* results, int32_t cap);

/* Requests submitted and not yet returned by lse_serve_poll. */
LSE_API int32_t lse_serve_in_flight(const lse_server* s);

/* Device memory the running groups hold, in bytes (the budgeted quantity). */
LSE_API uint64_t lse_serve_device_bytes(const lse_server* s);

/* Grow every slot's device buffers and fit workspace, once, for a full group
 * of max_group requests of up to n_max samples each (L = cfg->grid_size, or
 * 8 n_max rounded to the nearest power of two).  A slot otherwise grows when
 * a larger group first reaches it, and releasing device memory waits for
 * every fit running on the device, which stalls lse_serve_poll and the whole
 * admission loop behind the longest running group.  Call it before traffic
 * starts; it waits for the slots' running groups (their results stay
 * queued for lse_serve_poll) and for the device.  The reserved memory is not
 * counted against hbm_budget_bytes, which budgets running groups. */
LSE_API lse_status lse_serve_reserve(lse_server* s, int32_t n_max);

/* Wait for running groups and release everything.  NULL is accepted. */
LSE_API void lse_serve_destroy(lse_server* s);

/* Grid evaluation (Sec. III-D): for C = beta I + sum_k gamma_k psi(theta_k)
 * psi(theta_k)^H (eq. py), compute on theta_l = l/L, l = 0..L-1,
 *   q(theta) = psi(theta)^H C^{-1} y,   s(theta) = psi(theta)^H C^{-1} psi(theta)
 * and their first and second theta-derivatives.  All components given are
 * active; the evaluation uses the full C (C_{~k} = C for a component that is
 * not in the set, Sec. III-D).  Host pointers; y complex64 [2N]; theta, gamma
 * [K] (K >= 0); beta > 0; L a power of two with L >= 2N.  Outputs: q, dq, d2q
 * complex [2L], s, ds, d2s real [L], element type dtype (LSE_F64 for an
 * LSE_PREC_FP64 context, LSE_F32 for LSE_PREC_MIXED and LSE_PREC_MIXED_DF);
 * any output may be NULL.
 * Blocks until done. */
LSE_API lse_status lse_eval_grid(lse_ctx* ctx, const float* y, int32_t N, const double* theta,
                         const double* gamma, int32_t K, double beta, int32_t L, int32_t dtype,
                         void* q, void* dq, void* d2q, void* s, void* ds, void* d2s);

/* Batched device-pointer grid evaluation of B instances.
 * y_d: device complex64, instance b at y_offsets[b] (HOST array [B+1]).
 * theta_d, gamma_d: device double, instance b's components at
 * k_offsets[b] .. k_offsets[b+1] (HOST array [B+1]).  beta_d: device double
 * [B].  L: HOST int32 [B], each a power of two >= 2 N_b.  Outputs (device,
 * any may be NULL): instance b's grid occupies [g_b, g_b + L_b) with g_b the
 * prefix sum of L (complex outputs count complex elements).  dtype as for
 * lse_eval_grid.  Asynchronous on stream (NULL = the context's stream): the
 * call does not wait for the device except when the context must grow its
 * device memory or twiddle tables, and on the first batch of a new (element
 * type, L), which the grid-FFT autotuner times (LSE_FLAG_NO_AUTOTUNE).  The
 * factorisation and grid kernels may be stream-captured once a call with the
 * same shapes (offsets, L, the set of non-NULL outputs) has run outside
 * capture; otherwise the call returns LSE_EINVAL during capture. */
LSE_API lse_status lse_eval_grid_batch_d(lse_ctx* ctx, const float* y_d, const int64_t* y_offsets,
                                 int32_t B, const double* theta_d, const double* gamma_d,
                                 const int64_t* k_offsets, const double* beta_d,
                                 const int32_t* L, int32_t dtype, void* q, void* dq, void* d2q,
                                 void* s, void* ds, void* d2s, void* stream);

/* ---- Incomplete observations: the semifast evaluation (Sec. IV) ---------
 * Instance b observes M_b = m_offsets[b+1] - m_offsets[b] samples
 * y_m = z(n_m) of an N[b]-sample signal (Phi a row selection; obs_d holds
 * the indices n_m, ascending, in [0, N[b])).  At the state (theta, gamma,
 * beta) of its K_b components (as for lse_eval_grid_batch_d) C is the
 * M_b x M_b matrix beta I + A Gamma A^H with A = Phi Psi(theta) (eq. py), and
 * the evaluation follows Sec. IV: Woodbury's identity (eq. CfromSigma) with
 * one K_b x K_b Cholesky factorisation of Sigma^{-1} = A^H A / beta +
 * Gamma^{-1}, the K_b x K_b matrices A_{D^a}^H A of eq. (AhA) and the sums
 * A_{D^a}^H y by a non-uniform FFT, the grid q by an L-point FFT and the grid
 * s by the O(L K^2) contraction.  Outputs (device, written per instance):
 *   scal_d[2b] = ln|C| (matrix determinant lemma), scal_d[2b+1] = y^H C^{-1} y;
 *   vec_d: 14 doubles per component, complex q, r, u, s, t, v, x of eqs.
 *   (q)-(x) (s and x real, imaginary parts 0) at component k of instance b
 *   starting at double 14 (k_offsets[b] + k);
 *   q (complex) and s (real) on theta_l = l/L[b], instance b at the prefix
 *   sum of L as in lse_eval_grid_batch_d, element type dtype (LSE_F64 for an
 *   LSE_PREC_FP64 context, LSE_F32 otherwise); either may be NULL (both
 *   NULL: no grid);
 *   status_d[b] = LSE_OK, or LSE_ENUMERIC if Sigma^{-1} is not numerically
 *   positive definite.
 * y_d: device complex64 [2 sum M]; obs_d: device int32 [sum M];
 * m_offsets, N, k_offsets, L: HOST arrays.  0 <= K_b <= min(M_b, 96),
 * 1 <= M_b <= N[b] <= 131072, L[b] a power of two >= 2 N[b].  The K x K
 * algebra is FP64; the transforms, interpolations and the grid contraction
 * are FP64 on an LSE_PREC_FP64 context and double-float otherwise.
 * Asynchronous on stream as lse_eval_grid_batch_d (kernel time: which = 1 of
 * lse_kernel_time). */
LSE_API lse_status lse_eval_semifast_batch_d(lse_ctx* ctx, const float* y_d, const int32_t* obs_d,
                                             const int64_t* m_offsets, int32_t B, const int32_t* N,
                                             const double* theta_d, const double* gamma_d,
                                             const int64_t* k_offsets, const double* beta_d, const int32_t* L,
                                             int32_t dtype, double* scal_d, double* vec_d, void* q, void* s,
                                             int32_t* status_d, void* stream);

/* Fit instances from incomplete observations (Sec. II with the semifast
 * evaluation of Sec. IV for every model evaluation).  Instance b observes
 * M_b = m_offsets[b+1] - m_offsets[b] samples of an N[b]-sample signal at
 * the distinct indices obs_d[m_offsets[b] ..] (ascending, in [0, N[b])).
 * The estimator is lse_fit's with M where the paper counts observations
 * (K_max = M, zeta = K/M, beta divided by M, the M 1e-7 and M 1e-8
 * thresholds of Sec. II-D) and N where it measures resolution ((50N)^2,
 * 0.05/N); grid values are FP64-class on every path, so grid decisions are
 * taken on them directly.  At most min(M, 96) components are activated.
 * y_d: device complex64 [2 sum M]; obs_d: device int32 [sum M]; m_offsets,
 * N: HOST arrays; out: device arrays as in lse_batch_out with instance b's
 * theta, gamma, alpha slice at m_offsets[b].  L per instance: cfg->grid_size,
 * or 8 N rounded to the nearest power of two.  FP64 arithmetic on an
 * LSE_PREC_FP64 context, double-float (with FP64 K x K algebra) otherwise.
 * Asynchronous on stream (NULL = the context's stream); kernel time: which
 * = 0 of lse_kernel_time.  An index outside [0, N) ends that instance with
 * LSE_EINVAL. */
LSE_API lse_status lse_fit_incomplete_batch_d(lse_ctx* ctx, const float* y_d, const int32_t* obs_d,
                                              const int64_t* m_offsets, int32_t B, const int32_t* N,
                                              const lse_batch_out* out, void* stream);

/* One instance of lse_fit_incomplete_batch_d from host arrays: y complex64
 * [2 M], obs int32 [M]; out as for lse_fit (K_cap set by the caller).
 * Returns the instance's status.  Blocks until done. */
LSE_API lse_status lse_fit_incomplete(lse_ctx* ctx, const float* y, const int32_t* obs, int32_t M, int32_t N,
                                      lse_result* out);

/* Device time of this context's kernels, from CUDA events recorded on the
 * launch stream around every launch since the previous call.  which: 0 = fit
 * kernel, 1 = factorisation kernel (first column, Levinson recursion,
 * Gohberg-Semencul apply), 2 = grid kernel.  Waits for the recorded events,
 * writes the summed time in milliseconds and the number of launches, and
 * clears the record. */
LSE_API lse_status lse_kernel_time(lse_ctx* ctx, int32_t which, double* total_ms, int64_t* launches);

/* Fit one instance without allocating any device memory.
 *
 * For callers that must not allocate on the GPU when they run a fit: loops
 * with a hard per-frame deadline (cudaMalloc/cudaFree can stall for
 * milliseconds and synchronise the whole device), hosts embedded in a
 * framework that owns every device allocation, or code that has finished
 * its set-up phase and may no longer call the allocator.  No context is
 * needed; nothing here calls cudaMalloc, cudaFree or any allocating routine.
 *
 * The paper has no counterpart to this entry point.
 *
 * The caller passes y_d (device complex64 [2N floats]) and out: device
 * arrays as in lse_batch_out for B = 1 (theta, gamma capacity N, alpha 2N
 * doubles, and one element each for K, beta, objective, iters, n_evals,
 * n_grid, status).  cfg (host, may be NULL for the defaults) supplies tau,
 * the iteration limits, grid_size and precision; cfg->device and
 * hbm_budget_bytes are ignored -- the fit runs on the current device.
 * The fit is enqueued on `stream` (a cudaStream_t; NULL = legacy default
 * stream) and the call returns without waiting.
 *
 * Limits: 2 <= N <= 4096 and L <= 32768 (L = cfg->grid_size, or 8N rounded
 * to the nearest power of two), and the kernel workspace for (N, L) must fit
 * the library's 8 MiB static scratch array; anything larger returns
 * LSE_EINVAL before any work is enqueued.
 *
 * Every precision runs the arithmetic of lse_fit_batch_d with the same
 * configuration (the library's own twiddle tables are static arrays too).
 * cfg->flags accepts the LSE_FLAG_* bits only; grid_size must be >= 0.
 *
 * The scratch is a fixed array inside the library, present on every GPU
 * that loads it until the process exits, and shared by all calls: calls
 * whose work overlaps on the GPU (other streams, other host threads) race
 * on it, so serialise them.  Each call clears what must start at zero (the
 * launch's work counter, written together with the launch descriptor by a
 * small kernel that takes them as parameters); the rest keeps the previous
 * call's contents and is rewritten before it is read.  The first call on a
 * device does a one-time set-up there: it looks up the device addresses of
 * the static arrays, fills the twiddle tables on its stream and waits for
 * that fill; make that first call before any stream capture.  The addresses
 * belong to the device's primary context: do not use this entry point after
 * cudaDeviceReset. */
LSE_API lse_status lse_fit_noalloc_d(const lse_config* cfg, const float* y_d, int32_t N,
                                     const lse_batch_out* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* LSE_H */
