/*
 * uotk.h -- C ABI of the GB300 (sm_103a) kernel-summation library for entropic
 * unbalanced optimal transport and maximum mean discrepancies
 * (Lakshmanan & Pichler, arXiv 2306.13618).
 *
 * General conventions, valid for every entry point below:
 *  - Array arguments named as device arrays are DEVICE pointers owned by the
 *    caller.  The library never frees them and never keeps them past the call.
 *    Point clouds are row-major FP32 (point i occupies p[i*d .. i*d+d-1]).
 *    Every device pointer must be 4-byte aligned (8 for FP64 arrays).
 *  - `stream` is a cudaStream_t (passed as void*); all device work is enqueued
 *    on it.  Calls that return host scalars synchronise that stream.
 *  - Scratch memory is owned by the context (uotk_ctx) and grows on demand; a
 *    context serves one host thread at a time and one device.
 *  - Every call returns a uotk_status and never aborts, traps or prints.  On
 *    error, uotk_last_error(ctx) gives a message.  Arguments are validated on
 *    the host before any launch; data-dependent checks (negative or non-finite
 *    weights, non-finite coordinates) run on the device and are reported by
 *    the same call, which then synchronises its stream.
 *  - Notation: eps is the kernel width of K(x,y) = exp(-||x-y||^2/eps), the
 *    paper's Gibbs kernel k = exp(-lambda d^2) with lambda = 1/eps (Alg. 1,
 *    Def. def:526); rho (eta in the paper) is the KL marginal penalty.
 */
#ifndef UOTK_H
#define UOTK_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct uotk_ctx uotk_ctx;

typedef enum {
  UOTK_OK = 0,
  UOTK_ERR_INVALID = 1,        /* bad argument (null pointer, size, parameter range) */
  UOTK_ERR_NOMEM = 2,          /* device or pinned allocation failed */
  UOTK_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  UOTK_ERR_UNSUPPORTED = 4,    /* valid request the library does not implement (e.g. NFFT with d > 3) */
  UOTK_ERR_NONFINITE = 5,      /* NaN/Inf in inputs, or a non-finite dual/result */
  UOTK_ERR_NOT_CONVERGED = 6,  /* tol > 0 and max_sweeps reached; outputs are valid */
  UOTK_ERR_TIMEOUT = 7,        /* a bounded device-side wait gave up */
  UOTK_ERR_INTERNAL = 8
} uotk_status;

/* Form of every kernel summation of a call (never switched silently):
 * DIRECT      : the exact O(nm) sum of Alg. 1 in FP32 (any d <= 128).
 * NFFT        : the fast summation of Sec. 4 / Alg. 2 (d <= 3).
 * DIRECT_BF16 : the exact O(nm) sum with the cross term x.y of
 *               ||x-y||^2 = |x|^2 + |y|^2 - 2 x.y on the tensor cores from
 *               BF16-rounded centred points (FP32 accumulation, norms and
 *               exponentials in FP32); about 3 significant digits per term.
 * DIRECT_BF16X3: the same with each centred coordinate split into BF16 hi + lo
 *               and x.y = hi.hi + hi.lo + lo.hi (three tensor-core products),
 *               near FP32 accuracy.
 * The two tensor-core forms take d <= 128; they pay off for d >~ 16, where the
 * FP32 form spends d FMAs per pair on the distance. */
typedef enum {
  UOTK_DIRECT = 0,
  UOTK_NFFT = 1,
  UOTK_DIRECT_BF16 = 2,
  UOTK_DIRECT_BF16X3 = 3,
  /* the form chosen by uotk_autotune_sum for the problem at hand (cached per
   * context); accepted by uotk_kernel_sum, uotk_uot_sinkhorn,
   * uotk_sinkhorn_divergence, uotk_mmd2 and their gradients (Gaussian kernel) */
  UOTK_AUTO = 4
} uotk_method;

/* Reference measure of the entropy term.
 * PRODUCT : (1/lambda) D(pi || mu (x) nu), the paper's Eq. (W4); the update is
 *           beta_i = -q log sum_j k_ij nu_j e^{lambda gamma_j}  (Eq. Sinkhorn_uot_iteration).
 * COUNTING: the counting reference, whose scaling update reads
 *           u = (a / (K v))^{rho/(rho+eps)},  u = e^{lambda beta}, v = e^{lambda gamma}.
 * q = rho/(1 + rho*lambda) in both. */
typedef enum { UOTK_REF_PRODUCT = 0, UOTK_REF_COUNTING = 1 } uotk_ref;

/* Kernels of Table tab:0, r = ||x - x~||, parameter p:
 *   GAUSS   exp(-r^2/eps)       (the Gibbs kernel of Alg. 1/2; p^2 = eps)
 *   LAPLACE exp(-r/p)
 *   IMQ     1/sqrt(r^2 + p^2)   (p = the constant c of the table)
 *   ENERGY  -r                  (p unused; any positive value)
 * The non-Gaussian kernels are available in uotk_kernel_sum (eps = p) and
 * uotk_mmd2 (ell = p), in the direct FP32 form and the NFFT form (d <= 3);
 * every other combination returns UOTK_ERR_UNSUPPORTED.  Their NFFT form is the
 * regularised fast summation of Sec. 4.2: on the torus (period h, units
 * rbar = r/h) the kernel is replaced by K_R, equal to K for
 * eps_I <= rbar <= 1/2 - eps_B and by two-point Taylor polynomials of degree
 * 2p - 1 (p = reg_degree, matching K's derivatives of order < p) below eps_I and
 * up to 1/2, constant beyond; b_k is the DFT of K_R sampled on I_N^d, and the
 * near field |x - y| < eps_I h adds w (K - K_R) directly.  eps_I = eps_B = p/N;
 * h = (Euclidean diameter of the joint bounding box) / (1/2 - eps_B), so that
 * K_R = K wherever no near-field correction is made.  Defaults grid 256,
 * N = 128, p = 4 (max error about 1e-6 of sum|w| max|K| on uniform clouds);
 * the near field costs (number of pairs closer than eps_I h) kernel
 * evaluations, so the form pays when that is a small fraction of n m. */
typedef enum {
  UOTK_KERNEL_GAUSS = 0,
  UOTK_KERNEL_LAPLACE = 1,
  UOTK_KERNEL_IMQ = 2,
  UOTK_KERNEL_ENERGY = 3
} uotk_kernel;

/* Options of one kernel summation.  A NULL pointer means all defaults. */
typedef struct {
  int32_t method;      /* uotk_method; default UOTK_DIRECT */
  int32_t grid;        /* NFFT: oversampled grid size n per dimension, power of two in [16, 256]; 0 = 128 (256 for the non-Gaussian kernels) */
  int32_t bandwidth;   /* NFFT: bandwidth N, even, 4 <= N <= grid; 0 = grid/2 (oversampling sigma = 2) */
  int32_t cutoff;      /* NFFT: window cut-off m in [2, 8]; 0 = smallest of 6, 7, 8 meeting target_err */
  double period;       /* NFFT: torus period h; 0 = chosen from the data and eps (non-Gaussian kernels: must be >= the automatic choice) */
  double target_err;   /* NFFT: accuracy goal, max error relative to sum|w|; 0 = 1e-6.  Non-Gaussian kernels: bound on the error per unit weight relative to max|K| (the plan's Fourier series against K_R, checked at plan time; UNSUPPORTED if missed); 0 = 1e-3 (sums then measure about 1e-6 of sum|w| max|K| at the defaults) */
  int32_t kernel;      /* uotk_kernel; default UOTK_KERNEL_GAUSS */
  int32_t reg_degree;  /* NFFT, non-Gaussian kernels: regularisation degree p in [2, 12]; 0 = 4 */
} uotk_sum_opts;

/* Parameters of an NFFT fast summation as chosen by uotk_nfft_plan (Sec. 4).
 * Torus coordinates u = (p - center) * inv_h + 1/2, reduced mod 1; grid node l
 * sits at u = l/grid.  Grids are grid^3 FP32 arrays laid out [z][y][x] (x
 * fastest), d < 3 being embedded with the missing coordinates at the centre. */
typedef struct {
  int32_t d;           /* dimension of the points, 1..3 */
  int32_t grid;        /* oversampled grid n */
  int32_t bandwidth;   /* N: Fourier coefficients b_k kept for k in {-N/2..N/2-1}^3 */
  int32_t cutoff;      /* window cut-off m: each point touches (2m)^3 grid nodes */
  float center[3];     /* c */
  float inv_h;         /* 1/h as the FP32 value every kernel uses */
  double h;            /* torus period */
  double eps;          /* kernel width the plan was made for */
} uotk_nfft_plan_info;

/* ---- context ---------------------------------------------------------------- */

/* Create a context on CUDA device `device` (makes it current).  *out receives the
 * context; release it with uotk_destroy. */
uotk_status uotk_create(uotk_ctx** out, int device);
void uotk_destroy(uotk_ctx* ctx);
/* Message of the last error on this context ("" if none); owned by the context. */
const char* uotk_last_error(const uotk_ctx* ctx);
const char* uotk_status_string(int status);
/* Number of device kernels this context has launched so far (instrumentation). */
int64_t uotk_launch_count(const uotk_ctx* ctx);

/* Per-stage device timing (instrumentation; the paper reports wall time only).
 * With profiling enabled, every kernel launch of the library is bracketed by
 * CUDA events on its stream, grouped by stage name ("direct", "spread",
 * "fft", "gather", "update", ...).  uotk_profile_read synchronises the device,
 * writes up to `max` stages (names as a ';'-separated list into names[cap],
 * launches into counts[], summed milliseconds into ms[]) and returns the
 * number of stages; uotk_profile_reset clears the totals. */
uotk_status uotk_set_profiling(uotk_ctx* ctx, int enable);
int uotk_profile_read(uotk_ctx* ctx, char* names, int cap, int64_t* counts, double* ms, int max);
void uotk_profile_reset(uotk_ctx* ctx);

/* Failure-path controls (the paper has none; they let a caller, and the tests,
 * reach the NOMEM and TIMEOUT statuses without any device fault).
 * uotk_set_workspace_limit: the largest device workspace, in bytes, the context
 * may hold (0: no limit, the default).  A call that needs more returns
 * UOTK_ERR_NOMEM before it launches anything; the context stays usable.
 * uotk_set_wait_timeout_test: with cycles > 0, the first bounded wait of each
 * CTA of the NFFT spread and gather kernels waits on a barrier that nothing
 * completes, for at most `cycles` clock cycles, so that it times out; 0 (the
 * default) turns this off.  A wait that times out records it, waits (with the
 * normal limit of about 2^31 cycles) for the CTA's bulk copies still in
 * flight, and the CTA leaves; the call returns UOTK_ERR_TIMEOUT and its outputs
 * are not valid.  Both return UOTK_ERR_INVALID for a NULL context or a
 * negative value. */
uotk_status uotk_set_workspace_limit(uotk_ctx* ctx, int64_t bytes);
uotk_status uotk_set_wait_timeout_test(uotk_ctx* ctx, int64_t cycles);

/* Unit throughputs of this GPU (instrumentation for roofline denominators; the
 * paper has no counterpart).  Runs one CTA of 1024 threads per SM, each
 * thread 16 independent chains of 4096 ex2.approx.ftz.f32 (then of FP32 FMA),
 * and divides the operations of each CTA by its clock64() cycles:
 * *ex2_per_clk and *ffma_per_clk (host) receive the mean operations per clock
 * per SM.  Synchronises `stream`; takes a few milliseconds. */
uotk_status uotk_measure_unit_rates(uotk_ctx* ctx, void* stream, double* ex2_per_clk,
                                    double* ffma_per_clk);

/* ---- the kernel summation (Eq. fast_sum; the matrix-vector product of Alg. 1/2) --
 * out[j] = sum_i w[i] * exp(-||src_i - tgt_j||^2 / eps),  j = 0..m-1.
 *   src: device FP32 [n*d]; w: device FP32 [n], every w[i] >= 0 and finite;
 *   tgt: device FP32 [m*d]; out: device FP32 [m] (written, never read).
 *   d >= 1 (direct form: d <= 128; NFFT: d <= 3).  n >= 0, m >= 0 (n = 0 gives
 *   zeros).  eps > 0.  opts->method selects the exact direct O(nm) form or the
 *   NFFT fast summation of Eq. (1724) (spread, FFT, multiply by b_k/phihat^2,
 *   inverse FFT, gather).  Negative/non-finite weights or non-finite
 *   coordinates return UOTK_ERR_INVALID / UOTK_ERR_NONFINITE. */
uotk_status uotk_kernel_sum(uotk_ctx* ctx, void* stream, int d,
                            const float* src, int64_t n, const float* w,
                            const float* tgt, int64_t m, float* out,
                            double eps, const uotk_sum_opts* opts);

/* ---- autotuning of the summation form ---------------------------------------------
 * The paper chooses its NFFT parameters by hand (Rem. on NFFT parameters, Sec. 4);
 * this measures them.  For the Gaussian kernel sum src (n points, weights w) ->
 * tgt (m points) with width eps, on this GPU: the direct FP32 form, for d > 3
 * the tensor-core forms (BF16x3, BF16), and for d <= 3 the NFFT at grid 64 and
 * 128 with cut-off m = 4..8 (only in->grid / in->cutoff when those are set)
 * whose plans accept the data.  Each is timed (one full summation; the direct
 * forms on the first 32768 targets, scaled to m) and its error
 * max_j |s_j - s*_j| / sum_i |w_i| measured at 256 targets spread through tgt
 * against their exact sums, taken in FP64 on the device.  *out receives the
 * fastest form whose error is at most in->target_err (0: 1e-5); the direct
 * FP32 form always qualifies.  report (host double[8], may be NULL): {time of
 * the chosen form in ms, its measured error, time of the direct FP32 form in
 * ms, forms measured, chosen grid (0: direct), chosen cut-off, targets
 * sampled, target}.  The choice is cached in the context per (d, n, m, eps,
 * target, in->grid, in->cutoff, bounding box of the points); a cached problem
 * costs one bounding-box reduction.  in may be NULL; in->kernel must be GAUSS.
 * Runs several summations; synchronises `stream`. */
uotk_status uotk_autotune_sum(uotk_ctx* ctx, void* stream, int d, const float* src, int64_t n,
                              const float* w, const float* tgt, int64_t m, double eps,
                              const uotk_sum_opts* in, uotk_sum_opts* out, double* report);

/* ---- the direct kernel summation without allocation ------------------------------
 * The paper has no counterpart to this entry point; it serves callers that may
 * not allocate device memory while they run: a service that reserves all of its
 * memory when it starts and treats any later allocation as a fault, or code on a
 * latency-critical path where cudaMalloc would synchronise the device or could
 * fail under memory pressure.  It computes what uotk_kernel_sum computes with
 * the direct form, out[j] = sum_i w[i] * exp(-||src_i - tgt_j||^2 / eps),
 * needs no context, and allocates nothing: its scratch is one fixed device
 * array of 4 MiB + 4 KiB inside the library, present on every GPU that loads
 * the library until the process exits.
 *   Limits: 1 <= d <= 3, n <= 65536 sources, m <= 65536 targets; larger
 *   problems return UOTK_ERR_UNSUPPORTED (use uotk_kernel_sum).
 *   src, w, tgt, out: device arrays as for uotk_kernel_sum, owned by the caller.
 *   Uses the current CUDA device.  The first call on a device looks up the
 *   scratch's device address (a one-time set-up); make that first call before
 *   any stream capture.  Every call on a device shares the scratch, so calls
 *   whose work overlaps on the GPU (different streams, or different host
 *   threads) race; serialise them.  Synchronises `stream` to report data
 *   errors: negative weights -> UOTK_ERR_INVALID, non-finite values ->
 *   UOTK_ERR_NONFINITE. */
uotk_status uotk_kernel_sum_noalloc(void* stream, int d, const float* src, int64_t n,
                                    const float* w, const float* tgt, int64_t m, float* out,
                                    double eps);

/* ---- entropic UOT by Sinkhorn's algorithm (Alg. 1 direct, Alg. 2 NFFT) -------------
 * Solves Eq. (W4) (r = 2, lambda = 1/eps, eta1 = rho1, eta2 = rho2) through
 * its dual, Eq. (dual_euot), by the alternating updates of
 * Eq. (Sinkhorn_uot_iteration): one sweep = the beta half-step followed by the
 * gamma half-step, each one kernel summation plus an FP64 update.
 *   x: device FP32 [n*d], a (mu): device FP32 [n] > 0; y: device FP32 [m*d],
 *   b (nu): device FP32 [m] > 0.  beta: device FP64 [n] (output),
 *   gamma: device FP64 [m] (input gamma^0 if flags & UOTK_WARM_START, else
 *   gamma^0 = 0; output gamma^S).
 *   Runs max_sweeps sweeps; if tol > 0 it stops early once
 *   max(||lambda (beta^s - beta^{s-1})||_inf, ||lambda (gamma^s - gamma^{s-1})||_inf) < tol,
 *   tested every 10 sweeps, and returns UOTK_ERR_NOT_CONVERGED (outputs valid)
 *   if that never happens.
 *   sweeps_done (host, may be NULL) receives the sweeps run; value (host, may be
 *   NULL) receives D(beta, gamma) of Eq. (dual_euot) at the final duals (for
 *   ref = COUNTING the coupling term has no reference-mass constant).
 *   Synchronises `stream` before returning. */
#define UOTK_WARM_START 1u
/* flags & UOTK_LOG_DOMAIN: every half-step as a per-row log-sum-exp,
 *   log t_i = max_j a_ij + log sum_j exp(a_ij - max_j a_ij),
 *   a_ij = log w_j - ||x_i - y_j||^2/eps, w_j = nu_j e^{lambda gamma_j} (ref 0),
 * so that neither the weights nor the kernel values need to be representable
 * in FP32 (very small eps).  The direct forms: FP32 (a two-pass row maximum),
 * BF16 and BF16x3 (an online maximum per row in the tensor-core epilogue);
 * UNSUPPORTED with NFFT or another kernel.  The exponents a_ij are FP32: the
 * relative accuracy of each term is that of an FP32 number of the size of
 * |log w_j - M|, M = max_j lambda gamma_j (plus the cross-term error of the
 * BF16 forms). */
#define UOTK_LOG_DOMAIN 2u
/* flags & UOTK_CSTAR_INIT: gamma^0 = c* 1 with c* of Eq. (561) as computed by
 * uotk_cstar (the Remark on the initialisation of Sinkhorn's algorithm read
 * literally: the potential set to the number c*).  ref = PRODUCT only; not
 * together with UOTK_WARM_START (INVALID).
 * The cost: opts->kernel = GAUSS (default) solves Eq. (W4) with d^2 (r = 2, the
 * Gibbs kernel exp(-||x - y||^2/eps)); opts->kernel = LAPLACE solves it with the
 * cost ||x - y|| (r = 1, Gibbs kernel exp(-||x - y||/eps), the Laplace kernel of
 * Table tab:0 with p = eps), in the direct FP32 form or the regularised NFFT
 * (d <= 3; its accuracy needs eps above a few h/N, h the torus period).  Not
 * with UOTK_LOG_DOMAIN (UNSUPPORTED); the same for uotk_sinkhorn_divergence. */
#define UOTK_CSTAR_INIT 4u
uotk_status uotk_uot_sinkhorn(uotk_ctx* ctx, void* stream, int d,
                              const float* x, int64_t n, const float* a,
                              const float* y, int64_t m, const float* b,
                              double eps, double rho1, double rho2,
                              int max_sweeps, double tol, int ref, unsigned flags,
                              double* beta, double* gamma, int* sweeps_done,
                              double* value, const uotk_sum_opts* opts);

/* ---- mean cost and the optimal independent plan (Prop. prop:536) ---------------------
 * uotk_mean_cost: <mu (x) nu | d^r> = sum_i sum_j a_i b_j ||x_i - y_j||^r for
 *   r = 2: from the first and second moments of both clouds about x_0 in FP64,
 *          O((n + m) d), no kernel summation;
 *   r = 1: d = -k_e, the energy kernel of Table tab:0 (Sec. 4.4, complexity of
 *          the upper bounds): one kernel summation with k_e in the form
 *          opts->method (DIRECT, or NFFT for d <= 3: the regularised fast
 *          summation, O(n log n) plus its near field), then an FP64 dot
 *          product with a.
 *   x, a, y, b: as uotk_uot_sinkhorn (n, m >= 1, weights >= 0, d <= 128).
 *   out (host double [3]): {<mu (x) nu|d^r>, mu(X), nu(X)}.  opts may be NULL.
 * uotk_cstar: c*_{r;eta;lambda} of Eq. (561), lambda = 1/eps, eta_i = rho_i:
 *   log c* = -(<mu (x) nu|d^r> / (mu(X) nu(X)) + rho1 log nu(X) + rho2 log mu(X))
 *            / (rho1 + rho2 + eps),
 *   the constant c for which c mu (x) nu minimises Eq. (W4) among such plans.
 *   out (host double [3]): {c*, the Eq. (W4) objective at c* mu (x) nu (an
 *   upper bound of the regularised UOT value, Remark on upper bounds),
 *   <mu (x) nu|d^r>}.
 * Both synchronise `stream`; NONFINITE / INVALID for non-finite inputs or
 * negative weights, INVALID if a measure has zero mass (uotk_cstar) or r is
 * not 1 or 2. */
uotk_status uotk_mean_cost(uotk_ctx* ctx, void* stream, int d,
                           const float* x, int64_t n, const float* a,
                           const float* y, int64_t m, const float* b, int r, double* out,
                           const uotk_sum_opts* opts);
uotk_status uotk_cstar(uotk_ctx* ctx, void* stream, int d,
                       const float* x, int64_t n, const float* a,
                       const float* y, int64_t m, const float* b,
                       double eps, double rho1, double rho2, int r, double* out,
                       const uotk_sum_opts* opts);

/* ---- lambda-scaling (Sec. 5.1.2, "deformed iteration") --------------------------------
 * Alg. 1/2 solved for eps_schedule[0], eps_schedule[1], ... (lambda = 1/eps
 * increasing), each stage started from the previous stage's final gamma
 * (the first from gamma^0 = 0) and run until tol (or max_sweeps_per_stage).
 *   eps_schedule: host double [stages], finite, > 0.
 *   sweeps_per_stage (host int [stages], may be NULL): sweeps run per stage.
 *   beta, gamma, value: as uotk_uot_sinkhorn, for the last stage.
 *   Other arguments as uotk_uot_sinkhorn (flags: UOTK_LOG_DOMAIN only).
 *   Returns UOTK_ERR_NOT_CONVERGED when tol > 0 and the last stage did not
 *   reach it (outputs valid). */
uotk_status uotk_uot_sinkhorn_scaled(uotk_ctx* ctx, void* stream, int d,
                                     const float* x, int64_t n, const float* a,
                                     const float* y, int64_t m, const float* b,
                                     const double* eps_schedule, int stages, double rho1,
                                     double rho2, int max_sweeps_per_stage, double tol, int ref,
                                     unsigned flags, double* beta, double* gamma,
                                     int* sweeps_per_stage, double* value,
                                     const uotk_sum_opts* opts);

/* ---- many independent problems at once (batched Alg. 1 / Alg. 2) -----------------
 * npairs problems (x^p, a^p; y^p, b^p) of uneven sizes, each with its own eps_p,
 * rho1_p, rho2_p, all solved by Alg. 1 together: every half-step of every pair is
 * one grouped launch, and the sweep loop runs on the device (a CUDA graph whose
 * WHILE node repeats two sweeps and a control kernel, captured on the context's
 * own stream).  After every two sweeps the control kernel retires the pairs whose
 * last change met tol, while the others continue, and ends the loop when none is
 * left or max_sweeps would be passed; the host reads the outcome once at the end.
 * With per-stage profiling on, the launches stay eager and the host tests the
 * pairs every 10 sweeps.
 *   x_off, y_off: host int64 [npairs + 1], nondecreasing; pair p owns points
 *     x_off[p] .. x_off[p+1]-1 of x (device FP32 [.*d], row-major) and of a,
 *     and likewise y, b; every pair needs at least one point on each side.
 *   eps, rho1, rho2: host double [npairs], finite and > 0.
 *   beta, gamma: device FP64, indexed like a and b (gamma^0 = 0; output the
 *     final duals of each pair).
 *   sweeps_done (host int [npairs], may be NULL): sweeps run per pair;
 *   values (host double [npairs], may be NULL): D(beta, gamma) per pair.
 *   d in 1..3; opts (may be NULL) selects the direct form (UOTK_DIRECT) or
 *   UOTK_AUTO: every pair with at least 16384 points on both sides then has
 *   its form measured on its own data by the autotuner (as uotk_autotune_sum,
 *   within opts->target_err, default 1e-5, with opts->grid / cutoff fixed if
 *   given), each form timed as one sum on an already built plan, since a solve
 *   builds its plan once.  Pairs whose fastest form is the NFFT (Alg. 2) are
 *   solved one after another by the NFFT solver, the rest together as above;
 *   start, stopping rule, cap and outputs per pair are the same.
 *   uotk_batch_forms reports the form each pair used.
 *   Returns UOTK_ERR_NOT_CONVERGED if tol > 0 and some pair did not reach it
 *   (outputs valid).  Synchronises `stream`. */
uotk_status uotk_uot_sinkhorn_batch(uotk_ctx* ctx, void* stream, int d, int npairs,
                                    const int64_t* x_off, const float* x, const float* a,
                                    const int64_t* y_off, const float* y, const float* b,
                                    const double* eps, const double* rho1, const double* rho2,
                                    int max_sweeps, double tol, int ref, double* beta,
                                    double* gamma, int* sweeps_done, double* values,
                                    const uotk_sum_opts* opts);
/* uotk_batch_forms: forms (host int32 [npairs]) receives the uotk_method each
 * pair of the last uotk_uot_sinkhorn_batch call on ctx was solved with
 * (UOTK_DIRECT or UOTK_NFFT); npairs must be that call's.  Not part of the
 * paper: a report of the per-pair choice of UOTK_AUTO. */
uotk_status uotk_batch_forms(uotk_ctx* ctx, int npairs, int32_t* forms);

/* ---- unbalanced Sinkhorn divergence, Eq. (586) ---------------------------------------
 * sd = UOT(mu,nu) - UOT(mu,mu)/2 - UOT(nu,nu)/2 + (mu(X) - nu(X))^2 * eps/2,
 * each UOT value being D(beta, gamma) after max_sweeps sweeps (or tol, as
 * above) from gamma^0 = 0, product reference, rho1 = rho2 = rho.
 *   sd (host) receives the divergence; parts (host double[3], may be NULL)
 *   receives the three UOT values.  Synchronises `stream`. */
uotk_status uotk_sinkhorn_divergence(uotk_ctx* ctx, void* stream, int d,
                                     const float* x, int64_t n, const float* a,
                                     const float* y, int64_t m, const float* b,
                                     double eps, double rho, int max_sweeps, double tol,
                                     double* sd, double* parts, const uotk_sum_opts* opts);

/* ---- MMD^2, Eq. (1205), Gaussian kernel k(x,y) = exp(-||x-y||^2/ell^2) (Table tab:0) --
 * mmd2 = sum_ij a_i a_j k(x_i,x_j) - 2 sum_ij a_i b_j k(x_i,y_j) + sum_ij b_i b_j k(y_i,y_j),
 * three kernel summations (eps = ell^2) and FP64 dot products.
 *   a, b >= 0.  mmd2 (host) receives the value; parts (host double[3], may be
 *   NULL) receives the three double sums.  Synchronises `stream`. */
uotk_status uotk_mmd2(uotk_ctx* ctx, void* stream, int d,
                      const float* x, int64_t n, const float* a,
                      const float* y, int64_t m, const float* b,
                      double ell, double* mmd2, double* parts, const uotk_sum_opts* opts);

/* ---- gradients (an extension: the paper differentiates neither quantity) ----------
 * Both operations return the value and its partial derivatives with respect to
 * the weights a, b and the support points x, y, as device FP64 arrays in the
 * caller's order: grad_a [n], grad_x [n*d] (row-major like x), grad_b [m],
 * grad_y [m*d].  Any gradient pointer may be NULL (not computed; a NULL
 * point gradient also skips its 2d extra kernel summations per problem).
 * Arguments otherwise as for the value operations; the method in opts
 * (direct or NFFT) is used for every kernel summation.  Synchronises `stream`.
 *
 * uotk_mmd2_grad: exact derivatives of Eq. (1205) with the Gaussian kernel of
 *   Table tab:0 (eps = ell^2):
 *   d/da_i = 2 sum_j a_j k(x_i,x_j) - 2 sum_j b_j k(x_i,y_j),
 *   d/dx_i = -(4 a_i/eps) [ sum_j a_j (x_i-x_j) k(x_i,x_j) - sum_j b_j (x_i-y_j) k(x_i,y_j) ],
 *   and symmetrically for b, y.  Each (x_i - y_j)-weighted sum is formed as
 *   x'_i t_i - s_i from two kernel summations over shifted coordinates
 *   (origin x_0), so its absolute error is that of the sums times the
 *   diameter of the clouds.
 * uotk_sinkhorn_divergence_grad: derivative of Eq. (586) through the envelope
 *   theorem: each UOT value is the maximum over (beta, gamma) of D of
 *   Eq. (dual_euot), so its derivative is the partial derivative of D at the
 *   duals, evaluated at the duals after max_sweeps sweeps (or tol):
 *   d/da_i = -rho e^{-beta_i/rho} + rho - eps (e^{beta_i/eps} T_i - b(X)),
 *   d/dx_i = 2 a_i e^{beta_i/eps} sum_j b_j e^{gamma_j/eps} (x_i - y_j) k_ij,
 *   T_i = sum_j k_ij b_j e^{gamma_j/eps}, the symmetric problems counted
 *   through both roles, plus +-eps (a(X) - b(X)) on the weights.  Exact at
 *   the fixed point of Alg. 1; after finitely many sweeps it differs from the
 *   derivative of the returned value by the dual residual.
 *   sd, parts as for uotk_sinkhorn_divergence. */
uotk_status uotk_mmd2_grad(uotk_ctx* ctx, void* stream, int d,
                           const float* x, int64_t n, const float* a,
                           const float* y, int64_t m, const float* b,
                           double ell, double* mmd2, double* grad_a, double* grad_x,
                           double* grad_b, double* grad_y, const uotk_sum_opts* opts);
uotk_status uotk_sinkhorn_divergence_grad(uotk_ctx* ctx, void* stream, int d,
                                          const float* x, int64_t n, const float* a,
                                          const float* y, int64_t m, const float* b,
                                          double eps, double rho, int max_sweeps, double tol,
                                          double* sd, double* parts, double* grad_a,
                                          double* grad_x, double* grad_b, double* grad_y,
                                          const uotk_sum_opts* opts);

/* ---- NFFT stages (Sec. 4), exposed for inspection and testing ---------------------
 * uotk_nfft_plan: choose centre, period h, grid, bandwidth and cut-off for
 *   summing from src to tgt with kernel width eps (opts as for
 *   uotk_kernel_sum; method ignored).  Reads the point clouds on the device
 *   (bounding box) and synchronises `stream`.  d in 1..3.
 * uotk_nfft_cells: grid cell of every point, cells = device int32 [n*3]
 *   (x, y, z per point), by the FP32 rule
 *   cell = floor(((p - c) * inv_h + 0.5f) * grid) mod grid, one IEEE rounding
 *   per operation.
 * uotk_nfft_spread: adjoint-NFFT step 1, g_l = sum_i w_i prod_t phi(u_it - l_t/n)
 *   into grid (device FP32 [grid^3], overwritten).
 * uotk_nfft_convolve: grid_out = IFFT( scale_k * FFT(grid_in) ), with
 *   scale_k = b_k / prod_t (n phihat(k_t))^2 on {-N/2..N/2-1}^3 and 0 elsewhere;
 *   forward and inverse FFT unnormalised.  For the Gaussian at grid 128 the
 *   convolution runs as three real circulant passes, one per axis, over the
 *   symmetric band |k_t| <= N/2 - 1 (the k_t = -N/2 planes, whose coefficients
 *   are at the truncation error the plan balances, are left out).  grid_in and
 *   grid_out may alias.
 * uotk_nfft_gather: out_j = sum_l grid_l prod_t phi(u_jt - l_t/n), out = device FP32 [m]. */
uotk_status uotk_nfft_plan(uotk_ctx* ctx, void* stream, int d,
                           const float* src, int64_t n, const float* tgt, int64_t m,
                           double eps, const uotk_sum_opts* opts, uotk_nfft_plan_info* plan);
uotk_status uotk_nfft_cells(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                            const float* pts, int64_t n, int32_t* cells);
uotk_status uotk_nfft_spread(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                             const float* pts, int64_t n, const float* w, float* grid);
uotk_status uotk_nfft_convolve(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                               const float* grid_in, float* grid_out);
uotk_status uotk_nfft_gather(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                             const float* grid, const float* pts, int64_t m, float* out);

#ifdef __cplusplus
}
#endif

#endif /* UOTK_H */
