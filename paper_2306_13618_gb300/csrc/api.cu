// Exported C ABI (include/uotk.h): context management, host-side argument
// validation, and dispatch to the operations.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>

#include <new>

#include "engine.cuh"

namespace uotk {

uotk_status op_kernel_sum(uotk_ctx*, cudaStream_t, int, const float*, int64_t, const float*,
                          const float*, int64_t, float*, double, const uotk_sum_opts*);
uotk_status op_uot_sinkhorn(uotk_ctx*, cudaStream_t, int, const float*, int64_t, const float*,
                            const float*, int64_t, const float*, double, double, double, int,
                            double, int, unsigned, double*, double*, int*, double*,
                            const uotk_sum_opts*);
uotk_status op_sinkhorn_divergence(uotk_ctx*, cudaStream_t, int, const float*, int64_t,
                                   const float*, const float*, int64_t, const float*, double,
                                   double, int, double, double*, double*, const uotk_sum_opts*);
uotk_status op_mmd2(uotk_ctx*, cudaStream_t, int, const float*, int64_t, const float*,
                    const float*, int64_t, const float*, double, double*, double*,
                    const uotk_sum_opts*);
uotk_status op_measure_unit_rates(uotk_ctx*, cudaStream_t, double*, double*);
uotk_status op_uot_sinkhorn_batch(uotk_ctx*, cudaStream_t, int, int, const int64_t*,
                                  const float*, const float*, const int64_t*, const float*,
                                  const float*, const double*, const double*, const double*, int,
                                  double, int, double*, double*, int*, double*, const int*, int);
uotk_status op_mmd2_grad(uotk_ctx*, cudaStream_t, int, const float*, int64_t, const float*,
                         const float*, int64_t, const float*, double, double*, double*, double*,
                         double*, double*, const uotk_sum_opts*);
uotk_status op_sinkhorn_divergence_grad(uotk_ctx*, cudaStream_t, int, const float*, int64_t,
                                        const float*, const float*, int64_t, const float*,
                                        double, double, int, double, double*, double*, double*,
                                        double*, double*, double*, const uotk_sum_opts*);
uotk_status op_nfft_plan(uotk_ctx*, cudaStream_t, int, const float*, int64_t, const float*,
                         int64_t, double, const uotk_sum_opts*, uotk_nfft_plan_info*);
uotk_status op_nfft_cells(uotk_ctx*, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                          int64_t, int32_t*);
uotk_status op_nfft_spread(uotk_ctx*, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                           int64_t, const float*, float*);
uotk_status op_nfft_convolve(uotk_ctx*, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                             float*);
uotk_status op_nfft_gather(uotk_ctx*, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                           const float*, int64_t, float*);

uotk_status set_error(uotk_ctx* ctx, uotk_status st, const char* fmt, ...) {
  if (ctx) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
    va_end(ap);
  }
  return st;
}

uotk_status stream_fence(uotk_ctx* ctx, cudaStream_t from, cudaStream_t to, cudaEvent_t ev) {
  UOTK_CUDA(ctx, cudaEventRecord(ev, from));
  UOTK_CUDA(ctx, cudaStreamWaitEvent(to, ev, 0));
  return UOTK_OK;
}

uotk_status ws_reserve(uotk_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_cap) return UOTK_OK;
  if (ctx->ws_limit && bytes > ctx->ws_limit)
    return set_error(ctx, UOTK_ERR_NOMEM, "workspace of %zu bytes needed, above the limit of %zu",
                     bytes, ctx->ws_limit);
  size_t want = bytes + bytes / 8 + (1 << 20);
  if (ctx->ws_limit && want > ctx->ws_limit) want = ctx->ws_limit;
  if (ctx->ws) {
    UOTK_CUDA(ctx, cudaDeviceSynchronize());
    cudaFree(ctx->ws);
    ctx->ws = nullptr;
    ctx->ws_cap = 0;
  }
  if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
    cudaGetLastError();
    ctx->ws = nullptr;
    return set_error(ctx, UOTK_ERR_NOMEM, "workspace allocation of %zu bytes failed", want);
  }
  ctx->ws_cap = want;
  return UOTK_OK;
}

static void prof_fold(uotk_ctx* ctx) {
  uotk_prof& P = ctx->prof;
  if (!P.pending) return;
  cudaEventSynchronize(P.ev[2 * (P.pending - 1) + 1]);
  for (int i = 0; i < P.pending; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, P.ev[2 * i], P.ev[2 * i + 1]) == cudaSuccess) {
      P.ms[P.stage_of[i]] += ms;
      P.counts[P.stage_of[i]]++;
    }
  }
  cudaGetLastError();
  P.pending = 0;
}

int prof_begin(uotk_ctx* ctx, cudaStream_t s, const char* name) {
  uotk_prof& P = ctx->prof;
  if (!P.created) return -1;
  if (P.pending == UOTK_PROF_POOL) prof_fold(ctx);
  int st = -1;
  for (int i = 0; i < P.nstages; ++i)
    if (!strncmp(P.names[i], name, sizeof(P.names[i]) - 1)) { st = i; break; }
  if (st < 0) {
    if (P.nstages == UOTK_PROF_STAGES) return -1;
    st = P.nstages++;
    strncpy(P.names[st], name, sizeof(P.names[st]) - 1);
  }
  const int slot = P.pending;
  P.stage_of[slot] = st;
  cudaEventRecord(P.ev[2 * slot], s);
  return slot;
}

void prof_end(uotk_ctx* ctx, cudaStream_t s, int slot) {
  uotk_prof& P = ctx->prof;
  cudaEventRecord(P.ev[2 * slot + 1], s);
  P.pending = slot + 1;
}

}  // namespace uotk

using namespace uotk;

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

uotk_status check_cloud(uotk_ctx* ctx, const char* what, const float* p, int64_t n, int d) {
  if (n < 0) return set_error(ctx, UOTK_ERR_INVALID, "%s: negative size %lld", what, (long long)n);
  if (n > 0 && !p) return set_error(ctx, UOTK_ERR_INVALID, "%s: null pointer", what);
  if (p && !aligned(p, 4)) return set_error(ctx, UOTK_ERR_INVALID, "%s: not 4-byte aligned", what);
  if (n > (int64_t(1) << 31) - (int64_t(1) << 20))
    return set_error(ctx, UOTK_ERR_UNSUPPORTED, "%s: %lld points exceed the supported 2^31 - 2^20",
                     what, (long long)n);
  (void)d;
  return UOTK_OK;
}

// Kernels other than the Gaussian: in kernel_sum and mmd2 (allowed), and the
// Laplace kernel as the Gibbs kernel of the cost |x - y| in the Sinkhorn solves
// (cost_r1); direct FP32 or NFFT form only.
uotk_status check_kernel(uotk_ctx* ctx, const uotk_sum_opts* opts, bool allowed,
                         bool cost_r1 = false) {
  const int kernel = opts ? opts->kernel : UOTK_KERNEL_GAUSS;
  if (kernel < UOTK_KERNEL_GAUSS || kernel > UOTK_KERNEL_ENERGY)
    return set_error(ctx, UOTK_ERR_INVALID, "unknown kernel %d", kernel);
  if (kernel == UOTK_KERNEL_GAUSS) return UOTK_OK;
  const int method = opts->method;
  const bool ok = allowed || (cost_r1 && kernel == UOTK_KERNEL_LAPLACE);
  if (!ok || (method != UOTK_DIRECT && method != UOTK_NFFT))
    return set_error(ctx, UOTK_ERR_UNSUPPORTED,
                     "kernel %d: only kernel_sum and mmd2 (and the Laplace kernel, cost |x - y|, "
                     "in the Sinkhorn solves), in the direct FP32 or the NFFT form",
                     kernel);
  return UOTK_OK;
}

uotk_status check_common(uotk_ctx* ctx, int d, const uotk_sum_opts* opts) {
  if (d < 1) return set_error(ctx, UOTK_ERR_INVALID, "dimension d = %d < 1", d);
  const int method = opts ? opts->method : UOTK_DIRECT;
  if (method != UOTK_DIRECT && method != UOTK_NFFT && method != UOTK_DIRECT_BF16 &&
      method != UOTK_DIRECT_BF16X3 && method != UOTK_AUTO)
    return set_error(ctx, UOTK_ERR_INVALID, "unknown method %d", method);
  if (method == UOTK_AUTO && opts->kernel != UOTK_KERNEL_GAUSS)
    return set_error(ctx, UOTK_ERR_UNSUPPORTED, "UOTK_AUTO: the Gaussian kernel only");
  if (method != UOTK_NFFT && d > 128)
    return set_error(ctx, UOTK_ERR_UNSUPPORTED, "direct form: d = %d > 128", d);
  if (method == UOTK_NFFT) {
    if (d > 3)
      return set_error(ctx, UOTK_ERR_UNSUPPORTED,
                       "NFFT fast summation is limited to d <= 3 (grid grows like N^d), got d = %d", d);
    const int g = opts->grid ? opts->grid : 128;
    if (g < 16 || g > 256 || (g & (g - 1)))
      return set_error(ctx, UOTK_ERR_INVALID, "NFFT grid %d not a power of two in [16, 256]", g);
    const int N = opts->bandwidth ? opts->bandwidth : g / 2;
    if (N < 4 || N > g || (N & 1))
      return set_error(ctx, UOTK_ERR_INVALID, "NFFT bandwidth %d not even in [4, grid]", N);
    if (opts->cutoff && (opts->cutoff < 2 || opts->cutoff > 8))
      return set_error(ctx, UOTK_ERR_INVALID, "NFFT cut-off %d outside [2, 8]", opts->cutoff);
    if (!(opts->period >= 0.0) || !(opts->target_err >= 0.0))
      return set_error(ctx, UOTK_ERR_INVALID, "NFFT period/target_err must be >= 0");
  }
  return UOTK_OK;
}

// opts naming UOTK_AUTO: replaced by the autotuned form of the sum src -> tgt
// (kept in *store).
uotk_status resolve_auto(uotk_ctx* ctx, cudaStream_t s, int d, const float* src, int64_t n,
                         const float* w, const float* tgt, int64_t m, double eps,
                         const uotk_sum_opts*& opts, uotk_sum_opts* store) {
  if (!opts || opts->method != UOTK_AUTO) return UOTK_OK;
  UOTK_TRY(op_autotune_sum(ctx, s, d, src, n, w, tgt, m, eps, opts, store, nullptr));
  opts = store;
  return UOTK_OK;
}

uotk_status enter(uotk_ctx* ctx) {
  if (!ctx) return UOTK_ERR_INVALID;
  ctx->err[0] = 0;
  UOTK_CUDA(ctx, cudaSetDevice(ctx->device));
  return UOTK_OK;
}

}  // namespace

extern "C" {

uotk_status uotk_create(uotk_ctx** out, int device) {
  if (!out) return UOTK_ERR_INVALID;
  *out = nullptr;
  uotk_ctx* ctx = new (std::nothrow) uotk_ctx();
  if (!ctx) return UOTK_ERR_NOMEM;
  ctx->device = device;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device < 0 || device >= count) {
    cudaGetLastError();
    delete ctx;
    return UOTK_ERR_CUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaDeviceGetAttribute(&ctx->max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin,
                             device) != cudaSuccess) {
    cudaGetLastError();
    delete ctx;
    return UOTK_ERR_CUDA;
  }
  if (cudaMallocHost(reinterpret_cast<void**>(&ctx->host), 128 * sizeof(double)) != cudaSuccess ||
      cudaMalloc(reinterpret_cast<void**>(&ctx->dflags), NUM_FLAGS * sizeof(long long)) !=
          cudaSuccess) {
    cudaGetLastError();
    if (ctx->host) cudaFreeHost(ctx->host);
    delete ctx;
    return UOTK_ERR_NOMEM;
  }
  if (cudaStreamCreateWithFlags(&ctx->gs, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->fence_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->fence_out, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    if (ctx->gs) cudaStreamDestroy(ctx->gs);
    if (ctx->fence_in) cudaEventDestroy(ctx->fence_in);
    cudaFree(ctx->dflags);
    cudaFreeHost(ctx->host);
    delete ctx;
    return UOTK_ERR_CUDA;
  }
  cudaMemset(ctx->dflags, 0, NUM_FLAGS * sizeof(long long));
  cudaDeviceSynchronize();
  *out = ctx;
  return UOTK_OK;
}

void uotk_destroy(uotk_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  cudaDeviceSynchronize();
  if (ctx->ws) cudaFree(ctx->ws);
  if (ctx->dflags) cudaFree(ctx->dflags);
  if (ctx->host) cudaFreeHost(ctx->host);
  if (ctx->prof.created)
    for (int i = 0; i < 2 * UOTK_PROF_POOL; ++i) cudaEventDestroy(ctx->prof.ev[i]);
  if (ctx->gs) cudaStreamDestroy(ctx->gs);
  if (ctx->fence_in) cudaEventDestroy(ctx->fence_in);
  if (ctx->fence_out) cudaEventDestroy(ctx->fence_out);
  delete ctx;
}


const char* uotk_last_error(const uotk_ctx* ctx) { return ctx ? ctx->err : "null context"; }

const char* uotk_status_string(int st) {
  switch (st) {
    case UOTK_OK: return "ok";
    case UOTK_ERR_INVALID: return "invalid argument";
    case UOTK_ERR_NOMEM: return "out of memory";
    case UOTK_ERR_CUDA: return "CUDA error";
    case UOTK_ERR_UNSUPPORTED: return "unsupported";
    case UOTK_ERR_NONFINITE: return "non-finite value";
    case UOTK_ERR_NOT_CONVERGED: return "not converged";
    case UOTK_ERR_TIMEOUT: return "device wait timed out";
    case UOTK_ERR_INTERNAL: return "internal error";
    default: return "unknown status";
  }
}

int64_t uotk_launch_count(const uotk_ctx* ctx) { return ctx ? ctx->launches : 0; }

uotk_status uotk_set_profiling(uotk_ctx* ctx, int enable) {
  UOTK_TRY(enter(ctx));
  uotk_prof& P = ctx->prof;
  if (enable && !P.created) {
    for (int i = 0; i < 2 * UOTK_PROF_POOL; ++i)
      UOTK_CUDA(ctx, cudaEventCreate(&P.ev[i]));
    P.created = true;
  }
  if (!enable) prof_fold(ctx);
  P.on = enable != 0;
  return UOTK_OK;
}

uotk_status uotk_set_workspace_limit(uotk_ctx* ctx, int64_t bytes) {
  if (!ctx) return UOTK_ERR_INVALID;
  if (bytes < 0) return set_error(ctx, UOTK_ERR_INVALID, "workspace limit %lld < 0", (long long)bytes);
  ctx->ws_limit = (size_t)bytes;
  return UOTK_OK;
}

uotk_status uotk_set_wait_timeout_test(uotk_ctx* ctx, int64_t cycles) {
  if (!ctx) return UOTK_ERR_INVALID;
  if (cycles < 0)
    return set_error(ctx, UOTK_ERR_INVALID, "wait time-out test: %lld cycles < 0", (long long)cycles);
  ctx->wait_test = (long long)cycles;
  return UOTK_OK;
}

int uotk_profile_read(uotk_ctx* ctx, char* names, int cap, int64_t* counts, double* ms, int max) {
  if (!ctx) return 0;
  cudaSetDevice(ctx->device);
  prof_fold(ctx);
  uotk_prof& P = ctx->prof;
  int k = P.nstages < max ? P.nstages : max;
  if (names && cap > 0) {
    names[0] = 0;
    int used = 0;
    for (int i = 0; i < k; ++i) {
      int w = snprintf(names + used, cap - used, i ? ";%s" : "%s", P.names[i]);
      if (w < 0 || used + w >= cap) break;
      used += w;
    }
  }
  for (int i = 0; i < k; ++i) {
    if (counts) counts[i] = P.counts[i];
    if (ms) ms[i] = P.ms[i];
  }
  return k;
}

uotk_status uotk_measure_unit_rates(uotk_ctx* ctx, void* stream, double* ex2_per_clk,
                                    double* ffma_per_clk) {
  UOTK_TRY(enter(ctx));
  if (!ex2_per_clk || !ffma_per_clk)
    return set_error(ctx, UOTK_ERR_INVALID, "measure_unit_rates: null output");
  return op_measure_unit_rates(ctx, (cudaStream_t)stream, ex2_per_clk, ffma_per_clk);
}

void uotk_profile_reset(uotk_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  prof_fold(ctx);
  for (int i = 0; i < UOTK_PROF_STAGES; ++i) { ctx->prof.counts[i] = 0; ctx->prof.ms[i] = 0; }
}

uotk_status uotk_kernel_sum(uotk_ctx* ctx, void* stream, int d, const float* src, int64_t n,
                            const float* w, const float* tgt, int64_t m, float* out, double eps,
                            const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_common(ctx, d, opts));
  UOTK_TRY(check_kernel(ctx, opts, true));
  UOTK_TRY(check_cloud(ctx, "src", src, n, d));
  UOTK_TRY(check_cloud(ctx, "w", w, n, 1));
  UOTK_TRY(check_cloud(ctx, "tgt", tgt, m, d));
  UOTK_TRY(check_cloud(ctx, "out", out, m, 1));
  if (!(eps > 0.0) || !isfinite(eps))
    return set_error(ctx, UOTK_ERR_INVALID, "eps must be finite and > 0, got %g", eps);
  if (m == 0) return UOTK_OK;
  uotk_sum_opts chosen;
  if (n > 0)
    UOTK_TRY(resolve_auto(ctx, (cudaStream_t)stream, d, src, n, w, tgt, m, eps, opts, &chosen));
  else if (opts && opts->method == UOTK_AUTO)
    opts = nullptr;  // no sources: zeros whatever the form
  return op_kernel_sum(ctx, (cudaStream_t)stream, d, src, n, w, tgt, m, out, eps, opts);
}

uotk_status uotk_autotune_sum(uotk_ctx* ctx, void* stream, int d, const float* src, int64_t n,
                              const float* w, const float* tgt, int64_t m, double eps,
                              const uotk_sum_opts* in, uotk_sum_opts* out, double* report) {
  UOTK_TRY(enter(ctx));
  if (!out) return set_error(ctx, UOTK_ERR_INVALID, "autotune: out is null");
  if (d < 1 || d > 128) return set_error(ctx, UOTK_ERR_INVALID, "autotune: d = %d not in [1, 128]", d);
  UOTK_TRY(check_cloud(ctx, "src", src, n, d));
  UOTK_TRY(check_cloud(ctx, "w", w, n, 1));
  UOTK_TRY(check_cloud(ctx, "tgt", tgt, m, d));
  if (!(eps > 0.0) || !isfinite(eps))
    return set_error(ctx, UOTK_ERR_INVALID, "eps must be finite and > 0, got %g", eps);
  if (in && !(in->target_err >= 0.0))
    return set_error(ctx, UOTK_ERR_INVALID, "autotune: target_err must be >= 0");
  return op_autotune_sum(ctx, (cudaStream_t)stream, d, src, n, w, tgt, m, eps, in, out, report);
}

uotk_status uotk_uot_sinkhorn(uotk_ctx* ctx, void* stream, int d, const float* x, int64_t n,
                              const float* a, const float* y, int64_t m, const float* b,
                              double eps, double rho1, double rho2, int max_sweeps, double tol,
                              int ref, unsigned flags, double* beta, double* gamma,
                              int* sweeps_done, double* value, const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_common(ctx, d, opts));
  UOTK_TRY(check_kernel(ctx, opts, false, true));
  UOTK_TRY(check_cloud(ctx, "x", x, n, d));
  UOTK_TRY(check_cloud(ctx, "a", a, n, 1));
  UOTK_TRY(check_cloud(ctx, "y", y, m, d));
  UOTK_TRY(check_cloud(ctx, "b", b, m, 1));
  if (n < 1 || m < 1)
    return set_error(ctx, UOTK_ERR_INVALID, "uot_sinkhorn needs n >= 1 and m >= 1");
  if (!beta || !gamma || !aligned(beta, 8) || !aligned(gamma, 8))
    return set_error(ctx, UOTK_ERR_INVALID, "beta/gamma must be 8-byte aligned device arrays");
  if (!(eps > 0.0) || !isfinite(eps) || !(rho1 > 0.0) || !(rho2 > 0.0) || !isfinite(rho1) ||
      !isfinite(rho2))
    return set_error(ctx, UOTK_ERR_INVALID, "eps, rho1, rho2 must be finite and > 0");
  if (max_sweeps < 1) return set_error(ctx, UOTK_ERR_INVALID, "max_sweeps must be >= 1");
  if (ref != UOTK_REF_PRODUCT && ref != UOTK_REF_COUNTING)
    return set_error(ctx, UOTK_ERR_INVALID, "unknown reference measure %d", ref);
  if (!(tol >= 0.0) && !(tol <= 0.0)) return set_error(ctx, UOTK_ERR_INVALID, "tol is NaN");
  if (flags & ~(UOTK_WARM_START | UOTK_LOG_DOMAIN | UOTK_CSTAR_INIT))
    return set_error(ctx, UOTK_ERR_INVALID, "unknown flags 0x%x", flags);
  if ((flags & UOTK_CSTAR_INIT) && ((flags & UOTK_WARM_START) || ref != UOTK_REF_PRODUCT))
    return set_error(ctx, UOTK_ERR_INVALID,
                     "UOTK_CSTAR_INIT needs ref = PRODUCT and no UOTK_WARM_START");
  // UOTK_AUTO: the form of the beta half-step's sum y -> x with the weights b
  uotk_sum_opts chosen;
  UOTK_TRY(resolve_auto(ctx, (cudaStream_t)stream, d, y, m, b, x, n, eps, opts, &chosen));
  return op_uot_sinkhorn(ctx, (cudaStream_t)stream, d, x, n, a, y, m, b, eps, rho1, rho2,
                         max_sweeps, tol, ref, flags, beta, gamma, sweeps_done, value, opts);
}

static uotk_status check_pair(uotk_ctx* ctx, int d, const float* x, int64_t n, const float* a,
                              const float* y, int64_t m, const float* b) {
  UOTK_TRY(check_common(ctx, d, nullptr));
  UOTK_TRY(check_cloud(ctx, "x", x, n, d));
  UOTK_TRY(check_cloud(ctx, "a", a, n, 1));
  UOTK_TRY(check_cloud(ctx, "y", y, m, d));
  UOTK_TRY(check_cloud(ctx, "b", b, m, 1));
  if (n < 1 || m < 1) return set_error(ctx, UOTK_ERR_INVALID, "needs n >= 1 and m >= 1");
  return UOTK_OK;
}

static uotk_status check_cost(uotk_ctx* ctx, int d, int r, const uotk_sum_opts* opts) {
  if (r != 1 && r != 2) return set_error(ctx, UOTK_ERR_INVALID, "cost exponent r = %d not 1 or 2", r);
  const int method = opts ? opts->method : UOTK_DIRECT;
  if (method != UOTK_DIRECT && method != UOTK_NFFT)
    return set_error(ctx, UOTK_ERR_UNSUPPORTED, "mean cost: direct or NFFT form only");
  if (r == 1) {
    uotk_sum_opts o = opts ? *opts : uotk_sum_opts{};
    o.kernel = UOTK_KERNEL_ENERGY;
    UOTK_TRY(check_common(ctx, d, &o));
  }
  return UOTK_OK;
}

uotk_status uotk_mean_cost(uotk_ctx* ctx, void* stream, int d, const float* x, int64_t n,
                           const float* a, const float* y, int64_t m, const float* b, int r,
                           double* out, const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_pair(ctx, d, x, n, a, y, m, b));
  UOTK_TRY(check_cost(ctx, d, r, opts));
  if (!out) return set_error(ctx, UOTK_ERR_INVALID, "mean_cost: null output");
  return op_mean_cost(ctx, (cudaStream_t)stream, d, x, n, a, y, m, b, r,
                      opts ? opts->method : UOTK_DIRECT, out);
}

uotk_status uotk_cstar(uotk_ctx* ctx, void* stream, int d, const float* x, int64_t n,
                       const float* a, const float* y, int64_t m, const float* b, double eps,
                       double rho1, double rho2, int r, double* out,
                       const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_pair(ctx, d, x, n, a, y, m, b));
  UOTK_TRY(check_cost(ctx, d, r, opts));
  if (!(eps > 0.0) || !isfinite(eps) || !(rho1 > 0.0) || !(rho2 > 0.0) || !isfinite(rho1) ||
      !isfinite(rho2))
    return set_error(ctx, UOTK_ERR_INVALID, "eps, rho1, rho2 must be finite and > 0");
  if (!out) return set_error(ctx, UOTK_ERR_INVALID, "cstar: null output");
  return op_cstar(ctx, (cudaStream_t)stream, d, x, n, a, y, m, b, eps, rho1, rho2, r,
                  opts ? opts->method : UOTK_DIRECT, out);
}

uotk_status uotk_uot_sinkhorn_scaled(uotk_ctx* ctx, void* stream, int d, const float* x,
                                     int64_t n, const float* a, const float* y, int64_t m,
                                     const float* b, const double* eps_schedule, int stages,
                                     double rho1, double rho2, int max_sweeps_per_stage,
                                     double tol, int ref, unsigned flags, double* beta,
                                     double* gamma, int* sweeps_per_stage, double* value,
                                     const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  if (stages < 1 || !eps_schedule)
    return set_error(ctx, UOTK_ERR_INVALID, "uot_sinkhorn_scaled: empty schedule");
  if (flags & ~UOTK_LOG_DOMAIN)
    return set_error(ctx, UOTK_ERR_INVALID, "uot_sinkhorn_scaled: flags 0x%x", flags);
  for (int k = 0; k < stages; ++k)
    if (!(eps_schedule[k] > 0.0) || !isfinite(eps_schedule[k]))
      return set_error(ctx, UOTK_ERR_INVALID, "uot_sinkhorn_scaled: eps[%d] not finite > 0", k);
  uotk_status st = UOTK_OK;
  for (int k = 0; k < stages; ++k) {
    int sw = 0;
    // stage k > 0 starts from the previous stage's gamma
    st = uotk_uot_sinkhorn(ctx, stream, d, x, n, a, y, m, b, eps_schedule[k], rho1, rho2,
                           max_sweeps_per_stage, tol, ref,
                           flags | (k > 0 ? UOTK_WARM_START : 0u), beta, gamma, &sw,
                           k == stages - 1 ? value : nullptr, opts);
    if (sweeps_per_stage) sweeps_per_stage[k] = sw;
    if (st != UOTK_OK && st != UOTK_ERR_NOT_CONVERGED) return st;
  }
  return st;
}

uotk_status uotk_uot_sinkhorn_batch(uotk_ctx* ctx, void* stream, int d, int npairs,
                                    const int64_t* x_off, const float* x, const float* a,
                                    const int64_t* y_off, const float* y, const float* b,
                                    const double* eps, const double* rho1, const double* rho2,
                                    int max_sweeps, double tol, int ref, double* beta,
                                    double* gamma, int* sweeps_done, double* values,
                                    const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_common(ctx, d, opts));
  UOTK_TRY(check_kernel(ctx, opts, false));
  const int method = opts ? opts->method : UOTK_DIRECT;
  if (method != UOTK_DIRECT && method != UOTK_AUTO)
    return set_error(ctx, UOTK_ERR_UNSUPPORTED,
                     "uot_sinkhorn_batch: the direct FP32 form or UOTK_AUTO only");
  if (d > 3) return set_error(ctx, UOTK_ERR_UNSUPPORTED, "uot_sinkhorn_batch: d = %d > 3", d);
  if (npairs < 1 || npairs > (1 << 20))
    return set_error(ctx, UOTK_ERR_INVALID, "uot_sinkhorn_batch: npairs %d outside [1, 2^20]",
                     npairs);
  if (!x_off || !y_off || !eps || !rho1 || !rho2)
    return set_error(ctx, UOTK_ERR_INVALID, "uot_sinkhorn_batch: null host array");
  if (x_off[0] < 0 || y_off[0] < 0)
    return set_error(ctx, UOTK_ERR_INVALID, "uot_sinkhorn_batch: negative offset");
  for (int p = 0; p < npairs; ++p) {
    if (x_off[p + 1] <= x_off[p] || y_off[p + 1] <= y_off[p])
      return set_error(ctx, UOTK_ERR_INVALID,
                       "uot_sinkhorn_batch: pair %d has an empty side or decreasing offsets", p);
    if (!(eps[p] > 0.0) || !isfinite(eps[p]) || !(rho1[p] > 0.0) || !isfinite(rho1[p]) ||
        !(rho2[p] > 0.0) || !isfinite(rho2[p]))
      return set_error(ctx, UOTK_ERR_INVALID,
                       "uot_sinkhorn_batch: pair %d: eps and rho must be finite and > 0", p);
  }
  UOTK_TRY(check_cloud(ctx, "x", x, x_off[npairs], d));
  UOTK_TRY(check_cloud(ctx, "a", a, x_off[npairs], 1));
  UOTK_TRY(check_cloud(ctx, "y", y, y_off[npairs], d));
  UOTK_TRY(check_cloud(ctx, "b", b, y_off[npairs], 1));
  if (!beta || !gamma || !aligned(beta, 8) || !aligned(gamma, 8))
    return set_error(ctx, UOTK_ERR_INVALID, "beta/gamma null or not 8-byte aligned");
  if (max_sweeps < 1) return set_error(ctx, UOTK_ERR_INVALID, "max_sweeps must be >= 1");
  if (ref != UOTK_REF_PRODUCT && ref != UOTK_REF_COUNTING)
    return set_error(ctx, UOTK_ERR_INVALID, "unknown reference measure %d", ref);
  if (!(tol >= 0.0) && !(tol <= 0.0)) return set_error(ctx, UOTK_ERR_INVALID, "tol is NaN");
  cudaStream_t s = (cudaStream_t)stream;
  ctx->batch_forms.assign(npairs, UOTK_DIRECT);
  if (method == UOTK_DIRECT)
    return op_uot_sinkhorn_batch(ctx, s, d, npairs, x_off, x, a, y_off, y, b, eps, rho1, rho2,
                                 max_sweeps, tol, ref, beta, gamma, sweeps_done, values, nullptr, 0);
  // UOTK_AUTO.  Every pair with at least BATCH_AUTO_MIN points on both sides has
  // its form measured by the autotuner, per sum on a built engine (the plan is
  // paid once per solve): the beta half-step's sum y -> x within
  // opts->target_err.  Pairs whose fastest form is the NFFT are solved one by
  // one by the NFFT solver; the others together by the grouped direct batch,
  // first (it clears gamma of its pairs only).  Start, stopping rule, cap and
  // outputs per pair are those of the batch.
  constexpr int64_t BATCH_AUTO_MIN = 16384;
  uotk_sum_opts base = *opts;
  base.method = UOTK_DIRECT;
  std::vector<int> direct_pairs, nfft_pairs;
  std::vector<uotk_sum_opts> form(npairs);
  for (int p = 0; p < npairs; ++p) {
    const int64_t np_ = x_off[p + 1] - x_off[p], mp = y_off[p + 1] - y_off[p];
    if (np_ >= BATCH_AUTO_MIN && mp >= BATCH_AUTO_MIN) {
      uotk_sum_opts chosen{};
      UOTK_TRY(op_autotune_sum(ctx, s, d, y + y_off[p] * d, mp, b + y_off[p], x + x_off[p] * d,
                               np_, eps[p], &base, &chosen, nullptr, true));
      if (chosen.method == UOTK_NFFT) {
        form[p] = chosen;
        nfft_pairs.push_back(p);
        ctx->batch_forms[p] = UOTK_NFFT;
        continue;
      }
    }
    direct_pairs.push_back(p);
  }
  uotk_status st_direct = UOTK_OK;
  if (!direct_pairs.empty()) {
    st_direct = op_uot_sinkhorn_batch(ctx, s, d, npairs, x_off, x, a, y_off, y, b, eps, rho1,
                                      rho2, max_sweeps, tol, ref, beta, gamma, sweeps_done,
                                      values, direct_pairs.data(), (int)direct_pairs.size());
    if (st_direct != UOTK_OK && st_direct != UOTK_ERR_NOT_CONVERGED) return st_direct;
  }
  int nfft_open = 0;
  for (int p : nfft_pairs) {
    const int64_t np_ = x_off[p + 1] - x_off[p], mp = y_off[p + 1] - y_off[p];
    int sw = 0;
    double val = 0.0;
    const uotk_status st = op_uot_sinkhorn(ctx, s, d, x + x_off[p] * d, np_, a + x_off[p],
                                           y + y_off[p] * d, mp, b + y_off[p], eps[p], rho1[p],
                                           rho2[p], max_sweeps, tol, ref, 0u, beta + x_off[p],
                                           gamma + y_off[p], &sw, &val, &form[p]);
    if (st == UOTK_ERR_NOT_CONVERGED) ++nfft_open;
    else if (st != UOTK_OK) return st;
    if (sweeps_done) sweeps_done[p] = sw;
    if (values) values[p] = val;
  }
  if (st_direct == UOTK_ERR_NOT_CONVERGED || nfft_open > 0)
    return set_error(ctx, UOTK_ERR_NOT_CONVERGED,
                     "uot_sinkhorn_batch: pairs did not reach tol %g in %d sweeps (%d of %zu "
                     "NFFT-form pairs; direct-form pairs: %s)",
                     tol, max_sweeps, nfft_open, nfft_pairs.size(),
                     st_direct == UOTK_ERR_NOT_CONVERGED ? "some" : "none");
  return UOTK_OK;
}

uotk_status uotk_batch_forms(uotk_ctx* ctx, int npairs, int32_t* forms) {
  UOTK_TRY(enter(ctx));
  if (!forms || npairs != (int)ctx->batch_forms.size())
    return set_error(ctx, UOTK_ERR_INVALID,
                     "batch_forms: forms null or npairs %d != the last batch's %zu", npairs,
                     ctx->batch_forms.size());
  for (int p = 0; p < npairs; ++p) forms[p] = ctx->batch_forms[p];
  return UOTK_OK;
}

uotk_status uotk_sinkhorn_divergence(uotk_ctx* ctx, void* stream, int d, const float* x,
                                     int64_t n, const float* a, const float* y, int64_t m,
                                     const float* b, double eps, double rho, int max_sweeps,
                                     double tol, double* sd, double* parts,
                                     const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_common(ctx, d, opts));
  UOTK_TRY(check_kernel(ctx, opts, false, true));
  UOTK_TRY(check_cloud(ctx, "x", x, n, d));
  UOTK_TRY(check_cloud(ctx, "a", a, n, 1));
  UOTK_TRY(check_cloud(ctx, "y", y, m, d));
  UOTK_TRY(check_cloud(ctx, "b", b, m, 1));
  if (n < 1 || m < 1)
    return set_error(ctx, UOTK_ERR_INVALID, "sinkhorn_divergence needs n >= 1 and m >= 1");
  if (!sd) return set_error(ctx, UOTK_ERR_INVALID, "sd is null");
  if (!(eps > 0.0) || !isfinite(eps) || !(rho > 0.0) || !isfinite(rho))
    return set_error(ctx, UOTK_ERR_INVALID, "eps and rho must be finite and > 0");
  if (max_sweeps < 1) return set_error(ctx, UOTK_ERR_INVALID, "max_sweeps must be >= 1");
  uotk_sum_opts chosen;
  UOTK_TRY(resolve_auto(ctx, (cudaStream_t)stream, d, y, m, b, x, n, eps, opts, &chosen));
  return op_sinkhorn_divergence(ctx, (cudaStream_t)stream, d, x, n, a, y, m, b, eps, rho,
                                max_sweeps, tol, sd, parts, opts);
}

uotk_status uotk_mmd2(uotk_ctx* ctx, void* stream, int d, const float* x, int64_t n,
                      const float* a, const float* y, int64_t m, const float* b, double ell,
                      double* mmd2, double* parts, const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_common(ctx, d, opts));
  UOTK_TRY(check_kernel(ctx, opts, true));
  UOTK_TRY(check_cloud(ctx, "x", x, n, d));
  UOTK_TRY(check_cloud(ctx, "a", a, n, 1));
  UOTK_TRY(check_cloud(ctx, "y", y, m, d));
  UOTK_TRY(check_cloud(ctx, "b", b, m, 1));
  if (n < 1 || m < 1) return set_error(ctx, UOTK_ERR_INVALID, "mmd2 needs n >= 1 and m >= 1");
  if (!mmd2) return set_error(ctx, UOTK_ERR_INVALID, "mmd2 is null");
  if (!(ell > 0.0) || !isfinite(ell))
    return set_error(ctx, UOTK_ERR_INVALID, "ell must be finite and > 0");
  uotk_sum_opts chosen;
  UOTK_TRY(resolve_auto(ctx, (cudaStream_t)stream, d, y, m, b, x, n, ell * ell, opts, &chosen));
  return op_mmd2(ctx, (cudaStream_t)stream, d, x, n, a, y, m, b, ell, mmd2, parts, opts);
}

static uotk_status check_grad_outputs(uotk_ctx* ctx, int d, int64_t n, int64_t m, double* ga,
                                      double* gx, double* gb, double* gy) {
  (void)d;
  (void)n;
  (void)m;
  const double* p[4] = {ga, gx, gb, gy};
  const char* name[4] = {"grad_a", "grad_x", "grad_b", "grad_y"};
  for (int k = 0; k < 4; ++k)
    if (p[k] && !aligned(p[k], 8))
      return set_error(ctx, UOTK_ERR_INVALID, "%s: not 8-byte aligned", name[k]);
  return UOTK_OK;
}

uotk_status uotk_mmd2_grad(uotk_ctx* ctx, void* stream, int d, const float* x, int64_t n,
                           const float* a, const float* y, int64_t m, const float* b, double ell,
                           double* mmd2, double* grad_a, double* grad_x, double* grad_b,
                           double* grad_y, const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_common(ctx, d, opts));
  UOTK_TRY(check_kernel(ctx, opts, false));
  UOTK_TRY(check_cloud(ctx, "x", x, n, d));
  UOTK_TRY(check_cloud(ctx, "a", a, n, 1));
  UOTK_TRY(check_cloud(ctx, "y", y, m, d));
  UOTK_TRY(check_cloud(ctx, "b", b, m, 1));
  if (n < 1 || m < 1) return set_error(ctx, UOTK_ERR_INVALID, "mmd2_grad needs n >= 1 and m >= 1");
  UOTK_TRY(check_grad_outputs(ctx, d, n, m, grad_a, grad_x, grad_b, grad_y));
  if (!(ell > 0.0) || !isfinite(ell))
    return set_error(ctx, UOTK_ERR_INVALID, "ell must be finite and > 0");
  uotk_sum_opts chosen;
  UOTK_TRY(resolve_auto(ctx, (cudaStream_t)stream, d, y, m, b, x, n, ell * ell, opts, &chosen));
  return op_mmd2_grad(ctx, (cudaStream_t)stream, d, x, n, a, y, m, b, ell, mmd2, grad_a, grad_x,
                      grad_b, grad_y, opts);
}

uotk_status uotk_sinkhorn_divergence_grad(uotk_ctx* ctx, void* stream, int d, const float* x,
                                          int64_t n, const float* a, const float* y, int64_t m,
                                          const float* b, double eps, double rho, int max_sweeps,
                                          double tol, double* sd, double* parts, double* grad_a,
                                          double* grad_x, double* grad_b, double* grad_y,
                                          const uotk_sum_opts* opts) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_common(ctx, d, opts));
  UOTK_TRY(check_kernel(ctx, opts, false));
  UOTK_TRY(check_cloud(ctx, "x", x, n, d));
  UOTK_TRY(check_cloud(ctx, "a", a, n, 1));
  UOTK_TRY(check_cloud(ctx, "y", y, m, d));
  UOTK_TRY(check_cloud(ctx, "b", b, m, 1));
  if (n < 1 || m < 1)
    return set_error(ctx, UOTK_ERR_INVALID, "sinkhorn_divergence_grad needs n >= 1 and m >= 1");
  UOTK_TRY(check_grad_outputs(ctx, d, n, m, grad_a, grad_x, grad_b, grad_y));
  if (!(eps > 0.0) || !isfinite(eps) || !(rho > 0.0) || !isfinite(rho))
    return set_error(ctx, UOTK_ERR_INVALID, "eps and rho must be finite and > 0");
  if (max_sweeps < 1) return set_error(ctx, UOTK_ERR_INVALID, "max_sweeps must be >= 1");
  if (!(tol >= 0.0) && !(tol <= 0.0)) return set_error(ctx, UOTK_ERR_INVALID, "tol is NaN");
  uotk_sum_opts chosen;
  UOTK_TRY(resolve_auto(ctx, (cudaStream_t)stream, d, y, m, b, x, n, eps, opts, &chosen));
  return op_sinkhorn_divergence_grad(ctx, (cudaStream_t)stream, d, x, n, a, y, m, b, eps, rho,
                                     max_sweeps, tol, sd, parts, grad_a, grad_x, grad_b, grad_y,
                                     opts);
}

uotk_status uotk_nfft_plan(uotk_ctx* ctx, void* stream, int d, const float* src, int64_t n,
                           const float* tgt, int64_t m, double eps, const uotk_sum_opts* opts,
                           uotk_nfft_plan_info* plan) {
  UOTK_TRY(enter(ctx));
  uotk_sum_opts o = opts ? *opts : uotk_sum_opts{};
  o.method = UOTK_NFFT;
  UOTK_TRY(check_common(ctx, d, &o));
  UOTK_TRY(check_cloud(ctx, "src", src, n, d));
  UOTK_TRY(check_cloud(ctx, "tgt", tgt, m, d));
  if (!plan) return set_error(ctx, UOTK_ERR_INVALID, "plan is null");
  if (!(eps > 0.0) || !isfinite(eps))
    return set_error(ctx, UOTK_ERR_INVALID, "eps must be finite and > 0");
  return op_nfft_plan(ctx, (cudaStream_t)stream, d, src, n, tgt, m, eps, &o, plan);
}

static uotk_status check_plan(uotk_ctx* ctx, const uotk_nfft_plan_info* p) {
  if (!p) return set_error(ctx, UOTK_ERR_INVALID, "plan is null");
  if (p->d < 1 || p->d > 3 || p->grid < 16 || p->grid > 256 || (p->grid & (p->grid - 1)) ||
      p->bandwidth < 4 || p->bandwidth > p->grid || (p->bandwidth & 1) || p->cutoff < 2 ||
      p->cutoff > 8 || 2 * p->cutoff > p->grid || !(p->h > 0.0) || !(p->inv_h > 0.f) ||
      !(p->eps > 0.0))
    return set_error(ctx, UOTK_ERR_INVALID, "inconsistent NFFT plan");
  return UOTK_OK;
}

uotk_status uotk_nfft_cells(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                            const float* pts, int64_t n, int32_t* cells) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_plan(ctx, plan));
  UOTK_TRY(check_cloud(ctx, "pts", pts, n, plan->d));
  if (n > 0 && !cells) return set_error(ctx, UOTK_ERR_INVALID, "cells is null");
  return op_nfft_cells(ctx, (cudaStream_t)stream, plan, pts, n, cells);
}

uotk_status uotk_nfft_spread(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                             const float* pts, int64_t n, const float* w, float* grid) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_plan(ctx, plan));
  UOTK_TRY(check_cloud(ctx, "pts", pts, n, plan->d));
  UOTK_TRY(check_cloud(ctx, "w", w, n, 1));
  if (!grid || !aligned(grid, 16)) return set_error(ctx, UOTK_ERR_INVALID, "grid null or unaligned");
  return op_nfft_spread(ctx, (cudaStream_t)stream, plan, pts, n, w, grid);
}

uotk_status uotk_nfft_convolve(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                               const float* grid_in, float* grid_out) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_plan(ctx, plan));
  if (!grid_in || !grid_out || !aligned(grid_in, 16) || !aligned(grid_out, 16))
    return set_error(ctx, UOTK_ERR_INVALID, "grid null or unaligned");
  return op_nfft_convolve(ctx, (cudaStream_t)stream, plan, grid_in, grid_out);
}

uotk_status uotk_nfft_gather(uotk_ctx* ctx, void* stream, const uotk_nfft_plan_info* plan,
                             const float* grid, const float* pts, int64_t m, float* out) {
  UOTK_TRY(enter(ctx));
  UOTK_TRY(check_plan(ctx, plan));
  UOTK_TRY(check_cloud(ctx, "pts", pts, m, plan->d));
  UOTK_TRY(check_cloud(ctx, "out", out, m, 1));
  if (!grid || !aligned(grid, 16)) return set_error(ctx, UOTK_ERR_INVALID, "grid null or unaligned");
  return op_nfft_gather(ctx, (cudaStream_t)stream, plan, grid, pts, m, out);
}

}  // extern "C"
