// Autotuning of the summation form (the paper picks its NFFT parameters by
// hand: Rem. on NFFT parameters, Sec. 4).  For one summation problem (sources,
// weights, targets, eps) the candidate forms are measured on this GPU:
//   * time: one full kernel summation (the direct forms, whose cost is linear
//     in the number of targets, on a prefix of the targets, scaled up);
//   * error: max_j |s_j - s*_j| / sum |w| over 256 targets spread through the
//     target array, s* their exact sums taken in FP64 by k_ref64;
// and the fastest form whose error meets the target is kept, per (d, n, m,
// eps, target, fixed grid/cut-off, bounding box of the points, timing mode),
// in a small cache of the context.  With per_sum, each form is timed as one
// sum on an engine already built (the NFFT plan and binning, or the direct
// form's packing, excluded): the cost per sum of a solve that builds its
// engine once and sums hundreds of times.  Candidates: the direct FP32 form (always accepted: it
// is the exact sum up to FP32 rounding), the tensor-core forms for d > 3, and
// for d <= 3 the NFFT at grid 64 and 128 (or the caller's grid) with cut-off
// m = 4..8 (or the caller's), where the plan accepts them.
#include <math.h>
#include <string.h>

#include <memory>
#include <vector>

#include "nfft.cuh"

namespace uotk {

uotk_status op_kernel_sum(uotk_ctx* ctx, cudaStream_t s, int d, const float* src, int64_t n,
                          const float* w, const float* tgt, int64_t m, float* out, double eps,
                          const uotk_sum_opts* opts);

namespace {

constexpr int AT_SAMPLES = 256;
constexpr int AT_THREADS = 256;
constexpr int AT_SPLITS = 64;
constexpr int64_t AT_DIRECT_TARGETS = 32768;  // targets of the timed direct-form runs

// Exact (FP64) Gaussian sums at the sampled targets: block (j, split) adds the
// sources split, split + S, .. for target j; the warp and block partial sums
// are combined in a fixed order.
__global__ void __launch_bounds__(AT_THREADS)
    k_ref64(const float* __restrict__ src, const float* __restrict__ w, long long n, int d,
            const float* __restrict__ tgt_s, double neg_inv_eps, double* __restrict__ part) {
  __shared__ double sh[AT_THREADS / 32];
  const int j = blockIdx.x, split = blockIdx.y, S = gridDim.y;
  const float* t = tgt_s + (size_t)j * d;
  double acc = 0.0;
  for (long long i = (long long)split * AT_THREADS + threadIdx.x; i < n;
       i += (long long)S * AT_THREADS) {
    double r2 = 0.0;
    for (int k = 0; k < d; ++k) {
      const double df = (double)src[i * d + k] - (double)t[k];
      r2 += df * df;
    }
    acc += (double)w[i] * exp(r2 * neg_inv_eps);
  }
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < AT_THREADS / 32; ++k) s += sh[k];
    part[(size_t)split * gridDim.x + j] = s;
  }
}

__global__ void k_take_rows(const float* __restrict__ p, int d, const long long* __restrict__ idx,
                            int count, float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count * d; i += gridDim.x * blockDim.x)
    out[i] = p[idx[i / d] * d + i % d];
}

__global__ void k_take(const float* __restrict__ v, const long long* __restrict__ idx, int count,
                       float* __restrict__ out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < count; i += gridDim.x * blockDim.x)
    out[i] = v[idx[i]];
}

__global__ void k_abs_sum(const float* __restrict__ w, long long n, double* __restrict__ out) {
  __shared__ double sh[AT_THREADS / 32];
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += AT_THREADS) acc += fabs((double)w[i]);
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < AT_THREADS / 32; ++k) s += sh[k];
    *out = s;
  }
}

bool same_key(const AutoEntry& e, const AutoEntry& k) {
  return e.valid && e.d == k.d && e.n == k.n && e.m == k.m && e.eps == k.eps &&
         e.target == k.target && e.grid_in == k.grid_in && e.cutoff_in == k.cutoff_in &&
         e.per_sum == k.per_sum && memcmp(e.box, k.box, sizeof(e.box)) == 0;
}

// Scratch of one autotuning run, owned by it (the context's workspace is
// reallocated by the summations being timed).
struct AtScratch {
  char* base = nullptr;
  ~AtScratch() {
    if (base) cudaFree(base);
  }
};

}  // namespace

uotk_status op_autotune_sum(uotk_ctx* ctx, cudaStream_t s, int d, const float* src, int64_t n,
                            const float* w, const float* tgt, int64_t m, double eps,
                            const uotk_sum_opts* in, uotk_sum_opts* out, double* report,
                            bool per_sum) {
  const uotk_sum_opts base = in ? *in : uotk_sum_opts{};
  if (base.kernel != UOTK_KERNEL_GAUSS)
    return set_error(ctx, UOTK_ERR_UNSUPPORTED, "autotune: the Gaussian kernel only");
  if (n < 1 || m < 1) return set_error(ctx, UOTK_ERR_INVALID, "autotune: needs n, m >= 1");
  const double target = base.target_err > 0.0 ? base.target_err : 1e-5;
  // ---- the cache key: sizes, width, target, fixed options, bounding box ----
  AutoEntry key{};
  key.valid = true;
  key.d = d;
  key.n = n;
  key.m = m;
  key.eps = eps;
  key.target = target;
  key.grid_in = base.grid;
  key.cutoff_in = base.cutoff;
  key.per_sum = per_sum;
  if (d <= 3) {
    float lo[3], hi[3];
    UOTK_TRY(nfft_bbox(ctx, s, d, src, n, tgt, m, lo, hi));
    for (int t = 0; t < 3; ++t) {
      key.box[t] = lo[t];
      key.box[3 + t] = hi[t];
    }
  }
  for (int i = 0; i < UOTK_AUTO_CACHE; ++i)
    if (same_key(ctx->autos[i], key)) {
      *out = ctx->autos[i].chosen;
      if (report) memcpy(report, ctx->autos[i].report, sizeof(ctx->autos[i].report));
      return UOTK_OK;
    }

  // ---- scratch: sampled targets, their indices, exact sums, a full output ----
  const int ms = (int)(m < AT_SAMPLES ? m : AT_SAMPLES);
  Carver cv(nullptr);
  float* d_tgt = cv.take<float>((size_t)ms * d);
  long long* d_idx = cv.take<long long>(ms);
  double* d_part = cv.take<double>((size_t)AT_SPLITS * ms);
  double* d_wsum = cv.take<double>(1);
  float* d_samp = cv.take<float>(ms);
  float* d_full = cv.take<float>((size_t)m);
  AtScratch scr;
  if (cudaMalloc(&scr.base, cv.off) != cudaSuccess) {
    cudaGetLastError();
    return set_error(ctx, UOTK_ERR_NOMEM, "autotune: scratch of %zu bytes", cv.off);
  }
  Carver c2(scr.base);
  d_tgt = c2.take<float>((size_t)ms * d);
  d_idx = c2.take<long long>(ms);
  d_part = c2.take<double>((size_t)AT_SPLITS * ms);
  d_wsum = c2.take<double>(1);
  d_samp = c2.take<float>(ms);
  d_full = c2.take<float>((size_t)m);
  std::vector<long long> idx(ms);
  for (int k = 0; k < ms; ++k) idx[k] = (long long)(((double)k + 0.5) * (double)m / ms);
  UOTK_CUDA(ctx, cudaMemcpyAsync(d_idx, idx.data(), sizeof(long long) * ms,
                                 cudaMemcpyHostToDevice, s));
  k_take_rows<<<grid_for(ctx, (int64_t)ms * d, 256, 1), 256, 0, s>>>(tgt, d, d_idx, ms, d_tgt);
  UOTK_LAUNCHED(ctx);
  k_ref64<<<dim3(ms, AT_SPLITS), AT_THREADS, 0, s>>>(src, w, n, d, d_tgt, -1.0 / eps, d_part);
  UOTK_LAUNCHED(ctx);
  k_abs_sum<<<1, AT_THREADS, 0, s>>>(w, n, d_wsum);
  UOTK_LAUNCHED(ctx);
  std::vector<double> part((size_t)AT_SPLITS * ms), exact(ms, 0.0);
  double wsum = 0.0;
  UOTK_CUDA(ctx, cudaMemcpyAsync(part.data(), d_part, sizeof(double) * part.size(),
                                 cudaMemcpyDeviceToHost, s));
  UOTK_CUDA(ctx, cudaMemcpyAsync(&wsum, d_wsum, sizeof(double), cudaMemcpyDeviceToHost, s));
  UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  for (int sp = 0; sp < AT_SPLITS; ++sp)
    for (int k = 0; k < ms; ++k) exact[k] += part[(size_t)sp * ms + k];
  if (!(wsum > 0.0)) wsum = 1.0;

  cudaEvent_t e0, e1;
  UOTK_CUDA(ctx, cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return set_error(ctx, UOTK_ERR_CUDA, "autotune: event creation failed");
  }
  struct Meas {
    uotk_sum_opts o;
    double ms, err;
  };
  std::vector<Meas> meas;
  uotk_status bad = UOTK_OK;
  // error of a form at the sampled targets (d_samp)
  auto sample_err = [&]() -> double {
    std::vector<float> h(ms);
    if (cudaMemcpyAsync(h.data(), d_samp, sizeof(float) * ms, cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
      return INFINITY;
    double e = 0.0;
    for (int k = 0; k < ms; ++k) {
      const double v = fabs((double)h[k] - exact[k]);
      e = isfinite(v) ? fmax(e, v) : INFINITY;
    }
    return e / wsum;
  };
  // one timed call (after an untimed one); returns false if the form is refused
  auto timed = [&](const uotk_sum_opts& o, const float* t, int64_t mt, float* o_out,
                   double* msec) -> bool {
    uotk_status st = op_kernel_sum(ctx, s, d, src, n, w, t, mt, o_out, eps, &o);
    if (st == UOTK_ERR_UNSUPPORTED || st == UOTK_ERR_INVALID) return false;
    if (st != UOTK_OK) {
      bad = st;
      return false;
    }
    if (cudaEventRecord(e0, s) != cudaSuccess) return false;
    st = op_kernel_sum(ctx, s, d, src, n, w, t, mt, o_out, eps, &o);
    if (st != UOTK_OK) {
      bad = st;
      return false;
    }
    float f = 0.f;
    if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
        cudaEventElapsedTime(&f, e0, e1) != cudaSuccess)
      return false;
    *msec = f;
    return true;
  };
  // per_sum: one sum on an engine already built, after an untimed one
  auto timed_sum = [&](const uotk_sum_opts& o, const float* t, int64_t mt,
                       double* msec) -> bool {
    EngineSpec sp{o.method, d, t, mt, nullptr, src, n, w, eps, &o};
    Carver size(nullptr);
    const size_t eb = engine_bytes(ctx, sp);
    size.off = eb;
    size.take<float>(mt > 0 ? mt : 1);
    uotk_status st = ws_reserve(ctx, size.off);
    if (st == UOTK_OK) st = flags_reset(ctx, s);
    Engine* raw = nullptr;
    if (st == UOTK_OK) {
      Carver cv(ctx->ws);
      st = engine_create(ctx, s, sp, cv, &raw);
    }
    std::unique_ptr<Engine> E(raw);
    if (st == UOTK_ERR_UNSUPPORTED || st == UOTK_ERR_INVALID) return false;
    if (st != UOTK_OK) {
      bad = st;
      return false;
    }
    Carver cv(ctx->ws);
    cv.off = eb;
    float* tmp = cv.take<float>(mt > 0 ? mt : 1);
    st = E->plain(s, 1, 0, E->weights(1), tmp);
    if (st == UOTK_OK && cudaEventRecord(e0, s) != cudaSuccess) st = UOTK_ERR_CUDA;
    if (st == UOTK_OK) st = E->plain(s, 1, 0, E->weights(1), tmp);
    float f = 0.f;
    if (st == UOTK_OK &&
        (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
         cudaEventElapsedTime(&f, e0, e1) != cudaSuccess))
      st = UOTK_ERR_CUDA;
    if (st == UOTK_OK) st = flags_check(ctx, s, "autotune");
    if (st != UOTK_OK) {
      bad = st;
      return false;
    }
    *msec = f;
    return true;
  };
  // the direct forms: timed on a prefix of the targets, error on the samples
  std::vector<int> direct_forms = {UOTK_DIRECT};
  if (d > 3) {
    direct_forms.push_back(UOTK_DIRECT_BF16X3);
    direct_forms.push_back(UOTK_DIRECT_BF16);
  }
  const int64_t mt = m < AT_DIRECT_TARGETS ? m : AT_DIRECT_TARGETS;
  for (int meth : direct_forms) {
    if (bad != UOTK_OK) break;
    uotk_sum_opts o = base;
    o.method = meth;
    double t_ms;
    if (!(per_sum ? timed_sum(o, tgt, mt, &t_ms) : timed(o, tgt, mt, d_full, &t_ms))) continue;
    if (op_kernel_sum(ctx, s, d, src, n, w, d_tgt, ms, d_samp, eps, &o) != UOTK_OK) continue;
    meas.push_back({o, t_ms * (double)m / (double)mt, sample_err()});
  }
  // the NFFT: full sums, error at the sampled entries of the full output
  if (d <= 3 && bad == UOTK_OK) {
    std::vector<int> grids = base.grid ? std::vector<int>{base.grid} : std::vector<int>{64, 128};
    std::vector<int> cuts =
        base.cutoff ? std::vector<int>{base.cutoff} : std::vector<int>{4, 5, 6, 7, 8};
    for (int g : grids)
      for (int c : cuts) {
        if (bad != UOTK_OK) break;
        uotk_sum_opts o = base;
        o.method = UOTK_NFFT;
        o.grid = g;
        o.bandwidth = base.grid == g ? base.bandwidth : 0;
        o.cutoff = c;
        o.target_err = target;
        double t_ms;
        if (per_sum) {
          if (!timed_sum(o, tgt, m, &t_ms)) continue;
          const uotk_status st = op_kernel_sum(ctx, s, d, src, n, w, tgt, m, d_full, eps, &o);
          if (st != UOTK_OK) {
            if (st != UOTK_ERR_UNSUPPORTED && st != UOTK_ERR_INVALID) bad = st;
            continue;
          }
        } else if (!timed(o, tgt, m, d_full, &t_ms)) {
          continue;
        }
        k_take<<<grid_for(ctx, ms, 256, 1), 256, 0, s>>>(d_full, d_idx, ms, d_samp);
        UOTK_LAUNCHED(ctx);
        meas.push_back({o, t_ms, sample_err()});
      }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  ctx->err[0] = 0;  // refused candidates left messages
  if (bad != UOTK_OK) return set_error(ctx, bad, "autotune: a candidate failed (status %d)", bad);
  // the fastest form within the target; the direct FP32 form is always admissible
  int best = -1;
  for (size_t i = 0; i < meas.size(); ++i) {
    const bool ok = meas[i].err <= target || meas[i].o.method == UOTK_DIRECT;
    if (ok && (best < 0 || meas[i].ms < meas[best].ms)) best = (int)i;
  }
  if (best < 0) return set_error(ctx, UOTK_ERR_INTERNAL, "autotune: no form measured");
  *out = meas[best].o;
  double direct_ms = 0.0;
  for (const Meas& q : meas)
    if (q.o.method == UOTK_DIRECT) direct_ms = q.ms;
  key.chosen = *out;
  key.report[0] = meas[best].ms;
  key.report[1] = meas[best].err;
  key.report[2] = direct_ms;
  key.report[3] = (double)meas.size();
  key.report[4] = out->method == UOTK_NFFT ? out->grid : 0;
  key.report[5] = out->method == UOTK_NFFT ? out->cutoff : 0;
  key.report[6] = ms;
  key.report[7] = target;
  if (report) memcpy(report, key.report, sizeof(key.report));
  ctx->autos[ctx->auto_next] = key;
  ctx->auto_next = (ctx->auto_next + 1) % UOTK_AUTO_CACHE;
  return UOTK_OK;
}

}  // namespace uotk
