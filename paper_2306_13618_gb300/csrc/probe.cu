// Unit-throughput probe (uotk_measure_unit_rates): operations per clock per SM
// of the MUFU exp2 and of the FP32 FMA pipe on this GPU, the denominators of
// the ALU rooflines.  One CTA per SM; 16 independent dependency chains per
// thread keep both pipes full; each CTA times itself with clock64().
#include "uotk_internal.cuh"

namespace uotk {

namespace {

constexpr int PROBE_THREADS = 1024;
constexpr int PROBE_ITERS = 4096;
constexpr int PROBE_CHAINS = 16;

template <bool EX2>
__global__ void __launch_bounds__(PROBE_THREADS, 1)
    k_probe(float* __restrict__ sink, long long* __restrict__ cycles, float seed) {
  float v[PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) v[k] = seed * (float)(threadIdx.x + k) * 1e-6f;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < PROBE_ITERS; ++it) {
#pragma unroll
    for (int k = 0; k < PROBE_CHAINS; ++k) {
      if (EX2) v[k] = ex2_approx(v[k]);
      else v[k] = fmaf(v[k], 0.999f, 1e-7f);
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  float s = 0.f;
#pragma unroll
  for (int k = 0; k < PROBE_CHAINS; ++k) s += v[k];
  sink[blockIdx.x * PROBE_THREADS + threadIdx.x] = s;  // keeps the chains live
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

}  // namespace

uotk_status op_measure_unit_rates(uotk_ctx* ctx, cudaStream_t s, double* ex2, double* ffma) {
  const int sms = ctx->num_sms;
  const size_t bytes = sizeof(float) * (size_t)sms * PROBE_THREADS + sizeof(long long) * sms;
  UOTK_TRY(ws_reserve(ctx, bytes));
  Carver cv(ctx->ws);
  float* sink = cv.take<float>((size_t)sms * PROBE_THREADS);
  long long* cyc = cv.take<long long>(sms);
  long long* h = reinterpret_cast<long long*>(ctx->host);  // first 64 pinned doubles
  const int n = sms < 64 ? sms : 64;
  for (int kind = 0; kind < 2; ++kind) {
    for (int rep = 0; rep < 2; ++rep) {  // the first launch warms up clocks and caches
      if (kind == 0) k_probe<true><<<sms, PROBE_THREADS, 0, s>>>(sink, cyc, 1.f);
      else k_probe<false><<<sms, PROBE_THREADS, 0, s>>>(sink, cyc, 1.f);
      UOTK_LAUNCHED(ctx);
    }
    UOTK_CUDA(ctx, cudaMemcpyAsync(h, cyc, sizeof(long long) * n, cudaMemcpyDeviceToHost, s));
    UOTK_CUDA(ctx, cudaStreamSynchronize(s));
    double mean = 0.0;
    for (int i = 0; i < n; ++i) mean += (double)h[i];
    mean /= n;
    const double ops = (double)PROBE_THREADS * PROBE_ITERS * PROBE_CHAINS;
    if (!(mean > 0.0)) return set_error(ctx, UOTK_ERR_INTERNAL, "unit-rate probe: no cycles");
    (kind == 0 ? *ex2 : *ffma) = ops / mean;
  }
  return UOTK_OK;
}

}  // namespace uotk
