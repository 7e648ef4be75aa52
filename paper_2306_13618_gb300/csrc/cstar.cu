// The mean cost <mu (x) nu | d^r> and the constant c*_{r;eta;lambda} of
// Eq. (561) (Prop. prop:536): the best plan of the form c mu (x) nu for
// Eq. (W4), whose objective bounds the regularised UOT value from above
// (Remark on upper bounds), and the initial value gamma^0 = c* 1 of the
// Remark on the initialisation of Sinkhorn's algorithm.
//
// r = 2 needs no kernel summation: about any centre o,
//   <mu (x) nu | d^2> = nu(X) sum_i mu_i |x_i - o|^2 + mu(X) sum_j nu_j |y_j - o|^2
//                       - 2 (sum_i mu_i (x_i - o)) . (sum_j nu_j (y_j - o)),
// first and second moments in FP64, O((n + m) d).  The centre is x_0, so the
// moments are of the size of the clouds' joint diameter and the identity
// cancels no more than the cost itself.
// r = 1 is the energy kernel's cross term (d = -k_e, Sec. 4.4): one direct
// kernel summation with k_e and an FP64 dot product.
#include <math.h>

#include <memory>

#include "solver.cuh"

namespace uotk {

namespace {

constexpr int MOM_THREADS = 256;
constexpr int MOM_WARPS = MOM_THREADS / 32;
constexpr int MOM_DIMS = 128;            // = the largest d; 4 per lane
constexpr int MOM_WIDTH = 2 + MOM_DIMS;  // {sum w, sum w |p-o|^2, sum w (p-o)_k}

// Block partials of one cloud p (count points, row-major FP32 [count][d]) with
// weights w about the centre o (d FP32 values):
//   part[block][0] = sum w_i, [1] = sum w_i |p_i - o|^2, [2 + k] = sum w_i (p_ik - o_k).
// One warp per point (lane l holds dimensions l, l + 32, l + 64, l + 96);
// negative or non-finite weights and non-finite coordinates are counted in
// the context's flag slots.
__global__ void __launch_bounds__(MOM_THREADS)
k_moments(const float* __restrict__ p, long long count, int d, const float* __restrict__ w,
          const float* __restrict__ o, double* __restrict__ part, long long* __restrict__ flags) {
  __shared__ double sh[MOM_WARPS][MOM_WIDTH];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float ok[4];
  double s1[4] = {0.0, 0.0, 0.0, 0.0};
  double s0 = 0.0, s2 = 0.0;
  long long bad = 0, neg = 0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int k = lane + 32 * q;
    ok[q] = k < d ? o[k] : 0.f;
  }
  for (long long i = (long long)blockIdx.x * MOM_WARPS + warp; i < count;
       i += (long long)gridDim.x * MOM_WARPS) {
    const float wf = w[i];
    if (lane == 0) {
      if (!isfinite(wf)) ++bad;
      else if (wf < 0.f) ++neg;
    }
    const double wi = isfinite(wf) ? (double)wf : 0.0;
    s0 += wi;
    const float* pi = p + i * d;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int k = lane + 32 * q;
      if (k < d) {
        const float v = pi[k];
        if (!isfinite(v)) {
          ++bad;
          continue;
        }
        const double dv = (double)v - (double)ok[q];
        s1[q] += wi * dv;
        s2 += wi * dv * dv;
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s2 += __shfl_xor_sync(0xffffffffu, s2, off);
  if (lane == 0) {
    sh[warp][0] = s0;
    sh[warp][1] = s2;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) sh[warp][2 + lane + 32 * q] = s1[q];
  if (bad) atomicAdd(reinterpret_cast<unsigned long long*>(flags + FLAG_NONFINITE),
                     (unsigned long long)bad);
  if (neg) atomicAdd(reinterpret_cast<unsigned long long*>(flags + FLAG_NEG_WEIGHT),
                     (unsigned long long)neg);
  __syncthreads();
  for (int t = threadIdx.x; t < 2 + d; t += MOM_THREADS) {
    double acc = 0.0;
    for (int q = 0; q < MOM_WARPS; ++q) acc += sh[q][t];
    part[(long long)blockIdx.x * MOM_WIDTH + t] = acc;
  }
}

// Column sums of both clouds' partials (block order: deterministic), then
//   out = {<mu (x) nu|d^2>, mu(X), nu(X)}.
__global__ void __launch_bounds__(MOM_THREADS)
k_moments_final(const double* __restrict__ px, int bx, const double* __restrict__ py, int by,
                int d, double* __restrict__ out) {
  __shared__ double cx[MOM_WIDTH], cy[MOM_WIDTH];
  for (int t = threadIdx.x; t < 2 + d; t += MOM_THREADS) {
    double a = 0.0, b = 0.0;
    for (int q = 0; q < bx; ++q) a += px[(long long)q * MOM_WIDTH + t];
    for (int q = 0; q < by; ++q) b += py[(long long)q * MOM_WIDTH + t];
    cx[t] = a;
    cy[t] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double cross = 0.0;
    for (int k = 0; k < d; ++k) cross += cx[2 + k] * cy[2 + k];
    out[0] = cy[0] * cx[1] + cx[0] * cy[1] - 2.0 * cross;
    out[1] = cx[0];
    out[2] = cy[0];
  }
}

__global__ void k_fill(double* __restrict__ v, long long count, double value) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = value;
}

int moment_blocks(uotk_ctx* ctx, long long count) {
  const long long want = (count + MOM_WARPS - 1) / MOM_WARPS;
  const long long cap = 2LL * ctx->num_sms;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

// <mu (x) nu|d^2>, mu(X), nu(X) into host[0..3) (r = 2, moments).
uotk_status cost2(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                  const float* a, const float* y, int64_t m, const float* b, double* host) {
  const int bx = moment_blocks(ctx, n), by = moment_blocks(ctx, m);
  Carver size(nullptr);
  size.take<double>((size_t)(bx + by) * MOM_WIDTH + 4);
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  double* px = cv.take<double>((size_t)(bx + by) * MOM_WIDTH + 4);
  double* py = px + (size_t)bx * MOM_WIDTH;
  double* out = py + (size_t)by * MOM_WIDTH;
  {
    UOTK_PROF(ctx, s, "moments");
    k_moments<<<bx, MOM_THREADS, 0, s>>>(x, n, d, a, x, px, ctx->dflags);
    UOTK_LAUNCHED(ctx);
    k_moments<<<by, MOM_THREADS, 0, s>>>(y, m, d, b, x, py, ctx->dflags);
    UOTK_LAUNCHED(ctx);
    k_moments_final<<<1, MOM_THREADS, 0, s>>>(px, bx, py, by, d, out);
    UOTK_LAUNCHED(ctx);
  }
  UOTK_CUDA(ctx, cudaMemcpyAsync(host, out, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  return flags_check(ctx, s, "mean_cost");
}

// -<mu (x) nu|d>, mu(X), nu(X) into host[0..3) (r = 1, energy kernel).
uotk_status cost1(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                  const float* a, const float* y, int64_t m, const float* b, int method,
                  double* host) {
  uotk_sum_opts o{};
  o.method = method;
  o.kernel = UOTK_KERNEL_ENERGY;
  EngineSpec sp{method, d, x, n, a, y, m, b, 1.0, &o};
  Carver size(nullptr);
  size.off = engine_bytes(ctx, sp);
  size.take<float>(n + 4);
  Reducer R;
  carve_reducer(ctx, size, R);
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  Engine* raw = nullptr;
  UOTK_TRY(engine_create(ctx, s, sp, cv, &raw));
  std::unique_ptr<Engine> E(raw);
  cv.off = engine_bytes(ctx, sp);
  float* t = cv.take<float>(n + 4);
  carve_reducer(ctx, cv, R);
  UOTK_TRY(E->plain(s, 1, 0, E->weights(1), t));  // t_i = -sum_j nu_j |x_i - y_j|
  SumTerms T{};
  T.count = 3;
  T.k[0] = SumTerm{2, n, E->weights(0), nullptr, t, 1.0, 1.0, 0};
  T.k[1] = SumTerm{1, n, E->weights(0), nullptr, nullptr, 1.0, 1.0, 0};
  T.k[2] = SumTerm{1, m, E->weights(1), nullptr, nullptr, 1.0, 1.0, 0};
  UOTK_TRY(run_sums(ctx, s, R, T, host));
  return flags_check(ctx, s, "mean_cost");
}

}  // namespace

uotk_status op_mean_cost(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                         const float* a, const float* y, int64_t m, const float* b, int r,
                         int method, double* out) {
  double* h = ctx->host + 72;
  if (r == 2) {
    UOTK_TRY(cost2(ctx, s, d, x, n, a, y, m, b, h));
  } else {
    UOTK_TRY(cost1(ctx, s, d, x, n, a, y, m, b, method, h));
    h[0] = -h[0];
  }
  out[0] = h[0];
  out[1] = h[1];
  out[2] = h[2];
  return UOTK_OK;
}

// c* of Eq. (561) for the cost |x - y|^r (r = 1, 2), lambda = 1/eps, and the
// Eq. (W4) objective at c* mu (x) nu: cost c* C + eps m1 m2 (c* log c* - c* + 1)
// plus the two KL terms of the marginals c* m2 mu and c* m1 nu.
uotk_status op_cstar(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                     const float* a, const float* y, int64_t m, const float* b, double eps,
                     double rho1, double rho2, int r, int method, double* out) {
  double mc[3];
  UOTK_TRY(op_mean_cost(ctx, s, d, x, n, a, y, m, b, r, method, mc));
  const double C = mc[0], m1 = mc[1], m2 = mc[2];
  if (!(m1 > 0.0) || !(m2 > 0.0))
    return set_error(ctx, UOTK_ERR_INVALID, "cstar: a measure has zero mass");
  const double den = rho1 + rho2 + eps;
  const double lc = -(C / (m1 * m2) + rho1 * log(m2) + rho2 * log(m1)) / den;
  const double c = exp(lc);
  const double obj = c * C + eps * m1 * m2 * (c * lc - c + 1.0) +
                     rho1 * m1 * (c * m2 * (lc + log(m2)) - c * m2 + 1.0) +
                     rho2 * m2 * (c * m1 * (lc + log(m1)) - c * m1 + 1.0);
  out[0] = c;
  out[1] = obj;
  out[2] = C;
  return UOTK_OK;
}

uotk_status fill_f64(uotk_ctx* ctx, cudaStream_t s, double* v, int64_t count, double value) {
  const long long want = (count + 255) / 256;
  const int blocks = (int)(want < 1 ? 1 : (want < 4LL * ctx->num_sms ? want : 4LL * ctx->num_sms));
  k_fill<<<blocks, 256, 0, s>>>(v, count, value);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

}  // namespace uotk
