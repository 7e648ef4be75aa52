// Sinkhorn's algorithm for entropic UOT (Alg. 1 / Alg. 2), the dual value of
// Eq. (dual_euot), MMD^2 (Eq. 1205) and the unbalanced Sinkhorn divergence
// (Eq. 586), on top of a summation engine (direct or NFFT).
//
// Half-step (beta side; the gamma side exchanges the roles):
//   w_j    = nu_j * exp(lambda*gamma_j - M_gamma)        (product reference)
//   t_i    = sum_j exp(-||x_i - y_j||^2/eps) w_j          (FP32 kernel sum)
//   beta_i = -q (log t_i + M_gamma)                       (FP64)
//   beta_i =  q (log mu_i - log t_i - M_gamma)            (counting reference)
// with q = eta/(1 + eta*lambda) and M_gamma = max_j lambda*gamma_j, a global
// shift that keeps the FP32 weights in range and is added back after the log.
// Shifts are maxima taken with integer atomics on an order-preserving encoding,
// so every result is independent of scheduling.
#include <math.h>
#include <stdarg.h>

#include <memory>

#include "solver.cuh"

namespace uotk {

namespace {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS_PER_SM = 2;

// ---------------------------------------------------------------------------
// Direct engine.
// ---------------------------------------------------------------------------
struct DirectEngine : Engine {
  uotk_ctx* ctx = nullptr;
  int d = 0;
  int64_t n = 0, m = 0;
  const float* a = nullptr;
  const float* b = nullptr;
  double eps = 1.0;   // Gaussian width, or the parameter p of another kernel
  int kernel = UOTK_KERNEL_GAUSS;
  DirectLayout Lyx, Lxy, Lxx, Lyy;  // src -> tgt
  void* Px = nullptr;  // X packed as sources (weights a), also read as targets
  void* Py = nullptr;
  float* part = nullptr;
  void* multi = nullptr;  // scratch of the fused multi-sum (d <= 3)

  static void layouts(uotk_ctx* ctx, const EngineSpec& sp, DirectLayout& yx, DirectLayout& xy,
                      DirectLayout& xx, DirectLayout& yy) {
    yx = direct_layout(ctx, sp.d, sp.m, sp.n);
    xy = direct_layout(ctx, sp.d, sp.n, sp.m);
    xx = direct_layout(ctx, sp.d, sp.n, sp.n);
    yy = direct_layout(ctx, sp.d, sp.m, sp.m);
  }
  static void carve(uotk_ctx* ctx, const EngineSpec& sp, Carver& cv, DirectEngine* e) {
    DirectLayout yx, xy, xx, yy;
    layouts(ctx, sp, yx, xy, xx, yy);
    size_t part = yx.part_bytes;
    for (size_t p : {xy.part_bytes, xx.part_bytes, yy.part_bytes}) part = p > part ? p : part;
    // X is packed once as a source of xy/xx (n_pad rows >= n, also valid as targets).
    size_t bx = xy.src_bytes > yx.tgt_bytes ? xy.src_bytes : yx.tgt_bytes;
    size_t by = yx.src_bytes > xy.tgt_bytes ? yx.src_bytes : xy.tgt_bytes;
    void* px = cv.take<char>(bx > 0 ? bx : 16);
    void* py = cv.take<char>(by > 0 ? by : 16);
    // split partials: FP32 sums, or {M, S} pairs of the log-domain form
    float* pp = part ? cv.take<float>(2 * part / sizeof(float)) : nullptr;
    size_t mb = 0;
    if (sp.d <= 3)
      for (size_t b : {direct_multi_bytes(ctx, sp.d, sp.m, sp.n), direct_multi_bytes(ctx, sp.d, sp.n, sp.m),
                       direct_multi_bytes(ctx, sp.d, sp.n, sp.n), direct_multi_bytes(ctx, sp.d, sp.m, sp.m)})
        mb = b > mb ? b : mb;
    void* mp = mb ? cv.take<char>(mb) : nullptr;
    if (e) {
      e->Lyx = yx; e->Lxy = xy; e->Lxx = xx; e->Lyy = yy;
      e->Px = px; e->Py = py; e->part = pp; e->multi = mp;
    }
  }

  uotk_status half(cudaStream_t s, int side, const float* base, const double* pot, double lam,
                   const long long* shift_slot, float* out) override {
    const DirectLayout& L = side == 0 ? Lyx : Lxy;
    void* src = side == 0 ? Py : Px;
    void* tgt = side == 0 ? Px : Py;
    UOTK_TRY(direct_set_weights(ctx, s, L, src, base, pot, lam, shift_slot));
    DirectBufs bufs{src, tgt, part};
    // kernel LAPLACE: the Gibbs kernel of the cost |x - y| (r = 1), e^{-|x-y|/eps}
    return direct_run(ctx, s, L, bufs, eps, out, kernel);
  }
  uotk_status plain(cudaStream_t s, int src, int tgt, const float* w, float* out) override {
    const DirectLayout& L = src == 0 ? (tgt == 0 ? Lxx : Lxy) : (tgt == 0 ? Lyx : Lyy);
    void* P = src == 0 ? Px : Py;
    // the packed sources carry their current weights; rewrite them from w
    UOTK_TRY(direct_set_weights(ctx, s, L, P, w, nullptr, 0.0, nullptr));
    DirectBufs bufs{P, tgt == 0 ? Px : Py, part};
    return direct_run(ctx, s, L, bufs, eps, out, kernel);
  }
  uotk_status half_log(cudaStream_t s, int side, const float* base, const double* pot, double lam,
                       const long long* shift_slot, float2* out) override {
    const DirectLayout& L = side == 0 ? Lyx : Lxy;
    void* src = side == 0 ? Py : Px;
    void* tgt = side == 0 ? Px : Py;
    UOTK_TRY(direct_set_weights(ctx, s, L, src, base, pot, lam, shift_slot, true));
    DirectBufs bufs{src, tgt, part};
    return direct_run_lse(ctx, s, L, bufs, eps, out);
  }
  uotk_status sums_multi(cudaStream_t s, int src, int tgt, int nrhs, const float* const* base,
                         const double* pot, double lam, const long long* shift_slot,
                         float* const* out) override {
    if (kernel != UOTK_KERNEL_GAUSS || d > 3 || !multi)
      return Engine::sums_multi(s, src, tgt, nrhs, base, pot, lam, shift_slot, out);
    // the Gaussian sums share one distance and exponential per pair, 4 at a time
    for (int k0 = 0; k0 < nrhs; k0 += 4) {
      const int K = nrhs - k0 < 4 ? nrhs - k0 : 4;
      UOTK_TRY(direct_run_multi(ctx, s, d, src == 0 ? n : m, tgt == 0 ? n : m,
                                src == 0 ? Px : Py, tgt == 0 ? Px : Py, K, base + k0, pot, lam,
                                shift_slot, multi, eps, out + k0));
    }
    return UOTK_OK;
  }
  const int* perm(int) const override { return nullptr; }
  const float* weights(int side) const override { return side == 0 ? a : b; }
  uotk_status to_caller(cudaStream_t s, int side, const double* in, double* out) override {
    if (in != out)
      UOTK_CUDA(ctx, cudaMemcpyAsync(out, in, sizeof(double) * (side == 0 ? n : m),
                                     cudaMemcpyDeviceToDevice, s));
    return UOTK_OK;
  }
  uotk_status to_caller_f32(cudaStream_t s, int side, const float* in, float* out) override {
    if (in != out)
      UOTK_CUDA(ctx, cudaMemcpyAsync(out, in, sizeof(float) * (side == 0 ? n : m),
                                     cudaMemcpyDeviceToDevice, s));
    return UOTK_OK;
  }
  uotk_status from_caller(cudaStream_t s, int side, const double* in, double* out) override {
    return to_caller(s, side, in, out);
  }
  bool identity_order() const override { return true; }
};

// ---------------------------------------------------------------------------
// Kernels of the dual updates and reductions.
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_max(double v, double* sh) {
  v = warp_max(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : -INFINITY;
    v = warp_max(v);
  }
  __syncthreads();
  return v;
}

// pot_i <- dual update from the half-step sums; max of lam*pot -> *max_out;
// optional max |lam*change|.  LOG = false: t is FP32 t_i (log t_i = log t + shift);
// LOG = true: t is {M_i, S_i} of the log-domain form (log t_i = ln2 (M + log2 S) + shift).
template <bool LOG>
__global__ void k_dual_update(const void* __restrict__ t, const float* __restrict__ base,
                              long long count, double q, double lam, int ref,
                              long long* __restrict__ flags, int shift_in, int max_out,
                              int reset_slot, int delta_out, int reset_delta,
                              double* __restrict__ pot) {
  __shared__ double sh[32];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    flags[reset_slot] = ORDERED_NEG_INF;
    if (reset_delta >= 0) flags[reset_delta] = ORDERED_NEG_INF;
  }
  const double shift = ordered_to_dbl(flags[shift_in]);
  // v = -q (log t + shift) = -q log t - q shift (ref 0), q (log base - log t - shift)
  // (ref 1): the shift enters once per thread; lambda > 0 scales the maxima
  // once per block.  FP64 operations are scarce on this GPU.
  const double qs = q * shift;
  double mx = -INFINITY, dl = 0.0;
  long long bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    double lt;
    if (LOG) {
      const float2 v = reinterpret_cast<const float2*>(t)[i];
      lt = (v.y > 0.f && isfinite(v.x) && isfinite(v.y))
               ? ((double)v.x + log2((double)v.y)) * 0.6931471805599453
               : (double)NAN;
    } else {
      const float ti = reinterpret_cast<const float*>(t)[i];
      lt = ti > 0.f && isfinite(ti) ? log_f32(ti) : log((double)ti);
    }
    const double v = ref == 0 ? fma(-q, lt, -qs) : fma(q, log_f32(base[i]) - lt, -qs);
    if (delta_out >= 0) dl = fmax(dl, fabs(v - pot[i]));
    pot[i] = v;
    if (isfinite(v)) mx = fmax(mx, v);
    else bad++;
  }
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) atomicMax(&flags[max_out], dbl_to_ordered(lam * mx));
  if (delta_out >= 0) {
    dl = block_max(dl, sh);
    if (threadIdx.x == 0) atomicMax(&flags[delta_out], dbl_to_ordered(lam * dl));
  }
  if (bad) flag_add(&flags[FLAG_NONFINITE_DUAL], bad);
}

__global__ void k_max_pot(const double* __restrict__ pot, long long count, double lam,
                          long long* __restrict__ slot) {
  __shared__ double sh[32];
  double mx = -INFINITY;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    mx = fmax(mx, lam * pot[i]);
  mx = block_max(mx, sh);
  if (threadIdx.x == 0) atomicMax(slot, dbl_to_ordered(mx));
}

__global__ void k_flags_reset(long long* flags, long long wait_test) {
  const int i = threadIdx.x;
  if (i < NUM_FLAGS)
    flags[i] = (i >= FLAG_MAX_G0 && i <= FLAG_DELTA1) ? ORDERED_NEG_INF
               : i == FLAG_WAIT_TEST                  ? wait_test
                                                      : 0LL;
}

__global__ void k_sum_partials(SumTerms terms, const long long* __restrict__ flags,
                               double* __restrict__ part) {
  __shared__ double sh[32];
  for (int q = 0; q < terms.count; ++q) {
    const SumTerm T = terms.k[q];
    const double shift = T.kind >= 3 ? ordered_to_dbl(flags[T.shift_slot]) : 0.0;
    double acc = 0.0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < T.len;
         i += (long long)gridDim.x * blockDim.x) {
      const double bi = T.base ? (double)T.base[i] : 1.0;
      double v;
      if (T.kind == 0) v = bi * exp(-T.pot[i] / T.eta);
      else if (T.kind == 1) v = bi;
      else if (T.kind == 2) v = bi * (double)T.t[i];
      else if (T.kind == 3) v = bi * exp(T.lam * T.pot[i] + shift) * (double)T.t[i];
      else {
        const float2 ms = T.ms[i];
        v = ms.y > 0.f ? bi * exp(T.lam * T.pot[i] + shift +
                                  ((double)ms.x + log2((double)ms.y)) * 0.6931471805599453)
                       : 0.0;
      }
      acc += v;
    }
    acc = warp_sum(acc);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
      part[q * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

__global__ void k_sum_final(const double* __restrict__ part, int blocks, int count,
                            double* __restrict__ out) {
  // one warp per term, fixed order
  const int q = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (q >= count) return;
  double s = 0.0;
  for (int i = lane; i < blocks; i += 32) s += part[q * blocks + i];
  s = warp_sum(s);
  if (lane == 0) out[q] = s;
}

}  // namespace

uotk_status run_sums(uotk_ctx* ctx, cudaStream_t s, const Reducer& R, const SumTerms& T,
                     double* host_out) {
  {
    UOTK_PROF(ctx, s, "reduce");
    k_sum_partials<<<R.blocks, RED_THREADS, 0, s>>>(T, ctx->dflags, R.part);
  }
  UOTK_LAUNCHED(ctx);
  {
    UOTK_PROF(ctx, s, "reduce");
    k_sum_final<<<1, 32 * 5, 0, s>>>(R.part, R.blocks, T.count, R.out);
  }
  UOTK_LAUNCHED(ctx);
  UOTK_CUDA(ctx, cudaMemcpyAsync(host_out, R.out, sizeof(double) * T.count,
                                 cudaMemcpyDeviceToHost, s));
  return UOTK_OK;
}

void carve_reducer(uotk_ctx* ctx, Carver& cv, Reducer& R) {
  R.blocks = ctx->num_sms * RED_BLOCKS_PER_SM;
  R.part = cv.take<double>((size_t)5 * R.blocks);
  R.out = cv.take<double>(5);
}

void carve_solve(Carver& cv, int64_t n, int64_t m, bool need_copies, SolveBufs& B,
                 bool log_domain) {
  B.tx = cv.take<float>(n > 0 ? n : 1);
  B.ty = cv.take<float>(m > 0 ? m : 1);
  if (log_domain) {
    B.lx = cv.take<float2>(n > 0 ? n : 1);
    B.ly = cv.take<float2>(m > 0 ? m : 1);
  }
  if (need_copies) {
    B.beta = cv.take<double>(n > 0 ? n : 1);
    B.gamma = cv.take<double>(m > 0 ? m : 1);
  }
}

// Alg. 1 / Alg. 2 for up to max_sweeps sweeps on an engine, then D(beta, gamma).
uotk_status solve(uotk_ctx* ctx, cudaStream_t s, Engine* E, int64_t n, int64_t m, double eps,
                  double eta1, double eta2, int max_sweeps, double tol, int ref, bool warm,
                  const SolveBufs& B, const Reducer& R, SolveResult* res, bool log_domain) {
  const double lam = 1.0 / eps;
  const double q1 = eta1 / (1.0 + eta1 * lam), q2 = eta2 / (1.0 + eta2 * lam);
  const float* a = E->weights(0);
  const float* b = E->weights(1);
  long long* F = ctx->dflags;
  if (!warm) UOTK_CUDA(ctx, cudaMemsetAsync(B.gamma, 0, sizeof(double) * m, s));
  k_max_pot<<<grid_for(ctx, m, 256, 2), 256, 0, s>>>(B.gamma, m, lam, F + FLAG_MAX_G0);
  UOTK_LAUNCHED(ctx);
  const bool track = tol > 0.0;
  const int gu = grid_for(ctx, n > m ? n : m, 256, 4);
  // One sweep: the beta half-step (sum over Y into X, update beta), then the
  // gamma half-step (sum over X into Y, update gamma).  The flag slots
  // alternate with the sweep's parity (see k_dual_update).
  const bool fuse = !log_domain && E->fuses_dual();
  // The stream the sweeps go to: the caller's, or the context's own stream
  // while the loop is replayed from a graph (see below).
  cudaStream_t cs = s;
  auto sweep = [&](int sw) -> uotk_status {
    const int cur = sw & 1, nxt = cur ^ 1;
    if (fuse) {
      // the same updates, slots and counters as the two k_dual_update launches below
      const DualUpdate ub{a, B.beta, q1, lam, ref, FLAG_MAX_G0 + cur, FLAG_MAX_B0 + cur,
                          FLAG_MAX_G0 + nxt, track ? FLAG_DELTA0 + cur : -1,
                          track ? FLAG_DELTA0 + nxt : -1};
      UOTK_TRY(E->half_dual(cs, 0, ref == 0 ? b : nullptr, B.gamma, lam, F + FLAG_MAX_G0 + cur,
                            B.tx, ub));
      const DualUpdate ug{b, B.gamma, q2, lam, ref, FLAG_MAX_B0 + cur, FLAG_MAX_G0 + nxt,
                          FLAG_MAX_B0 + nxt, track ? FLAG_DELTA0 + cur : -1, -1};
      return E->half_dual(cs, 1, ref == 0 ? a : nullptr, B.beta, lam, F + FLAG_MAX_B0 + cur,
                          B.ty, ug);
    }
    if (log_domain)
      UOTK_TRY(E->half_log(cs, 0, ref == 0 ? b : nullptr, B.gamma, lam, F + FLAG_MAX_G0 + cur, B.lx));
    else
      UOTK_TRY(E->half(cs, 0, ref == 0 ? b : nullptr, B.gamma, lam, F + FLAG_MAX_G0 + cur, B.tx));
    {
      UOTK_PROF(ctx, cs, "dual_update");
      auto upd = log_domain ? k_dual_update<true> : k_dual_update<false>;
      upd<<<gu, 256, 0, cs>>>(log_domain ? (const void*)B.lx : (const void*)B.tx, a, n, q1, lam,
                             ref, F, FLAG_MAX_G0 + cur, FLAG_MAX_B0 + cur, FLAG_MAX_G0 + nxt,
                             track ? FLAG_DELTA0 + cur : -1, track ? FLAG_DELTA0 + nxt : -1,
                             B.beta);
    }
    UOTK_LAUNCHED(ctx);
    if (log_domain)
      UOTK_TRY(E->half_log(cs, 1, ref == 0 ? a : nullptr, B.beta, lam, F + FLAG_MAX_B0 + cur, B.ly));
    else
      UOTK_TRY(E->half(cs, 1, ref == 0 ? a : nullptr, B.beta, lam, F + FLAG_MAX_B0 + cur, B.ty));
    {
      UOTK_PROF(ctx, cs, "dual_update");
      auto upd = log_domain ? k_dual_update<true> : k_dual_update<false>;
      upd<<<gu, 256, 0, cs>>>(log_domain ? (const void*)B.ly : (const void*)B.ty, b, m, q2, lam,
                             ref, F, FLAG_MAX_B0 + cur, FLAG_MAX_G0 + nxt, FLAG_MAX_B0 + nxt,
                             track ? FLAG_DELTA0 + cur : -1, -1, B.gamma);
    }
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  };
  auto converged_now = [&](int done_sweeps, bool* conv) -> uotk_status {
    UOTK_CUDA(ctx, cudaMemcpyAsync(ctx->host, F + FLAG_DELTA0 + ((done_sweeps - 1) & 1),
                                   sizeof(long long), cudaMemcpyDeviceToHost, cs));
    UOTK_CUDA(ctx, cudaStreamSynchronize(cs));
    long long enc;
    memcpy(&enc, ctx->host, sizeof(long long));
    *conv = ordered_to_dbl(enc) < tol;
    return UOTK_OK;
  };
  int done = 0;
  bool converged = false;
  int next_check = 10;
  // Sweeps 0 and 1 run eagerly (they also set kernel attributes); later sweeps
  // are replayed from a CUDA graph of two sweeps (even, odd) when the loop is
  // long enough to pay for the capture, so that the convergence checks fall on
  // multiples of 10 sweeps as in the eager loop.  With profiling on, launches
  // stay eager so that every launch is timed by its own events.
  UOTK_TRY(sweep(0));
  done = 1;
  cudaGraphExec_t exec = nullptr;
  int64_t body_launches = 0;
  const bool graph_loop = !ctx->prof.on && max_sweeps >= 9;
  if (graph_loop) {
    UOTK_TRY(sweep(1));
    done = 2;
  }
  if (graph_loop) {
    // Capture two sweeps (even, odd) on the context's stream, ordered after
    // the caller's stream; the rest of the loop runs there and the caller's
    // stream waits for it at the end.
    UOTK_TRY(stream_fence(ctx, s, ctx->gs, ctx->fence_in));
    cs = ctx->gs;
    cudaGraph_t graph = nullptr;
    const int64_t l0 = ctx->launches;
    cudaError_t ec = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    if (ec == cudaSuccess) {
      const uotk_status st1 = sweep(2);
      const uotk_status st2 = st1 == UOTK_OK ? sweep(3) : st1;
      ec = cudaStreamEndCapture(cs, &graph);
      if (st2 == UOTK_OK && ec == cudaSuccess && graph)
        ec = cudaGraphInstantiate(&exec, graph, 0);
      else if (ec == cudaSuccess)
        ec = cudaErrorUnknown;
      if (graph) cudaGraphDestroy(graph);
    }
    body_launches = ctx->launches - l0;
    ctx->launches = l0;
    if (ec != cudaSuccess) {
      cudaGetLastError();
      if (exec) cudaGraphExecDestroy(exec);
      return set_error(ctx, UOTK_ERR_CUDA, "capture of the sweep loop failed: %s",
                       cudaGetErrorString(ec));
    }
  }
  while (done < max_sweeps) {
    if (exec && done + 2 <= max_sweeps && (done & 1) == 0) {
      if (cudaGraphLaunch(exec, cs) != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        return set_error(ctx, UOTK_ERR_CUDA, "graph launch of the sweep loop failed");
      }
      ctx->launches += body_launches;
      done += 2;
    } else {
      UOTK_TRY(sweep(done));
      done += 1;
    }
    if (track && (done >= next_check || done == max_sweeps)) {
      next_check = done + 10;
      const uotk_status st = converged_now(done, &converged);
      if (st != UOTK_OK) {
        if (exec) cudaGraphExecDestroy(exec);
        return st;
      }
      if (converged) break;
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (cs != s) UOTK_TRY(stream_fence(ctx, cs, s, ctx->fence_out));
  cs = s;
  if (track && done == 1 && max_sweeps == 1) {
    UOTK_TRY(converged_now(done, &converged));
  }
  // Dual value, Eq. (dual_euot), at the final duals.  The last gamma half-step
  // left t_y = sum_i k_ij mu_i e^{lambda beta_i - M_beta}, so the coupling sum is
  // sum_j nu_j e^{lambda gamma_j + M_beta} t_y,j.
  const int last = (done - 1) & 1;
  SumTerms T{};
  T.count = 5;
  T.k[0] = SumTerm{0, n, a, B.beta, nullptr, eta1, lam, 0};
  T.k[1] = SumTerm{0, m, b, B.gamma, nullptr, eta2, lam, 0};
  T.k[2] = SumTerm{1, n, a, nullptr, nullptr, 1.0, lam, 0};
  T.k[3] = SumTerm{1, m, b, nullptr, nullptr, 1.0, lam, 0};
  T.k[4] = SumTerm{log_domain ? 4 : 3, m, ref == 0 ? b : nullptr, B.gamma, B.ty, 1.0, lam,
                   FLAG_MAX_B0 + last, B.ly};
  UOTK_TRY(run_sums(ctx, s, R, T, ctx->host + 8));
  UOTK_TRY(flags_check(ctx, s, "uot_sinkhorn"));
  const double* h = ctx->host + 8;
  double coupling = h[4];
  if (ref == 0) coupling -= h[2] * h[3];
  res->value = -eta1 * h[0] - eta2 * h[1] + eta1 * h[2] + eta2 * h[3] - coupling / lam;
  res->sweeps = done;
  res->converged = converged;
  return UOTK_OK;
}


// ---------------------------------------------------------------------------
// Engine construction.
// ---------------------------------------------------------------------------
size_t engine_bytes(uotk_ctx* ctx, const EngineSpec& sp) {
  if (sp.method == UOTK_NFFT) return nfft_engine_bytes(ctx, sp);
  if (sp.method == UOTK_DIRECT_BF16 || sp.method == UOTK_DIRECT_BF16X3)
    return tc_engine_bytes(ctx, sp);
  Carver cv(nullptr);
  DirectEngine::carve(ctx, sp, cv, nullptr);
  return cv.off;
}

uotk_status engine_create(uotk_ctx* ctx, cudaStream_t s, const EngineSpec& sp, Carver& cv,
                          Engine** out) {
  if (sp.method == UOTK_NFFT) return nfft_engine_create(ctx, s, sp, cv, out);
  if (sp.method == UOTK_DIRECT_BF16 || sp.method == UOTK_DIRECT_BF16X3)
    return tc_engine_create(ctx, s, sp, cv, out);
  std::unique_ptr<DirectEngine> e(new DirectEngine());
  e->ctx = ctx; e->d = sp.d; e->n = sp.n; e->m = sp.m; e->a = sp.a; e->b = sp.b;
  e->eps = sp.eps;
  e->kernel = sp.opts ? sp.opts->kernel : UOTK_KERNEL_GAUSS;
  DirectEngine::carve(ctx, sp, cv, e.get());
  UOTK_TRY(direct_pack_sources(ctx, s, e->Lxy, sp.x, sp.a, e->Px));
  UOTK_TRY(direct_pack_sources(ctx, s, e->Lyx, sp.y, sp.b, e->Py));
  *out = e.release();
  return UOTK_OK;
}

uotk_status flags_reset(uotk_ctx* ctx, cudaStream_t s) {
  k_flags_reset<<<1, 32, 0, s>>>(ctx->dflags, ctx->wait_test);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status flags_check(uotk_ctx* ctx, cudaStream_t s, const char* what) {
  long long* h = reinterpret_cast<long long*>(ctx->host + 32);
  UOTK_CUDA(ctx, cudaMemcpyAsync(h, ctx->dflags, sizeof(long long) * NUM_FLAGS,
                                 cudaMemcpyDeviceToHost, s));
  UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  if (h[FLAG_NONFINITE])
    return set_error(ctx, UOTK_ERR_NONFINITE, "%s: %lld non-finite input values", what,
                     h[FLAG_NONFINITE]);
  if (h[FLAG_NEG_WEIGHT])
    return set_error(ctx, UOTK_ERR_INVALID, "%s: %lld negative weights", what, h[FLAG_NEG_WEIGHT]);
  if (h[FLAG_TIMEOUT])
    return set_error(ctx, UOTK_ERR_TIMEOUT, "%s: a device-side wait timed out", what);
  if (h[FLAG_INTERNAL])
    return set_error(ctx, UOTK_ERR_INTERNAL, "%s: internal bound check failed (%lld)", what,
                     h[FLAG_INTERNAL]);
  if (h[FLAG_NONFINITE_DUAL])
    return set_error(ctx, UOTK_ERR_NONFINITE,
                     "%s: %lld non-finite dual values (a kernel sum underflowed: eps too small "
                     "for the spread of the points?)", what, h[FLAG_NONFINITE_DUAL]);
  return UOTK_OK;
}

// ---------------------------------------------------------------------------
// Public operations (called from api.cu after validation).
// ---------------------------------------------------------------------------
uotk_status op_kernel_sum(uotk_ctx* ctx, cudaStream_t s, int d, const float* src, int64_t n,
                          const float* w, const float* tgt, int64_t m, float* out, double eps,
                          const uotk_sum_opts* opts) {
  // X = targets (no weights), Y = sources.
  EngineSpec sp{opts ? opts->method : UOTK_DIRECT, d, tgt, m, nullptr, src, n, w, eps, opts};
  Carver size(nullptr);
  const size_t eb = engine_bytes(ctx, sp);
  size.off = eb;
  float* tmp_off = size.take<float>(m > 0 ? m : 1);
  (void)tmp_off;
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  Engine* raw = nullptr;
  UOTK_TRY(engine_create(ctx, s, sp, cv, &raw));
  std::unique_ptr<Engine> E(raw);
  cv.off = eb;
  float* tmp = cv.take<float>(m > 0 ? m : 1);
  if (E->identity_order()) {
    UOTK_TRY(E->plain(s, 1, 0, E->weights(1), out));
  } else {
    UOTK_TRY(E->plain(s, 1, 0, E->weights(1), tmp));
    UOTK_TRY(E->to_caller_f32(s, 0, tmp, out));
  }
  return flags_check(ctx, s, "kernel_sum");
}

uotk_status op_uot_sinkhorn(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                            const float* a, const float* y, int64_t m, const float* b, double eps,
                            double rho1, double rho2, int max_sweeps, double tol, int ref,
                            unsigned flags, double* beta, double* gamma, int* sweeps_done,
                            double* value, const uotk_sum_opts* opts) {
  EngineSpec sp{opts ? opts->method : UOTK_DIRECT, d, x, n, a, y, m, b, eps, opts};
  const bool copies = sp.method == UOTK_NFFT;
  const bool logd = (flags & UOTK_LOG_DOMAIN) != 0;
  const int kernel = opts ? opts->kernel : UOTK_KERNEL_GAUSS;
  if (logd && (sp.method == UOTK_NFFT || kernel != UOTK_KERNEL_GAUSS))
    return set_error(ctx, UOTK_ERR_UNSUPPORTED,
                     "uot_sinkhorn: the log domain is implemented for the direct forms (FP32, "
                     "BF16, BF16x3) of the squared-distance cost only");
  // gamma^0 = c* 1 (Remark on the initialisation; c* of Eq. 561), computed
  // before the solve's workspace is carved.
  const bool cstar_init = (flags & UOTK_CSTAR_INIT) != 0;
  double cst[3] = {0.0, 0.0, 0.0};
  if (cstar_init)
    UOTK_TRY(op_cstar(ctx, s, d, x, n, a, y, m, b, eps, rho1, rho2,
                      kernel == UOTK_KERNEL_LAPLACE ? 1 : 2, sp.method, cst));
  Carver size(nullptr);
  size.off = engine_bytes(ctx, sp);
  SolveBufs B;
  Reducer R;
  carve_solve(size, n, m, copies, B, logd);
  carve_reducer(ctx, size, R);
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  Engine* raw = nullptr;
  UOTK_TRY(engine_create(ctx, s, sp, cv, &raw));
  std::unique_ptr<Engine> E(raw);
  cv.off = engine_bytes(ctx, sp);
  carve_solve(cv, n, m, copies, B, logd);
  carve_reducer(ctx, cv, R);
  if (!copies) { B.beta = beta; B.gamma = gamma; }
  const bool warm = (flags & (UOTK_WARM_START | UOTK_CSTAR_INIT)) != 0;
  if (cstar_init) UOTK_TRY(fill_f64(ctx, s, B.gamma, m, cst[0]));
  else if (copies && warm) UOTK_TRY(E->from_caller(s, 1, gamma, B.gamma));
  SolveResult res;
  UOTK_TRY(solve(ctx, s, E.get(), n, m, eps, rho1, rho2, max_sweeps, tol, ref, warm, B, R, &res,
                 logd));
  if (copies) {
    UOTK_TRY(E->to_caller(s, 0, B.beta, beta));
    UOTK_TRY(E->to_caller(s, 1, B.gamma, gamma));
    UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  }
  if (sweeps_done) *sweeps_done = res.sweeps;
  if (value) *value = res.value;
  if (tol > 0.0 && !res.converged)
    return set_error(ctx, UOTK_ERR_NOT_CONVERGED, "uot_sinkhorn: tol %g not reached in %d sweeps",
                     tol, max_sweeps);
  return UOTK_OK;
}

uotk_status op_sinkhorn_divergence(uotk_ctx* ctx, cudaStream_t s, int d, const float* x,
                                   int64_t n, const float* a, const float* y, int64_t m,
                                   const float* b, double eps, double rho, int max_sweeps,
                                   double tol, double* sd, double* parts,
                                   const uotk_sum_opts* opts) {
  const int method = opts ? opts->method : UOTK_DIRECT;
  const EngineSpec specs[3] = {
      {method, d, x, n, a, y, m, b, eps, opts},
      {method, d, x, n, a, x, n, a, eps, opts},
      {method, d, y, m, b, y, m, b, eps, opts}};
  const bool copies = method == UOTK_NFFT;
  size_t need = 0;
  for (const EngineSpec& sp : specs) {
    Carver c(nullptr);
    c.off = engine_bytes(ctx, sp);
    SolveBufs B;
    Reducer R;
    carve_solve(c, sp.n, sp.m, true, B);
    carve_reducer(ctx, c, R);
    need = c.off > need ? c.off : need;
  }
  UOTK_TRY(ws_reserve(ctx, need));
  double v[3];
  double masses[2] = {0, 0};
  bool all_converged = true;
  for (int k = 0; k < 3; ++k) {
    const EngineSpec& sp = specs[k];
    UOTK_TRY(flags_reset(ctx, s));
    Carver cv(ctx->ws);
    Engine* raw = nullptr;
    UOTK_TRY(engine_create(ctx, s, sp, cv, &raw));
    std::unique_ptr<Engine> E(raw);
    cv.off = engine_bytes(ctx, sp);
    SolveBufs B;
    Reducer R;
    carve_solve(cv, sp.n, sp.m, true, B);
    carve_reducer(ctx, cv, R);
    (void)copies;
    SolveResult res;
    UOTK_TRY(solve(ctx, s, E.get(), sp.n, sp.m, eps, rho, rho, max_sweeps, tol, 0, false, B, R,
                   &res));
    all_converged = all_converged && res.converged;
    v[k] = res.value;
    if (k == 0) {
      masses[0] = ctx->host[8 + 2];
      masses[1] = ctx->host[8 + 3];
    }
  }
  const double dm = masses[0] - masses[1];
  *sd = v[0] - 0.5 * v[1] - 0.5 * v[2] + 0.5 * eps * dm * dm;
  if (parts) { parts[0] = v[0]; parts[1] = v[1]; parts[2] = v[2]; }
  if (tol > 0.0 && !all_converged)
    return set_error(ctx, UOTK_ERR_NOT_CONVERGED, "sinkhorn_divergence: tol %g not reached", tol);
  return UOTK_OK;
}

uotk_status op_mmd2(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                    const float* a, const float* y, int64_t m, const float* b, double ell,
                    double* mmd2, double* parts, const uotk_sum_opts* opts) {
  // the Gaussian of Eq. (1205) has width eps = ell^2; the other kernels take ell as p
  const int kernel = opts ? opts->kernel : UOTK_KERNEL_GAUSS;
  EngineSpec sp{opts ? opts->method : UOTK_DIRECT, d, x, n, a, y, m, b,
                kernel == UOTK_KERNEL_GAUSS ? ell * ell : ell, opts};
  Carver size(nullptr);
  size.off = engine_bytes(ctx, sp);
  size.take<float>(2 * (n > 0 ? n : 1) + (m > 0 ? m : 1));
  Reducer R;
  carve_reducer(ctx, size, R);
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  Engine* raw = nullptr;
  UOTK_TRY(engine_create(ctx, s, sp, cv, &raw));
  std::unique_ptr<Engine> E(raw);
  cv.off = engine_bytes(ctx, sp);
  float* t1 = cv.take<float>(2 * (n > 0 ? n : 1) + (m > 0 ? m : 1));
  float* t2 = t1 + (n > 0 ? n : 1);
  float* t3 = t2 + (n > 0 ? n : 1);
  carve_reducer(ctx, cv, R);
  const float* ai = E->weights(0);
  const float* bi = E->weights(1);
  UOTK_TRY(E->plain(s, 0, 0, ai, t1));  // (K_xx a)_i
  UOTK_TRY(E->plain(s, 1, 0, bi, t2));  // (K_xy b)_i
  UOTK_TRY(E->plain(s, 1, 1, bi, t3));  // (K_yy b)_j
  SumTerms T{};
  T.count = 3;
  T.k[0] = SumTerm{2, n, ai, nullptr, t1, 1.0, 1.0, 0};
  T.k[1] = SumTerm{2, n, ai, nullptr, t2, 1.0, 1.0, 0};
  T.k[2] = SumTerm{2, m, bi, nullptr, t3, 1.0, 1.0, 0};
  UOTK_TRY(run_sums(ctx, s, R, T, ctx->host + 16));
  UOTK_TRY(flags_check(ctx, s, "mmd2"));
  const double* h = ctx->host + 16;
  *mmd2 = h[0] - 2.0 * h[1] + h[2];
  if (parts) { parts[0] = h[0]; parts[1] = h[1]; parts[2] = h[2]; }
  return UOTK_OK;
}

}  // namespace uotk
