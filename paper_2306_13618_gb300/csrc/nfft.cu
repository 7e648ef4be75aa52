// NFFT engine (Alg. 2): both point sets binned once per solve; every
// half-step is spread -> convolve -> gather on the sorted points.  Also the
// stage-level entry points of the C ABI.
#include <math.h>

#include <memory>
#include <vector>

#include "nfft.cuh"

namespace uotk {

namespace {

__global__ void k_gather_f32(const int* __restrict__ perm, const float* __restrict__ in, long long n,
                             float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}
__global__ void k_scatter_f32(const int* __restrict__ perm, const float* __restrict__ in,
                              long long n, float* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[perm[i]] = in[i];
}
__global__ void k_gather_f64(const int* __restrict__ perm, const double* __restrict__ in,
                             long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = in[perm[i]];
}
__global__ void k_scatter_f64(const int* __restrict__ perm, const double* __restrict__ in,
                              long long n, double* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[perm[i]] = in[i];
}
// Validation of weights (sorted copies): negative / non-finite counters.
__global__ void k_check_weights(const float* __restrict__ w, long long n, long long* flags) {
  long long neg = 0, bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float v = w[i];
    neg += v < 0.f;
    bad += !isfinite(v);
  }
  neg = warp_sum(neg);
  bad = warp_sum(bad);
  if ((threadIdx.x & 31) == 0) {
    if (neg) flag_add(&flags[FLAG_NEG_WEIGHT], neg);
    if (bad) flag_add(&flags[FLAG_NONFINITE], bad);
  }
}
__global__ void k_check_points(const float* __restrict__ p, long long count, long long* flags) {
  long long bad = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x)
    bad += !isfinite(p[i]);
  bad = warp_sum(bad);
  if ((threadIdx.x & 31) == 0 && bad) flag_add(&flags[FLAG_NONFINITE], bad);
}

NfftParams params_from_info(const uotk_nfft_plan_info* p) {
  NfftParams P;
  P.d = p->d;
  P.n = p->grid;
  P.N = p->bandwidth;
  P.m = p->cutoff;
  for (int t = 0; t < 3; ++t) P.c[t] = p->center[t];
  P.inv_h = p->inv_h;
  P.h = p->h;
  P.eps = p->eps;
  P.b = (float)(M_PI * (2.0 - (double)P.N / P.n));
  P.tiles1 = P.n / NFFT_TILE;
  P.E = NFFT_TILE + 2 * P.m - 1;
  return P;
}

void info_from_params(const NfftParams& P, uotk_nfft_plan_info* p) {
  p->d = P.d;
  p->grid = P.n;
  p->bandwidth = P.N;
  p->cutoff = P.m;
  for (int t = 0; t < 3; ++t) p->center[t] = P.c[t];
  p->inv_h = P.inv_h;
  p->h = P.h;
  p->eps = P.eps;
}

uotk_status upload_scale(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, float* dev) {
  std::vector<float> t(3 * P.N);
  nfft_scale_table(P, t.data());
  UOTK_CUDA(ctx, cudaMemcpyAsync(dev, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice, s));
  UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  return UOTK_OK;
}

// Sizing params: everything that decides buffer sizes is data independent.
NfftParams sizing_params(uotk_ctx* ctx, int d, double eps, const uotk_sum_opts* opts) {
  NfftParams P;
  const float z[3] = {0, 0, 0};
  uotk_sum_opts o = opts ? *opts : uotk_sum_opts{};
  o.period = 1.0;  // skip the data-dependent period check
  nfft_make_params(ctx, d, z, z, eps, &o, &P);
  return P;
}

struct NfftEngine : Engine {
  uotk_ctx* ctx = nullptr;
  NfftParams P;
  int64_t n = 0, m = 0;
  NfftPoints X, Y;
  NfftWork W;
  float* as = nullptr;   // sorted weights of X
  float* bs = nullptr;   // sorted weights of Y

  static void carve(const NfftParams& P, int64_t n, int64_t m, Carver& cv, NfftEngine* e) {
    NfftPoints X, Y;
    NfftWork W;
    nfft_points_carve(cv, P, n, X);
    nfft_points_carve(cv, P, m, Y);
    nfft_work_carve(cv, P, n > m ? n : m, W);
    float* as = cv.take<float>((n > 0 ? n : 1) + 4);
    float* bs = cv.take<float>((m > 0 ? m : 1) + 4);
    if (e) { e->X = X; e->Y = Y; e->W = W; e->as = as; e->bs = bs; }
  }

  uotk_status half(cudaStream_t s, int side, const float* base, const double* pot, double lam,
                   const long long* shift_slot, float* out) override {
    const NfftPoints& src = side == 0 ? Y : X;
    const NfftPoints& tgt = side == 0 ? X : Y;
    SpreadWeights w{base, pot, lam, shift_slot};
    UOTK_TRY(nfft_spread(ctx, s, P, src, w, W, W.grid));
    UOTK_TRY(nfft_convolve(ctx, s, P, W, W.grid, W.grid));
    UOTK_TRY(nfft_gather(ctx, s, P, tgt, W.grid, out));
    // cost |x - y| (Laplace kernel): the near field with the spread's weights
    if (P.kernel != UOTK_KERNEL_GAUSS)
      UOTK_TRY(nfft_near(ctx, s, P, src, pot ? W.wts : base, tgt, W, out));
    return UOTK_OK;
  }
  // Gaussian kernel: the gather is the half-step's last kernel and takes the
  // dual update (the non-smooth kernels add their near field after it).
  bool fuses_dual() const override {
    return P.kernel == UOTK_KERNEL_GAUSS && X.n > 0 && Y.n > 0;
  }
  uotk_status half_dual(cudaStream_t s, int side, const float* base, const double* pot,
                        double lam, const long long* shift_slot, float* out,
                        const DualUpdate& du) override {
    if (!fuses_dual()) return UOTK_ERR_INTERNAL;
    const NfftPoints& src = side == 0 ? Y : X;
    const NfftPoints& tgt = side == 0 ? X : Y;
    SpreadWeights w{base, pot, lam, shift_slot};
    UOTK_TRY(nfft_spread(ctx, s, P, src, w, W, W.grid));
    UOTK_TRY(nfft_convolve(ctx, s, P, W, W.grid, W.grid));
    return nfft_gather(ctx, s, P, tgt, W.grid, out, &du);
  }
  uotk_status plain(cudaStream_t s, int src, int tgt, const float* w, float* out) override {
    SpreadWeights sw{w, nullptr, 0.0, nullptr};
    const NfftPoints& S = src == 0 ? X : Y;
    const NfftPoints& T = tgt == 0 ? X : Y;
    UOTK_TRY(nfft_spread(ctx, s, P, S, sw, W, W.grid));
    UOTK_TRY(nfft_convolve(ctx, s, P, W, W.grid, W.grid));
    UOTK_TRY(nfft_gather(ctx, s, P, T, W.grid, out));
    // non-smooth kernels: the Fourier part sums K_R; add w (K - K_R) of the near field
    if (P.kernel != UOTK_KERNEL_GAUSS) UOTK_TRY(nfft_near(ctx, s, P, S, w, T, W, out));
    return UOTK_OK;
  }
  const float* weights(int side) const override { return side == 0 ? as : bs; }
  const int* perm(int side) const override { return side == 0 ? X.perm : Y.perm; }
  uotk_status to_caller(cudaStream_t s, int side, const double* in, double* out) override {
    const NfftPoints& S = side == 0 ? X : Y;
    if (S.n == 0) return UOTK_OK;
    k_scatter_f64<<<grid_for(ctx, S.n, 256), 256, 0, s>>>(S.perm, in, S.n, out);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  }
  uotk_status to_caller_f32(cudaStream_t s, int side, const float* in, float* out) override {
    const NfftPoints& S = side == 0 ? X : Y;
    if (S.n == 0) return UOTK_OK;
    k_scatter_f32<<<grid_for(ctx, S.n, 256), 256, 0, s>>>(S.perm, in, S.n, out);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  }
  uotk_status from_caller(cudaStream_t s, int side, const double* in, double* out) override {
    const NfftPoints& S = side == 0 ? X : Y;
    if (S.n == 0) return UOTK_OK;
    k_gather_f64<<<grid_for(ctx, S.n, 256), 256, 0, s>>>(S.perm, in, S.n, out);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  }
  bool identity_order() const override { return false; }
};

uotk_status sorted_weights(uotk_ctx* ctx, cudaStream_t s, const NfftPoints& S, const float* w,
                           float* out) {
  if (S.n == 0) return UOTK_OK;
  UOTK_CUDA(ctx, cudaMemsetAsync(out, 0, sizeof(float) * (S.n + 4), s));
  if (!w) return UOTK_OK;
  k_gather_f32<<<grid_for(ctx, S.n, 256), 256, 0, s>>>(S.perm, w, S.n, out);
  UOTK_LAUNCHED(ctx);
  k_check_weights<<<grid_for(ctx, S.n, 256, 2), 256, 0, s>>>(out, S.n, ctx->dflags);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status check_points(uotk_ctx* ctx, cudaStream_t s, const float* p, int64_t count) {
  if (count == 0) return UOTK_OK;
  k_check_points<<<grid_for(ctx, count, 256, 2), 256, 0, s>>>(p, count, ctx->dflags);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

}  // namespace

size_t nfft_engine_bytes(uotk_ctx* ctx, const EngineSpec& sp) {
  const NfftParams P = sizing_params(ctx, sp.d, sp.eps, sp.opts);
  Carver cv(nullptr);
  NfftEngine::carve(P, sp.n, sp.m, cv, nullptr);
  return cv.off;
}

uotk_status nfft_engine_create(uotk_ctx* ctx, cudaStream_t s, const EngineSpec& sp, Carver& cv,
                               Engine** out) {
  UOTK_TRY(check_points(ctx, s, sp.x, sp.n * sp.d));
  UOTK_TRY(check_points(ctx, s, sp.y, sp.m * sp.d));
  float lo[3], hi[3];
  UOTK_TRY(nfft_bbox(ctx, s, sp.d, sp.x, sp.n, sp.y, sp.m, lo, hi));
  std::unique_ptr<NfftEngine> e(new NfftEngine());
  e->ctx = ctx;
  e->n = sp.n;
  e->m = sp.m;
  UOTK_TRY(nfft_make_params(ctx, sp.d, lo, hi, sp.eps, sp.opts, &e->P));
  NfftEngine::carve(e->P, sp.n, sp.m, cv, e.get());
  UOTK_TRY(nfft_points_build(ctx, s, e->P, sp.x, sp.n, e->X));
  UOTK_TRY(nfft_points_build(ctx, s, e->P, sp.y, sp.m, e->Y));
  UOTK_TRY(sorted_weights(ctx, s, e->X, sp.a, e->as));
  UOTK_TRY(sorted_weights(ctx, s, e->Y, sp.b, e->bs));
  if (e->P.kernel != UOTK_KERNEL_GAUSS)
    UOTK_TRY(nfft_reg_table(ctx, s, e->P, e->W));
  else
    UOTK_TRY(upload_scale(ctx, s, e->P, e->W.scale));
  *out = e.release();
  return UOTK_OK;
}

// ------------------------------------------------------------ stage ops ----
uotk_status op_nfft_plan(uotk_ctx* ctx, cudaStream_t s, int d, const float* src, int64_t n,
                         const float* tgt, int64_t m, double eps, const uotk_sum_opts* opts,
                         uotk_nfft_plan_info* plan) {
  UOTK_TRY(flags_reset(ctx, s));
  UOTK_TRY(check_points(ctx, s, src, n * d));
  UOTK_TRY(check_points(ctx, s, tgt, m * d));
  float lo[3], hi[3];
  UOTK_TRY(nfft_bbox(ctx, s, d, src, n, tgt, m, lo, hi));
  UOTK_TRY(flags_check(ctx, s, "nfft_plan"));
  NfftParams P;
  UOTK_TRY(nfft_make_params(ctx, d, lo, hi, eps, opts, &P));
  info_from_params(P, plan);
  return UOTK_OK;
}

uotk_status op_nfft_spread(uotk_ctx* ctx, cudaStream_t s, const uotk_nfft_plan_info* plan,
                           const float* pts, int64_t n, const float* w, float* grid) {
  const NfftParams P = params_from_info(plan);
  Carver size(nullptr);
  NfftPoints S;
  NfftWork W;
  nfft_points_carve(size, P, n, S);
  nfft_work_carve(size, P, n, W);
  size.take<float>((n > 0 ? n : 1) + 4);
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  nfft_points_carve(cv, P, n, S);
  nfft_work_carve(cv, P, n, W);
  float* ws = cv.take<float>((n > 0 ? n : 1) + 4);
  UOTK_TRY(check_points(ctx, s, pts, n * P.d));
  UOTK_TRY(nfft_points_build(ctx, s, P, pts, n, S));
  UOTK_TRY(sorted_weights(ctx, s, S, w, ws));
  SpreadWeights sw{ws, nullptr, 0.0, nullptr};
  UOTK_TRY(nfft_spread(ctx, s, P, S, sw, W, grid));
  return flags_check(ctx, s, "nfft_spread");
}

uotk_status op_nfft_convolve(uotk_ctx* ctx, cudaStream_t s, const uotk_nfft_plan_info* plan,
                             const float* grid_in, float* grid_out) {
  const NfftParams P = params_from_info(plan);
  Carver size(nullptr);
  NfftWork W;
  nfft_work_carve(size, P, 0, W);
  UOTK_TRY(ws_reserve(ctx, size.off));
  Carver cv(ctx->ws);
  nfft_work_carve(cv, P, 0, W);
  UOTK_TRY(upload_scale(ctx, s, P, W.scale));
  UOTK_TRY(nfft_convolve(ctx, s, P, W, grid_in, grid_out));
  UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  return UOTK_OK;
}

uotk_status op_nfft_gather(uotk_ctx* ctx, cudaStream_t s, const uotk_nfft_plan_info* plan,
                           const float* grid, const float* pts, int64_t m, float* out) {
  if (m == 0) return UOTK_OK;
  const NfftParams P = params_from_info(plan);
  Carver size(nullptr);
  NfftPoints S;
  nfft_points_carve(size, P, m, S);
  size.take<float>(m);
  UOTK_TRY(ws_reserve(ctx, size.off));
  UOTK_TRY(flags_reset(ctx, s));
  Carver cv(ctx->ws);
  nfft_points_carve(cv, P, m, S);
  float* tmp = cv.take<float>(m);
  UOTK_TRY(check_points(ctx, s, pts, m * P.d));
  UOTK_TRY(nfft_points_build(ctx, s, P, pts, m, S));
  UOTK_TRY(nfft_gather(ctx, s, P, S, grid, tmp));
  k_scatter_f32<<<grid_for(ctx, m, 256), 256, 0, s>>>(S.perm, tmp, m, out);
  UOTK_LAUNCHED(ctx);
  return flags_check(ctx, s, "nfft_gather");
}

}  // namespace uotk
