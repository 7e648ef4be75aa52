// Batched unbalanced Sinkhorn: Alg. 1 (direct form, d <= 3) on many independent
// pairs of point clouds of uneven sizes, each with its own eps and marginal
// penalties, advanced together.
//
// Every half-step of every pair is one grouped launch: a table of work items
// (pair, target block, source split) built once per call assigns CTAs to
// pairs, so a sweep over all pairs costs six launches whatever their number,
// and the sweep loop runs on the device: one CUDA graph whose WHILE
// conditional node repeats a body of two sweeps and a control kernel.  Per-pair
// state (shift maxima, convergence deltas) lives in per-pair slots that
// alternate with the sweep parity exactly as in the single-problem solver.
// After every body the control kernel retires the pairs whose last change met
// the tolerance (their CTAs return at once in later sweeps, and their duals stay
// as they were) and ends the loop when none is left or the sweep cap is near:
// no host round trip inside the loop.  With per-stage profiling on, the
// launches stay eager and the host checks the deltas every 10 sweeps.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "direct_body.cuh"
#include "engine.cuh"

namespace uotk {

namespace {

constexpr int BATCH_R = 4;                                  // targets per thread
constexpr int BATCH_TARGETS = DIRECT_THREADS * BATCH_R;     // targets per CTA
constexpr int BATCH_MAX_TILES = 64;                         // source tiles per CTA
constexpr int BATCH_CHUNK = 4096;                           // elements per update block
enum { SL_MAXG0 = 0, SL_MAXG1, SL_MAXB0, SL_MAXB1, SL_DELTA0, SL_DELTA1, SL_COUNT };

struct PairDev {
  long long x_off, y_off;    // first point of the pair in the caller's arrays
  long long n, m;
  long long px_off, py_off;  // first packed float4 (tile aligned)
  int tiles_x, tiles_y;
  int splits_x, splits_y;    // source splits of the X <- Y and Y <- X sums
  int tps_x, tps_y;          // source tiles per split
  long long part_x, part_y;  // first partial sum of the pair ([split][n], [split][m])
  float neg_c;               // -log2(e)/eps
  double lam, q1, q2, eta1, eta2;
};
struct SumItem {
  int pair, block, split, pad;
};
struct ElemItem {
  int pair, pad;
  long long start;
};

__device__ __forceinline__ double block_max_b(double v, double* sh) {
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
__device__ __forceinline__ double block_sum_b(double v, double* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    v = warp_sum(v);
  }
  __syncthreads();
  return v;
}

// Packed points of one side (float4 (x, y, z, w), w set per half-step) and
// validation counters; the buffer was zeroed, so padding rows stay zero.
template <int SIDE>  // 0: X (weights a), 1: Y (weights b)
__global__ void k_batch_pack(const ElemItem* __restrict__ items, const PairDev* __restrict__ pairs,
                             const float* __restrict__ pts, const float* __restrict__ w, int d,
                             float4* __restrict__ packed, long long* __restrict__ flags) {
  const ElemItem it = items[blockIdx.x];
  const PairDev P = pairs[it.pair];
  const long long cnt = SIDE == 0 ? P.n : P.m;
  const long long off = SIDE == 0 ? P.x_off : P.y_off;
  const long long poff = SIDE == 0 ? P.px_off : P.py_off;
  const long long end = min(it.start + (long long)BATCH_CHUNK, cnt);
  long long neg = 0, bad = 0;
  for (long long i = it.start + threadIdx.x; i < end; i += blockDim.x) {
    const long long g = off + i;
    float4 p = make_float4(pts[g * d], d > 1 ? pts[g * d + 1] : 0.f, d > 2 ? pts[g * d + 2] : 0.f,
                           0.f);
    bad += !isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z) || !isfinite(w[g]);
    neg += w[g] < 0.f;
    packed[poff + i] = p;
  }
  neg = warp_sum(neg);
  bad = warp_sum(bad);
  if ((threadIdx.x & 31) == 0) {
    if (neg) flag_add(&flags[FLAG_NEG_WEIGHT], neg);
    if (bad) flag_add(&flags[FLAG_NONFINITE], bad);
  }
}

// Source weights w = base * exp(lam pot - shift) of one side for the next sum.
template <int SIDE>  // 0: sources Y (gamma, b), 1: sources X (beta, a)
__global__ void k_batch_weights(const ElemItem* __restrict__ items,
                                const PairDev* __restrict__ pairs, const int* __restrict__ active,
                                const float* __restrict__ base, const double* __restrict__ pot,
                                const long long* __restrict__ slots, int shift_slot,
                                float4* __restrict__ packed) {
  const ElemItem it = items[blockIdx.x];
  if (!active[it.pair]) return;
  const PairDev P = pairs[it.pair];
  const long long cnt = SIDE == 0 ? P.m : P.n;
  const long long off = SIDE == 0 ? P.y_off : P.x_off;
  const long long poff = SIDE == 0 ? P.py_off : P.px_off;
  const double shift = ordered_to_dbl(slots[(long long)it.pair * SL_COUNT + shift_slot]);
  const long long end = min(it.start + (long long)BATCH_CHUNK, cnt);
  for (long long i = it.start + threadIdx.x; i < end; i += blockDim.x) {
    float v = exp_shifted(P.lam * pot[off + i] - shift);
    if (base) v *= base[off + i];
    packed[poff + i].w = v;
  }
}

// One CTA of a grouped direct sum: BATCH_TARGETS targets of one pair against
// one split of its source tiles.
template <int DIR, int D>  // DIR 0: targets X, sources Y; 1: targets Y, sources X
__global__ void __launch_bounds__(DIRECT_THREADS)
    k_batch_sum(const SumItem* __restrict__ items, const PairDev* __restrict__ pairs,
                const int* __restrict__ active, const float4* __restrict__ px,
                const float4* __restrict__ py, float* __restrict__ part,
                long long* __restrict__ flags) {
  const SumItem it = items[blockIdx.x];
  if (!active[it.pair]) return;
  const PairDev P = pairs[it.pair];
  const float4* src = DIR == 0 ? py + P.py_off : px + P.px_off;
  const float4* tgt = DIR == 0 ? px + P.px_off : py + P.py_off;
  const long long m = DIR == 0 ? P.n : P.m;
  const int tiles = DIR == 0 ? P.tiles_y : P.tiles_x;
  const int tps = DIR == 0 ? P.tps_x : P.tps_y;
  const long long t_begin = (long long)it.split * tps;
  const int count = (int)max(0LL, min((long long)tps, (long long)tiles - t_begin));
  float* o = part + (DIR == 0 ? P.part_x : P.part_y) + (long long)it.split * m;
  direct_body<D, BATCH_R, 0>(src, t_begin, count, tgt, m, (long long)it.block * BATCH_TARGETS,
                             P.neg_c, 0.f, o, flags);
}

// Dual update of one side from the split partial sums (Eq. Sinkhorn_uot_iteration),
// per-pair shift, maximum and change; optionally stores the reduced sums.
template <int DIR>  // 0: beta from the X <- Y sums; 1: gamma from the Y <- X sums
__global__ void k_batch_update(const ElemItem* __restrict__ items,
                               const PairDev* __restrict__ pairs, const int* __restrict__ active,
                               const float* __restrict__ part, const float* __restrict__ base,
                               int ref, long long* __restrict__ slots, int shift_in, int max_out,
                               int reset_slot, int delta_out, int reset_delta,
                               double* __restrict__ pot, float* __restrict__ t_store,
                               long long* __restrict__ flags) {
  __shared__ double sh[32];
  const ElemItem it = items[blockIdx.x];
  if (!active[it.pair]) return;
  const PairDev P = pairs[it.pair];
  long long* S = slots + (long long)it.pair * SL_COUNT;
  if (it.start == 0 && threadIdx.x == 0) {
    S[reset_slot] = ORDERED_NEG_INF;
    if (reset_delta >= 0) S[reset_delta] = ORDERED_NEG_INF;
  }
  const long long cnt = DIR == 0 ? P.n : P.m;
  const long long off = DIR == 0 ? P.x_off : P.y_off;
  const int splits = DIR == 0 ? P.splits_x : P.splits_y;
  const float* pp = part + (DIR == 0 ? P.part_x : P.part_y);
  const double q = DIR == 0 ? P.q1 : P.q2;
  const double shift = ordered_to_dbl(S[shift_in]);
  const long long end = min(it.start + (long long)BATCH_CHUNK, cnt);
  double mx = -INFINITY, dl = 0.0;
  long long bad = 0;
  for (long long i = it.start + threadIdx.x; i < end; i += blockDim.x) {
    double t = 0.0;
    for (int k = 0; k < splits; ++k) t += (double)pp[(long long)k * cnt + i];
    if (t_store) t_store[off + i] = (float)t;
    const double lt = log(t) + shift;
    const double v = ref == 0 ? -q * lt : q * (log_f32(base[off + i]) - lt);
    if (delta_out >= 0) dl = fmax(dl, fabs(P.lam * (v - pot[off + i])));
    pot[off + i] = v;
    if (isfinite(v)) mx = fmax(mx, P.lam * v);
    else bad++;
  }
  mx = block_max_b(mx, sh);
  if (threadIdx.x == 0) atomicMax(&S[max_out], dbl_to_ordered(mx));
  if (delta_out >= 0) {
    dl = block_max_b(dl, sh);
    if (threadIdx.x == 0) atomicMax(&S[delta_out], dbl_to_ordered(dl));
  }
  if (bad) flag_add(&flags[FLAG_NONFINITE_DUAL], bad);
}

__global__ void k_batch_init(const PairDev* __restrict__ pairs, int npairs,
                             long long* __restrict__ slots, int* __restrict__ active) {
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < npairs; p += gridDim.x * blockDim.x) {
    for (int k = 0; k < SL_COUNT; ++k) slots[(long long)p * SL_COUNT + k] = ORDERED_NEG_INF;
    slots[(long long)p * SL_COUNT + SL_MAXG0] = dbl_to_ordered(0.0);  // gamma^0 = 0
    active[p] = 1;
  }
}

// The five FP64 sums of the dual value of pair blockIdx.x (fixed order):
//   sum a e^{-beta/eta1}, sum b e^{-gamma/eta2}, sum a, sum b,
//   sum (b or 1) e^{lam gamma + M_beta} t_y  (t_y: last Y <- X sum).
__global__ void k_batch_values(const PairDev* __restrict__ pairs, const float* __restrict__ a,
                               const float* __restrict__ b, const double* __restrict__ beta,
                               const double* __restrict__ gamma, const float* __restrict__ ty,
                               const long long* __restrict__ slots,
                               const int* __restrict__ lastpar, int ref,
                               double* __restrict__ out) {
  __shared__ double sh[32];
  const int p = blockIdx.x;
  const PairDev P = pairs[p];
  const double shift_b =
      ordered_to_dbl(slots[(long long)p * SL_COUNT + SL_MAXB0 + lastpar[p]]);
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0, s4 = 0.0;
  for (long long i = threadIdx.x; i < P.n; i += blockDim.x) {
    const double ai = (double)a[P.x_off + i];
    s0 += ai * exp(-beta[P.x_off + i] / P.eta1);
    s2 += ai;
  }
  for (long long j = threadIdx.x; j < P.m; j += blockDim.x) {
    const double bj = (double)b[P.y_off + j];
    const double g = gamma[P.y_off + j];
    s1 += bj * exp(-g / P.eta2);
    s3 += bj;
    s4 += (ref == 0 ? bj : 1.0) * exp(P.lam * g + shift_b) * (double)ty[P.y_off + j];
  }
  const double v[5] = {block_sum_b(s0, sh), block_sum_b(s1, sh), block_sum_b(s2, sh),
                       block_sum_b(s3, sh), block_sum_b(s4, sh)};
  if (threadIdx.x == 0)
    for (int k = 0; k < 5; ++k) out[(long long)p * 5 + k] = v[k];
}

// Loop control after a body of two sweeps (one CTA): state[0] = sweeps done
// before the body, state[1] = pairs still active after it.  A pair whose
// largest change lambda |delta| in the body's last sweep is below tol retires
// with its sweep count; the WHILE condition drops to 0 when no pair is left or
// another body would pass max_sweeps.
__global__ void k_batch_control(int npairs, int* __restrict__ active, int* __restrict__ dsweeps,
                                const long long* __restrict__ slots, int* __restrict__ state,
                                double tol, int max_sweeps, cudaGraphConditionalHandle cond) {
  __shared__ int rem[32];
  const int done = state[0] + 2;
  const int par = (done - 1) & 1;
  int r = 0;
  for (int p = threadIdx.x; p < npairs; p += blockDim.x) {
    if (!active[p]) continue;
    if (tol > 0.0 &&
        ordered_to_dbl(slots[(long long)p * SL_COUNT + SL_DELTA0 + par]) < tol) {
      active[p] = 0;
      dsweeps[p] = done;
      continue;
    }
    ++r;
  }
  r = warp_sum(r);
  if ((threadIdx.x & 31) == 0) rem[threadIdx.x >> 5] = r;
  __syncthreads();
  if (threadIdx.x == 0) {
    int total = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) total += rem[w];
    state[0] = done;
    state[1] = total;
    if (total == 0 || done + 2 > max_sweeps) cudaGraphSetConditional(cond, 0);
  }
}

template <class T>
uotk_status upload(uotk_ctx* ctx, cudaStream_t s, T* dst, const std::vector<T>& src) {
  if (src.empty()) return UOTK_OK;
  UOTK_CUDA(ctx, cudaMemcpyAsync(dst, src.data(), sizeof(T) * src.size(),
                                 cudaMemcpyHostToDevice, s));
  return UOTK_OK;
}

}  // namespace

uotk_status op_uot_sinkhorn_batch(uotk_ctx* ctx, cudaStream_t s, int d, int npairs_all,
                                  const int64_t* x_off, const float* x, const float* a,
                                  const int64_t* y_off, const float* y, const float* b,
                                  const double* eps_all, const double* rho1_all,
                                  const double* rho2_all, int max_sweeps, double tol, int ref,
                                  double* beta, double* gamma, int* sweeps_done_all,
                                  double* values_all, const int* subset, int nsub) {
  // With `subset`, only the pairs subset[0 .. nsub-1] of the caller's npairs_all
  // are solved (each keeps its own point ranges and outputs); pair k below is
  // the caller's pair orig[k].
  const int npairs = subset ? nsub : npairs_all;
  std::vector<int> orig(npairs);
  for (int k = 0; k < npairs; ++k) orig[k] = subset ? subset[k] : k;
  std::vector<double> eps(npairs), rho1(npairs), rho2(npairs);
  for (int k = 0; k < npairs; ++k) {
    eps[k] = eps_all[orig[k]];
    rho1[k] = rho1_all[orig[k]];
    rho2[k] = rho2_all[orig[k]];
  }
  if (npairs == 0) return UOTK_OK;
  // ---- per-pair layout and work-item tables (host) ----
  std::vector<PairDev> P(npairs);
  std::vector<SumItem> sx, sy;
  std::vector<ElemItem> ex, ey;
  long long px = 0, py = 0, partx = 0, party = 0;
  const long long tile = DIRECT_TILE;
  for (int p = 0; p < npairs; ++p) {
    PairDev& q = P[p];
    const int o = orig[p];
    q.x_off = x_off[o];
    q.y_off = y_off[o];
    q.n = x_off[o + 1] - x_off[o];
    q.m = y_off[o + 1] - y_off[o];
    q.tiles_x = (int)((q.n + tile - 1) / tile);
    q.tiles_y = (int)((q.m + tile - 1) / tile);
    q.px_off = px;
    q.py_off = py;
    px += (long long)q.tiles_x * tile;
    py += (long long)q.tiles_y * tile;
    q.splits_x = (q.tiles_y + BATCH_MAX_TILES - 1) / BATCH_MAX_TILES;
    q.tps_x = (q.tiles_y + q.splits_x - 1) / q.splits_x;
    q.splits_y = (q.tiles_x + BATCH_MAX_TILES - 1) / BATCH_MAX_TILES;
    q.tps_y = (q.tiles_x + q.splits_y - 1) / q.splits_y;
    q.part_x = partx;
    q.part_y = party;
    partx += (long long)q.splits_x * q.n;
    party += (long long)q.splits_y * q.m;
    q.lam = 1.0 / eps[p];
    q.neg_c = (float)(-1.4426950408889634 * q.lam);
    q.eta1 = rho1[p];
    q.eta2 = rho2[p];
    q.q1 = rho1[p] / (1.0 + rho1[p] * q.lam);
    q.q2 = rho2[p] / (1.0 + rho2[p] * q.lam);
    const int bx = (int)((q.n + BATCH_TARGETS - 1) / BATCH_TARGETS);
    const int by = (int)((q.m + BATCH_TARGETS - 1) / BATCH_TARGETS);
    for (int k = 0; k < q.splits_x; ++k)
      for (int t = 0; t < bx; ++t) sx.push_back({p, t, k, 0});
    for (int k = 0; k < q.splits_y; ++k)
      for (int t = 0; t < by; ++t) sy.push_back({p, t, k, 0});
    for (long long i = 0; i < q.n; i += BATCH_CHUNK) ex.push_back({p, 0, i});
    for (long long j = 0; j < q.m; j += BATCH_CHUNK) ey.push_back({p, 0, j});
  }
  if (sx.size() > 0x7fffffff || sy.size() > 0x7fffffff)
    return set_error(ctx, UOTK_ERR_UNSUPPORTED, "uot_sinkhorn_batch: too many work items");
  const long long total_n = x_off[npairs_all] - x_off[0], total_m = y_off[npairs_all] - y_off[0];

  // ---- workspace ----
  auto carve = [&](Carver& cv, PairDev** dp, SumItem** dsx, SumItem** dsy, ElemItem** dex,
                   ElemItem** dey, int** act, long long** slots, int** lastpar, float4** dpx,
                   float4** dpy, float** dpartx, float** dparty, float** ty, double** vals,
                   int** dsw, int** state) {
    *dp = cv.take<PairDev>(npairs);
    *dsw = cv.take<int>(npairs);
    *state = cv.take<int>(2);
    *dsx = cv.take<SumItem>(sx.size() ? sx.size() : 1);
    *dsy = cv.take<SumItem>(sy.size() ? sy.size() : 1);
    *dex = cv.take<ElemItem>(ex.size() ? ex.size() : 1);
    *dey = cv.take<ElemItem>(ey.size() ? ey.size() : 1);
    *act = cv.take<int>(npairs);
    *slots = cv.take<long long>((size_t)npairs * SL_COUNT);
    *lastpar = cv.take<int>(npairs);
    *dpx = cv.take<float4>(px > 0 ? px : 1);
    *dpy = cv.take<float4>(py > 0 ? py : 1);
    *dpartx = cv.take<float>(partx > 0 ? partx : 1);
    *dparty = cv.take<float>(party > 0 ? party : 1);
    *ty = cv.take<float>(total_m > 0 ? total_m + y_off[0] : 1);
    *vals = cv.take<double>((size_t)npairs * 5);
  };
  PairDev* dP;
  SumItem *dSX, *dSY;
  ElemItem *dEX, *dEY;
  int *act, *lastpar;
  long long* slots;
  float4 *dPX, *dPY;
  float *partX, *partY, *ty;
  double* vals;
  int *dsw, *state;
  {
    Carver size(nullptr);
    carve(size, &dP, &dSX, &dSY, &dEX, &dEY, &act, &slots, &lastpar, &dPX, &dPY, &partX, &partY,
          &ty, &vals, &dsw, &state);
    UOTK_TRY(ws_reserve(ctx, size.off));
  }
  Carver cv(ctx->ws);
  carve(cv, &dP, &dSX, &dSY, &dEX, &dEY, &act, &slots, &lastpar, &dPX, &dPY, &partX, &partY, &ty,
        &vals, &dsw, &state);
  (void)total_n;

  UOTK_TRY(flags_reset(ctx, s));
  UOTK_TRY(upload(ctx, s, dP, P));
  UOTK_TRY(upload(ctx, s, dSX, sx));
  UOTK_TRY(upload(ctx, s, dSY, sy));
  UOTK_TRY(upload(ctx, s, dEX, ex));
  UOTK_TRY(upload(ctx, s, dEY, ey));
  UOTK_CUDA(ctx, cudaMemsetAsync(dPX, 0, sizeof(float4) * (px > 0 ? px : 1), s));
  UOTK_CUDA(ctx, cudaMemsetAsync(dPY, 0, sizeof(float4) * (py > 0 ? py : 1), s));
  if (!subset) {
    UOTK_CUDA(ctx, cudaMemsetAsync(gamma + y_off[0], 0, sizeof(double) * total_m, s));
  } else {
    for (int p = 0; p < npairs; ++p)
      UOTK_CUDA(ctx, cudaMemsetAsync(gamma + P[p].y_off, 0, sizeof(double) * P[p].m, s));
  }
  k_batch_init<<<grid_for(ctx, npairs, 256), 256, 0, s>>>(dP, npairs, slots, act);
  UOTK_LAUNCHED(ctx);
  if (!ex.empty()) {
    k_batch_pack<0><<<(unsigned)ex.size(), 256, 0, s>>>(dEX, dP, x, a, d, dPX, ctx->dflags);
    UOTK_LAUNCHED(ctx);
  }
  if (!ey.empty()) {
    k_batch_pack<1><<<(unsigned)ey.size(), 256, 0, s>>>(dEY, dP, y, b, d, dPY, ctx->dflags);
    UOTK_LAUNCHED(ctx);
  }
  UOTK_TRY(flags_check(ctx, s, "uot_sinkhorn_batch"));

  // ---- the sweep loop (shared structure with the single-problem solver) ----
  const bool track = tol > 0.0;
  // the stream of the sweeps: the caller's, or the context's own stream while
  // the device loop is captured and run
  cudaStream_t cs = s;
  auto sum_x = [&]() -> uotk_status {
    if (sx.empty()) return UOTK_OK;
    UOTK_PROF(ctx, cs, "direct");
    if (d == 1) k_batch_sum<0, 1><<<(unsigned)sx.size(), DIRECT_THREADS, 0, cs>>>(dSX, dP, act, dPX, dPY, partX, ctx->dflags);
    else if (d == 2) k_batch_sum<0, 2><<<(unsigned)sx.size(), DIRECT_THREADS, 0, cs>>>(dSX, dP, act, dPX, dPY, partX, ctx->dflags);
    else k_batch_sum<0, 3><<<(unsigned)sx.size(), DIRECT_THREADS, 0, cs>>>(dSX, dP, act, dPX, dPY, partX, ctx->dflags);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  };
  auto sum_y = [&]() -> uotk_status {
    if (sy.empty()) return UOTK_OK;
    UOTK_PROF(ctx, cs, "direct");
    if (d == 1) k_batch_sum<1, 1><<<(unsigned)sy.size(), DIRECT_THREADS, 0, cs>>>(dSY, dP, act, dPX, dPY, partY, ctx->dflags);
    else if (d == 2) k_batch_sum<1, 2><<<(unsigned)sy.size(), DIRECT_THREADS, 0, cs>>>(dSY, dP, act, dPX, dPY, partY, ctx->dflags);
    else k_batch_sum<1, 3><<<(unsigned)sy.size(), DIRECT_THREADS, 0, cs>>>(dSY, dP, act, dPX, dPY, partY, ctx->dflags);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  };
  auto sweep = [&](int sw) -> uotk_status {
    const int cur = sw & 1, nxt = cur ^ 1;
    {
      UOTK_PROF(ctx, cs, "weights");
      k_batch_weights<0><<<(unsigned)ey.size(), 256, 0, cs>>>(dEY, dP, act, ref == 0 ? b : nullptr,
                                                             gamma, slots, SL_MAXG0 + cur, dPY);
    }
    UOTK_LAUNCHED(ctx);
    UOTK_TRY(sum_x());
    {
      UOTK_PROF(ctx, cs, "dual_update");
      k_batch_update<0><<<(unsigned)ex.size(), 256, 0, cs>>>(
          dEX, dP, act, partX, a, ref, slots, SL_MAXG0 + cur, SL_MAXB0 + cur, SL_MAXG0 + nxt,
          track ? SL_DELTA0 + cur : -1, track ? SL_DELTA0 + nxt : -1, beta, nullptr,
          ctx->dflags);
    }
    UOTK_LAUNCHED(ctx);
    {
      UOTK_PROF(ctx, cs, "weights");
      k_batch_weights<1><<<(unsigned)ex.size(), 256, 0, cs>>>(dEX, dP, act, ref == 0 ? a : nullptr,
                                                             beta, slots, SL_MAXB0 + cur, dPX);
    }
    UOTK_LAUNCHED(ctx);
    UOTK_TRY(sum_y());
    {
      UOTK_PROF(ctx, cs, "dual_update");
      k_batch_update<1><<<(unsigned)ey.size(), 256, 0, cs>>>(
          dEY, dP, act, partY, b, ref, slots, SL_MAXB0 + cur, SL_MAXG0 + nxt, SL_MAXB0 + nxt,
          track ? SL_DELTA0 + cur : -1, -1, gamma, ty, ctx->dflags);
    }
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  };

  std::vector<int> sweeps(npairs, 0), host_act(npairs, 1);
  std::vector<long long> host_slots((size_t)npairs * SL_COUNT);
  int remaining = npairs;
  // Retire the pairs whose last change is below tol (after `done` sweeps).
  auto check = [&](int done) -> uotk_status {
    UOTK_CUDA(ctx, cudaMemcpyAsync(host_slots.data(), slots,
                                   sizeof(long long) * host_slots.size(),
                                   cudaMemcpyDeviceToHost, s));
    UOTK_CUDA(ctx, cudaStreamSynchronize(s));
    const int par = (done - 1) & 1;
    bool changed = false;
    for (int p = 0; p < npairs; ++p) {
      if (!host_act[p]) continue;
      const double dl = ordered_to_dbl(host_slots[(size_t)p * SL_COUNT + SL_DELTA0 + par]);
      if (dl < tol) {
        host_act[p] = 0;
        sweeps[p] = done;
        --remaining;
        changed = true;
      }
    }
    if (changed) {
      UOTK_TRY(upload(ctx, s, act, host_act));
      UOTK_CUDA(ctx, cudaStreamSynchronize(s));  // host_act is reused
    }
    return UOTK_OK;
  };

  int done = 0;
  UOTK_TRY(sweep(0));
  done = 1;
  uotk_status st = UOTK_OK;
  if (!ctx->prof.on && max_sweeps >= 3) {
    // The loop on the device: WHILE (condition) { sweep; sweep; control }.
    const int init[2] = {done, npairs};
    int* hstate = reinterpret_cast<int*>(ctx->host);
    memcpy(hstate, init, sizeof(init));
    UOTK_CUDA(ctx, cudaMemcpyAsync(state, hstate, sizeof(init), cudaMemcpyHostToDevice, s));
    UOTK_CUDA(ctx, cudaMemsetAsync(dsw, 0, sizeof(int) * npairs, s));
    UOTK_TRY(stream_fence(ctx, s, ctx->gs, ctx->fence_in));
    cs = ctx->gs;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaGraphConditionalHandle cond;
    UOTK_CUDA(ctx, cudaGraphCreate(&graph, 0));
    cudaError_t ce = cudaGraphConditionalHandleCreate(&cond, graph, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = cond;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    if (ce == cudaSuccess) ce = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np);
    const int64_t l0 = ctx->launches;
    int64_t body_launches = 0;
    if (ce == cudaSuccess) {
      cudaGraph_t body = np.conditional.phGraph_out[0];
      ce = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0,
                                         cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        uotk_status cst = sweep(1);
        if (cst == UOTK_OK) cst = sweep(2);
        if (cst == UOTK_OK) {
          k_batch_control<<<1, 256, 0, cs>>>(npairs, act, dsw, slots, state, tol, max_sweeps,
                                             cond);
          if (cudaGetLastError() != cudaSuccess) cst = UOTK_ERR_CUDA;
          else ctx->launches++;
        }
        const cudaError_t ec = cudaStreamEndCapture(cs, &body);
        if (cst != UOTK_OK || ec != cudaSuccess) ce = cudaErrorUnknown;
      }
      body_launches = ctx->launches - l0;
    }
    ctx->launches = l0;
    if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce == cudaSuccess) ce = cudaGraphLaunch(exec, cs);
    if (exec) cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
      cudaGetLastError();
      return set_error(ctx, UOTK_ERR_CUDA, "uot_sinkhorn_batch: device sweep loop failed: %s",
                       cudaGetErrorString(ce));
    }
    // one read-back after the loop: sweeps done, per-pair retirement counts
    UOTK_CUDA(ctx, cudaMemcpyAsync(hstate, state, 2 * sizeof(int), cudaMemcpyDeviceToHost, cs));
    UOTK_CUDA(ctx, cudaMemcpyAsync(sweeps.data(), dsw, sizeof(int) * npairs,
                                   cudaMemcpyDeviceToHost, cs));
    UOTK_CUDA(ctx, cudaMemcpyAsync(host_act.data(), act, sizeof(int) * npairs,
                                   cudaMemcpyDeviceToHost, cs));
    UOTK_CUDA(ctx, cudaStreamSynchronize(cs));
    UOTK_TRY(stream_fence(ctx, cs, s, ctx->fence_out));
    cs = s;
    const int bodies = (hstate[0] - done) / 2;
    ctx->launches += (int64_t)bodies * body_launches;
    done = hstate[0];
    remaining = hstate[1];
    // an odd remainder of the cap: the last sweep eagerly, then its check
    if (remaining > 0 && done < max_sweeps) {
      UOTK_TRY(sweep(done));
      done += 1;
      if (track) UOTK_TRY(check(done));
    }
  } else {
    int next_check = 10;
    while (done < max_sweeps && remaining > 0) {
      st = sweep(done);
      if (st != UOTK_OK) break;
      done += 1;
      if (track && (done >= next_check || done == max_sweeps)) {
        next_check = done + 10;
        st = check(done);
        if (st != UOTK_OK) break;
      }
    }
  }
  UOTK_TRY(st);
  if (track && done == 1 && max_sweeps == 1) UOTK_TRY(check(done));
  for (int p = 0; p < npairs; ++p)
    if (host_act[p]) sweeps[p] = done;

  // ---- per-pair dual values, Eq. (dual_euot) ----
  std::vector<int> lp(npairs);
  for (int p = 0; p < npairs; ++p) lp[p] = (sweeps[p] - 1) & 1;
  UOTK_TRY(upload(ctx, s, lastpar, lp));
  k_batch_values<<<npairs, 256, 0, s>>>(dP, a, b, beta, gamma, ty, slots, lastpar, ref, vals);
  UOTK_LAUNCHED(ctx);
  std::vector<double> hv((size_t)npairs * 5);
  UOTK_CUDA(ctx, cudaMemcpyAsync(hv.data(), vals, sizeof(double) * hv.size(),
                                 cudaMemcpyDeviceToHost, s));
  UOTK_TRY(flags_check(ctx, s, "uot_sinkhorn_batch"));
  for (int p = 0; p < npairs; ++p) {
    const double* h = &hv[(size_t)p * 5];
    double coupling = h[4];
    if (ref == 0) coupling -= h[2] * h[3];
    if (values_all)
      values_all[orig[p]] = -P[p].eta1 * h[0] - P[p].eta2 * h[1] + P[p].eta1 * h[2] +
                            P[p].eta2 * h[3] - coupling / P[p].lam;
    if (sweeps_done_all) sweeps_done_all[orig[p]] = sweeps[p];
  }
  if (track && remaining > 0)
    return set_error(ctx, UOTK_ERR_NOT_CONVERGED,
                     "uot_sinkhorn_batch: %d of %d pairs did not reach tol %g in %d sweeps",
                     remaining, npairs, tol, max_sweeps);
  return UOTK_OK;
}

}  // namespace uotk
