// Exact direct kernel summation, the matrix-vector product of Alg. 1 without
// ever forming the Gibbs matrix k_ij = exp(-||x_i - y_j||^2/eps):
//
//   out_j = sum_i w_i * 2^{-c ||s_i - t_j||^2},   c = log2(e)/eps.
//
// Design (d <= 3): sources packed as float4 (x, y, z, w); each CTA keeps
// DIRECT_THREADS*R targets in registers and streams source tiles of
// DIRECT_TILE float4 through shared memory with 1-D bulk copies (TMA,
// cp.async.bulk) completing on mbarriers.  Every thread reads a source with one
// broadcast shared load and evaluates R pairs: 3 FADD + 1 FMUL + 2 FFMA for the
// squared distance in unscaled coordinates (x - y is exact to half an ulp of
// the difference), 1 FMUL by -c, one MUFU ex2, 1 FFMA into the accumulator.
// FP32 partial sums over 32 sources are folded into a Neumaier-compensated
// (hi, lo) pair.  Sources are split across blockIdx.y when there are too few
// target blocks to fill the GPU; split partials are added in FP64 in a fixed
// order, so the result is deterministic.
#include <math.h>

#include <mutex>

#include "direct_body.cuh"

namespace uotk {

namespace {

constexpr int GEN_TILE = 64;  // sources per tile on the general-d path

template <int D, int R, int KIND = 0>
__global__ void __launch_bounds__(DIRECT_THREADS)
    k_direct_small(const float4* __restrict__ src, long long tiles, int tiles_per_split,
                   const float4* __restrict__ tgt, long long m, float neg_c,
                   float* __restrict__ out, long long* __restrict__ flags, float c1 = 0.f) {
  const long long t_begin = (long long)blockIdx.y * tiles_per_split;
  const long long t_end = min(t_begin + (long long)tiles_per_split, tiles);
  const int count = t_end > t_begin ? (int)(t_end - t_begin) : 0;
  direct_body<D, R, KIND>(src, t_begin, count, tgt, m,
                          (long long)blockIdx.x * (DIRECT_THREADS * R), neg_c, c1,
                          out + (long long)blockIdx.y * m, flags);
}

// General dimension: packed points of dp floats (coordinates, zeros, weight last).
template <int DMAX, int KIND = 0>
__global__ void __launch_bounds__(DIRECT_THREADS)
    k_direct_general(const float* __restrict__ src, long long tiles, int tiles_per_split,
                     const float* __restrict__ tgt, long long m, int d, int dp, float neg_c,
                     float* __restrict__ out, float c1 = 0.f) {
  extern __shared__ float gs[];  // [GEN_TILE][dp]
  const int tid = threadIdx.x;
  const long long j = (long long)blockIdx.x * DIRECT_THREADS + tid;
  float tc[DMAX];
#pragma unroll
  for (int t = 0; t < DMAX; ++t) tc[t] = (j < m && t < d) ? tgt[j * dp + t] : 0.f;
  const long long t_begin = (long long)blockIdx.y * tiles_per_split;
  const long long t_end = min(t_begin + (long long)tiles_per_split, tiles);
  float hi = 0.f, lo = 0.f;
  for (long long tile = t_begin; tile < t_end; ++tile) {
    __syncthreads();
    const float* g = src + tile * GEN_TILE * dp;
    for (int q = tid; q < GEN_TILE * dp; q += DIRECT_THREADS) gs[q] = g[q];
    __syncthreads();
    for (int i0 = 0; i0 < GEN_TILE; i0 += 32) {
      float acc = 0.f;
      for (int i = i0; i < i0 + 32; ++i) {
        const float* p = gs + i * dp;
        float r2 = 0.f;
#pragma unroll
        for (int t = 0; t < DMAX; ++t)
          if (t < d) { const float u = tc[t] - p[t]; r2 = fmaf(u, u, r2); }
        acc = fmaf(p[dp - 1], kpair<KIND>(r2, neg_c, c1), acc);
      }
      neumaier(hi, lo, acc);
    }
  }
  if (j < m) out[(long long)blockIdx.y * m + j] = hi + lo;
}

__global__ void k_reduce_splits(const float* __restrict__ part, int splits, long long m,
                                float* __restrict__ out) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
       j += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += (double)part[(long long)k * m + j];
    out[j] = (float)s;
  }
}

__device__ __forceinline__ void count_flags(long long* flags, bool neg, bool nonfinite) {
  const unsigned bn = __ballot_sync(0xffffffffu, neg);
  const unsigned bf = __ballot_sync(0xffffffffu, nonfinite);
  if ((threadIdx.x & 31) == 0) {
    if (bn) flag_add(&flags[FLAG_NEG_WEIGHT], (long long)__popc(bn));
    if (bf) flag_add(&flags[FLAG_NONFINITE], (long long)__popc(bf));
  }
}

// Sources: float4 (x, y, z, w) for d <= 3, or dp floats; rows >= n are zero.
__global__ void k_pack(const float* __restrict__ pts, const float* __restrict__ w, long long n,
                       long long n_pad, int d, int dp, int small, void* __restrict__ packed,
                       long long* __restrict__ flags) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  // every lane of a warp runs the same number of iterations (for the ballots)
  const long long iters = (n_pad + stride - 1) / stride;
  for (long long it = 0; it < iters; ++it) {
    const long long i = start + it * stride;
    bool neg = false, bad = false;
    if (i < n_pad) {
      if (small) {
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < n) {
          p.x = pts[i * d];
          if (d > 1) p.y = pts[i * d + 1];
          if (d > 2) p.z = pts[i * d + 2];
          p.w = w ? w[i] : 0.f;
          bad = !isfinite(p.x) || !isfinite(p.y) || !isfinite(p.z) || !isfinite(p.w);
          neg = p.w < 0.f;
        }
        reinterpret_cast<float4*>(packed)[i] = p;
      } else {
        float* o = reinterpret_cast<float*>(packed) + i * dp;
        for (int t = 0; t < dp; ++t) {
          float v = 0.f;
          if (i < n) {
            if (t < d) v = pts[i * d + t];
            else if (t == dp - 1 && w) v = w[i];
            bad |= !isfinite(v);
          }
          o[t] = v;
        }
        if (i < n && w) neg = w[i] < 0.f;
      }
    }
    count_flags(flags, neg, bad);
  }
}

// Source weights of the packed points i < n_pad (padding rows: weight 0):
//   LOG = false: w_i = base_i * exp(lam*pot_i - shift)    (FP32)
//   LOG = true : w_i = log2(base_i) + (lam*pot_i - shift) log2(e)  (padding -inf)
// shift from the ordered slot (pot NULL: no potential; base NULL: 1).
template <bool LOG>
__global__ void k_set_weights(void* __restrict__ packed, long long n, long long n_pad, int small,
                              int dp, const float* __restrict__ base,
                              const double* __restrict__ pot, double lam,
                              const long long* __restrict__ shift_slot) {
  const double shift = pot ? ordered_to_dbl(*shift_slot) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
       i += (long long)gridDim.x * blockDim.x) {
    float v;
    if (i >= n) {
      v = LOG ? -INFINITY : 0.f;
    } else if (LOG) {
      double lw = pot ? (lam * pot[i] - shift) * 1.4426950408889634 : 0.0;
      if (base) lw += log2((double)base[i]);
      v = (float)lw;
    } else {
      v = pot ? exp_shifted(lam * pot[i] - shift) : 1.f;
      if (base) v *= base[i];
    }
    if (small) reinterpret_cast<float4*>(packed)[i].w = v;
    else reinterpret_cast<float*>(packed)[i * dp + dp - 1] = v;
  }
}

// ---- per-row log-sum-exp form (log domain) ----
// out[j] = {M_j, S_j} with log2 sum_i 2^{lw_i - c ||s_i - t_j||^2} = M_j + log2 S_j:
// M_j the largest exponent seen, S_j >= 1 the sum scaled by 2^{-M_j} (M = -inf,
// S = 0 when no source contributes).  Sources carry lw = log2 of their weight
// in the weight slot.  Exponents of a chunk of 16 sources are formed first, the
// running sum is rescaled once per chunk when its maximum grows.
template <int R>
__device__ __forceinline__ void lse_fold(float (&a)[R][16], float (&M)[R], float (&hi)[R],
                                         float (&lo)[R]) {
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float cm = a[r][0];
#pragma unroll
    for (int j = 1; j < 16; ++j) cm = fmaxf(cm, a[r][j]);
    const float mn = fmaxf(M[r], cm);
    if (mn == -INFINITY) continue;
    if (mn > M[r]) {
      const float f = ex2_approx(M[r] - mn);  // 0 while M = -inf
      hi[r] *= f;
      lo[r] *= f;
      M[r] = mn;
    }
    float acc = 0.f;
#pragma unroll
    for (int j = 0; j < 16; ++j) acc += ex2_approx(a[r][j] - mn);
    neumaier(hi[r], lo[r], acc);
  }
}

template <int D, int R>
__global__ void __launch_bounds__(DIRECT_THREADS)
    k_direct_lse(const float4* __restrict__ src, long long tiles, int tiles_per_split,
                 const float4* __restrict__ tgt, long long m, float neg_c,
                 float2* __restrict__ out, long long* __restrict__ flags) {
  __shared__ __align__(128) float4 sm[STAGES][DIRECT_TILE];
  __shared__ __align__(8) unsigned long long bar[STAGES];
  const int tid = threadIdx.x;
  const long long tb = (long long)blockIdx.x * (DIRECT_THREADS * R) + tid;

  float tx[R], ty[R], tz[R], M[R], hi[R], lo[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long j = tb + (long long)r * DIRECT_THREADS;
    const float4 p = j < m ? tgt[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    tx[r] = p.x; ty[r] = p.y; tz[r] = p.z;
    M[r] = -INFINITY; hi[r] = 0.f; lo[r] = 0.f;
  }

  const long long t_begin = (long long)blockIdx.y * tiles_per_split;
  const long long t_end = min(t_begin + (long long)tiles_per_split, tiles);
  const int count = t_end > t_begin ? (int)(t_end - t_begin) : 0;
  constexpr unsigned BYTES = DIRECT_TILE * sizeof(float4);

  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < STAGES && s < count; ++s)
      { mbar_expect(&bar[s], BYTES); bulk_copy(sm[s], src + (t_begin + s) * DIRECT_TILE, BYTES, &bar[s]); }
  }

  for (int k = 0; k < count; ++k) {
    const int s = k % STAGES;
    const bool ok = mbar_wait(&bar[s], (unsigned)(k / STAGES) & 1u);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        flag_add(&flags[FLAG_TIMEOUT], 1LL);
        for (int q = k; q < count && q < k + STAGES; ++q)
          mbar_wait(&bar[q % STAGES], (unsigned)(q / STAGES) & 1u);
      }
      return;
    }
    const float4* T = sm[s];
#pragma unroll 1
    for (int j0 = 0; j0 < DIRECT_TILE; j0 += 16) {
      float a[R][16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float4 q = T[j0 + j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float dx = tx[r] - q.x;
          float r2 = dx * dx;
          if (D > 1) { const float dy = ty[r] - q.y; r2 = fmaf(dy, dy, r2); }
          if (D > 2) { const float dz = tz[r] - q.z; r2 = fmaf(dz, dz, r2); }
          a[r][j] = fmaf(r2, neg_c, q.w);
        }
      }
      lse_fold<R>(a, M, hi, lo);
    }
    __syncthreads();
    if (tid == 0 && k + STAGES < count)
      { mbar_expect(&bar[s], BYTES); bulk_copy(sm[s], src + (t_begin + k + STAGES) * DIRECT_TILE, BYTES, &bar[s]); }
  }

  float2* o = out + (long long)blockIdx.y * m;
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long j = tb + (long long)r * DIRECT_THREADS;
    if (j < m) o[j] = make_float2(M[r], hi[r] + lo[r]);
  }
}

// General dimension, log domain (packed points of dp floats, log-weight last).
template <int DMAX>
__global__ void __launch_bounds__(DIRECT_THREADS)
    k_direct_general_lse(const float* __restrict__ src, long long tiles, int tiles_per_split,
                         const float* __restrict__ tgt, long long m, int d, int dp, float neg_c,
                         float2* __restrict__ out) {
  extern __shared__ float gs[];  // [GEN_TILE][dp]
  const int tid = threadIdx.x;
  const long long j = (long long)blockIdx.x * DIRECT_THREADS + tid;
  float tc[DMAX];
#pragma unroll
  for (int t = 0; t < DMAX; ++t) tc[t] = (j < m && t < d) ? tgt[j * dp + t] : 0.f;
  const long long t_begin = (long long)blockIdx.y * tiles_per_split;
  const long long t_end = min(t_begin + (long long)tiles_per_split, tiles);
  float M[1] = {-INFINITY}, hi[1] = {0.f}, lo[1] = {0.f};
  for (long long tile = t_begin; tile < t_end; ++tile) {
    __syncthreads();
    const float* g = src + tile * GEN_TILE * dp;
    for (int q = tid; q < GEN_TILE * dp; q += DIRECT_THREADS) gs[q] = g[q];
    __syncthreads();
    for (int i0 = 0; i0 < GEN_TILE; i0 += 16) {
      float a[1][16];
      for (int i = 0; i < 16; ++i) {
        const float* p = gs + (i0 + i) * dp;
        float r2 = 0.f;
#pragma unroll
        for (int t = 0; t < DMAX; ++t)
          if (t < d) { const float u = tc[t] - p[t]; r2 = fmaf(u, u, r2); }
        a[0][i] = fmaf(r2, neg_c, p[dp - 1]);
      }
      lse_fold<1>(a, M, hi, lo);
    }
  }
  if (j < m) out[(long long)blockIdx.y * m + j] = make_float2(M[0], hi[0] + lo[0]);
}

// Split partials {M_k, S_k} -> {M, S}: M = max M_k, S = sum S_k 2^{M_k - M} (FP64).
__global__ void k_reduce_splits_lse(const float2* __restrict__ part, int splits, long long m,
                                    float2* __restrict__ out) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
       j += (long long)gridDim.x * blockDim.x) {
    float mx = -INFINITY;
    for (int k = 0; k < splits; ++k) mx = fmaxf(mx, part[(long long)k * m + j].x);
    double s = 0.0;
    if (mx > -INFINITY)
      for (int k = 0; k < splits; ++k) {
        const float2 v = part[(long long)k * m + j];
        if (v.x > -INFINITY) s += (double)v.y * exp2((double)v.x - (double)mx);
      }
    out[j] = make_float2(mx, (float)s);
  }
}

}  // namespace

int grid_for(const uotk_ctx* ctx, int64_t work, int threads, int per_sm) {
  const int64_t want = (work + threads - 1) / threads;
  const int64_t cap = (int64_t)ctx->num_sms * per_sm;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

DirectLayout direct_layout(const uotk_ctx* ctx, int d, int64_t n, int64_t m, int force_r) {
  DirectLayout L;
  L.d = d;
  L.n = n;
  L.m = m;
  const bool small = d <= 3;
  const int tile = small ? DIRECT_TILE : GEN_TILE;
  // targets per thread: enough CTAs to fill the GPU with the most reuse of each
  // staged source (2 and 4 take the packed FP32x2 path of the Gaussian)
  const int64_t per_wave = (int64_t)DIRECT_THREADS * ctx->num_sms;
  L.reg_targets = !small ? 1 : (m >= 4 * per_wave ? 4 : (m >= 2 * per_wave ? 2 : 1));
  if (force_r > 0) L.reg_targets = force_r;
  L.blocks_x = (int)((m + (int64_t)DIRECT_THREADS * L.reg_targets - 1) /
                     ((int64_t)DIRECT_THREADS * L.reg_targets));
  if (L.blocks_x < 1) L.blocks_x = 1;
  L.tiles = (n + tile - 1) / tile;
  const int64_t want = 32LL * ctx->num_sms;  // ~8 waves of 4 resident CTAs per SM
  int64_t splits = (want + L.blocks_x - 1) / L.blocks_x;
  int64_t max_splits = L.tiles / 2 > 0 ? L.tiles / 2 : 1;
  if (splits > max_splits) splits = max_splits;
  if (splits > 65535) splits = 65535;
  if (splits < 1) splits = 1;
  L.tiles_per_split = (int)((L.tiles + splits - 1) / splits);
  if (L.tiles_per_split < 1) L.tiles_per_split = 1;
  L.splits = (int)((L.tiles + L.tiles_per_split - 1) / L.tiles_per_split);
  if (L.splits < 1) L.splits = 1;
  L.dp = small ? 4 : ((d + 1 + 3) / 4) * 4;
  const int64_t n_pad = L.tiles * tile;
  L.src_bytes = (size_t)n_pad * L.dp * sizeof(float);
  L.tgt_bytes = (size_t)(m > 0 ? m : 1) * L.dp * sizeof(float);
  L.part_bytes = L.splits > 1 ? (size_t)L.splits * m * sizeof(float) : 0;
  return L;
}

void direct_carve(Carver& cv, const DirectLayout& L, DirectBufs& b) {
  b.src = cv.take<char>(L.src_bytes > 0 ? L.src_bytes : 16);
  b.tgt = cv.take<char>(L.tgt_bytes);
  b.part = L.part_bytes ? cv.take<float>(L.part_bytes / sizeof(float)) : nullptr;
}

uotk_status direct_pack_sources(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                                const float* pts, const float* w, void* packed) {
  const int tile = L.d <= 3 ? DIRECT_TILE : GEN_TILE;
  const int64_t n_pad = L.tiles * tile;
  if (n_pad == 0) return UOTK_OK;
  UOTK_PROF(ctx, s, "pack");
  k_pack<<<grid_for(ctx, n_pad, 256), 256, 0, s>>>(pts, w, L.n, n_pad, L.d, L.dp, L.d <= 3,
                                                   packed, ctx->dflags);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status direct_pack_targets(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                                const float* pts, void* packed) {
  if (L.m == 0) return UOTK_OK;
  UOTK_PROF(ctx, s, "pack");
  k_pack<<<grid_for(ctx, L.m, 256), 256, 0, s>>>(pts, nullptr, L.m, L.m, L.d, L.dp, L.d <= 3,
                                                 packed, ctx->dflags);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status direct_set_weights(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                               void* packed, const float* base, const double* pot, double lam,
                               const long long* shift_slot, bool log2_weights) {
  if (L.n == 0) return UOTK_OK;
  UOTK_PROF(ctx, s, "weights");
  const int64_t n_pad = L.tiles * (L.d <= 3 ? DIRECT_TILE : GEN_TILE);
  if (log2_weights)
    k_set_weights<true><<<grid_for(ctx, n_pad, 256), 256, 0, s>>>(
        packed, L.n, n_pad, L.d <= 3, L.dp, base, pot, lam, shift_slot);
  else
    k_set_weights<false><<<grid_for(ctx, n_pad, 256), 256, 0, s>>>(
        packed, L.n, n_pad, L.d <= 3, L.dp, base, pot, lam, shift_slot);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

template <int KIND>
void direct_launch(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L, const DirectBufs& b,
                   float c0, float c1, float* dst) {
  const dim3 grid(L.blocks_x, L.splits);
  if (L.d <= 3) {
    const float4* src = reinterpret_cast<const float4*>(b.src);
    const float4* tgt = reinterpret_cast<const float4*>(b.tgt);
#define UOTK_DIRECT_CASE(DD, RR)                                                          \
  if (L.d == DD && L.reg_targets == RR)                                                   \
    k_direct_small<DD, RR, KIND><<<grid, DIRECT_THREADS, 0, s>>>(                         \
        src, L.tiles, L.tiles_per_split, tgt, L.m, c0, dst, ctx->dflags, c1);
    UOTK_DIRECT_CASE(1, 1) UOTK_DIRECT_CASE(1, 2) UOTK_DIRECT_CASE(1, 4)
    UOTK_DIRECT_CASE(2, 1) UOTK_DIRECT_CASE(2, 2) UOTK_DIRECT_CASE(2, 4)
    UOTK_DIRECT_CASE(3, 1) UOTK_DIRECT_CASE(3, 2) UOTK_DIRECT_CASE(3, 4)
#undef UOTK_DIRECT_CASE
  } else {
    const float* src = reinterpret_cast<const float*>(b.src);
    const float* tgt = reinterpret_cast<const float*>(b.tgt);
    const size_t smem = (size_t)GEN_TILE * L.dp * sizeof(float);
#define UOTK_DIRECT_GEN(DM)                                                                   \
  k_direct_general<DM, KIND><<<grid, DIRECT_THREADS, smem, s>>>(src, L.tiles, L.tiles_per_split, \
                                                                 tgt, L.m, L.d, L.dp, c0, dst, c1);
    if (L.d <= 8) { UOTK_DIRECT_GEN(8) }
    else if (L.d <= 16) { UOTK_DIRECT_GEN(16) }
    else if (L.d <= 32) { UOTK_DIRECT_GEN(32) }
    else if (L.d <= 64) { UOTK_DIRECT_GEN(64) }
    else { UOTK_DIRECT_GEN(128) }
#undef UOTK_DIRECT_GEN
  }
}

uotk_status direct_run(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L, const DirectBufs& b,
                       double eps, float* out, int kernel) {
  if (L.m == 0) return UOTK_OK;
  if (L.n == 0) {
    UOTK_CUDA(ctx, cudaMemsetAsync(out, 0, sizeof(float) * L.m, s));
    return UOTK_OK;
  }
  // eps: the Gaussian width, or the parameter p of the other kernels
  const float c0 = (float)(-1.4426950408889634 / eps);
  const float c1 = (float)(eps * eps);
  float* dst = L.splits > 1 ? b.part : out;
  {
    UOTK_PROF(ctx, s, "direct");
    switch (kernel) {
      case UOTK_KERNEL_LAPLACE: direct_launch<1>(ctx, s, L, b, c0, c1, dst); break;
      case UOTK_KERNEL_IMQ: direct_launch<2>(ctx, s, L, b, c0, c1, dst); break;
      case UOTK_KERNEL_ENERGY: direct_launch<3>(ctx, s, L, b, c0, c1, dst); break;
      default: direct_launch<0>(ctx, s, L, b, c0, c1, dst); break;
    }
  }
  UOTK_LAUNCHED(ctx);
  if (L.splits > 1) {
    UOTK_PROF(ctx, s, "split_reduce");
    k_reduce_splits<<<grid_for(ctx, L.m, 256), 256, 0, s>>>(b.part, L.splits, L.m, out);
    UOTK_LAUNCHED(ctx);
  }
  return UOTK_OK;
}

uotk_status direct_run_lse(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                           const DirectBufs& b, double eps, float2* out) {
  if (L.m == 0) return UOTK_OK;
  if (L.n == 0) return set_error(ctx, UOTK_ERR_INVALID, "log-domain sum with no sources");
  const float neg_c = (float)(-1.4426950408889634 / eps);
  float2* part = reinterpret_cast<float2*>(b.part);
  float2* dst = L.splits > 1 ? part : out;
  const dim3 grid(L.blocks_x, L.splits);
  {
    UOTK_PROF(ctx, s, "direct_lse");
    if (L.d <= 3) {
      const float4* src = reinterpret_cast<const float4*>(b.src);
      const float4* tgt = reinterpret_cast<const float4*>(b.tgt);
#define UOTK_LSE_CASE(DD, RR)                                                             \
  if (L.d == DD && L.reg_targets == RR)                                                   \
    k_direct_lse<DD, RR><<<grid, DIRECT_THREADS, 0, s>>>(src, L.tiles, L.tiles_per_split,  \
                                                         tgt, L.m, neg_c, dst, ctx->dflags);
      UOTK_LSE_CASE(1, 1) UOTK_LSE_CASE(1, 2) UOTK_LSE_CASE(1, 4)
      UOTK_LSE_CASE(2, 1) UOTK_LSE_CASE(2, 2) UOTK_LSE_CASE(2, 4)
      UOTK_LSE_CASE(3, 1) UOTK_LSE_CASE(3, 2) UOTK_LSE_CASE(3, 4)
#undef UOTK_LSE_CASE
    } else {
      const float* src = reinterpret_cast<const float*>(b.src);
      const float* tgt = reinterpret_cast<const float*>(b.tgt);
      const size_t smem = (size_t)GEN_TILE * L.dp * sizeof(float);
#define UOTK_LSE_GEN(DM)                                                                      \
  k_direct_general_lse<DM><<<grid, DIRECT_THREADS, smem, s>>>(src, L.tiles, L.tiles_per_split, \
                                                               tgt, L.m, L.d, L.dp, neg_c, dst);
      if (L.d <= 8) { UOTK_LSE_GEN(8) }
      else if (L.d <= 16) { UOTK_LSE_GEN(16) }
      else if (L.d <= 32) { UOTK_LSE_GEN(32) }
      else if (L.d <= 64) { UOTK_LSE_GEN(64) }
      else { UOTK_LSE_GEN(128) }
#undef UOTK_LSE_GEN
    }
  }
  UOTK_LAUNCHED(ctx);
  if (L.splits > 1) {
    UOTK_PROF(ctx, s, "split_reduce");
    k_reduce_splits_lse<<<grid_for(ctx, L.m, 256), 256, 0, s>>>(part, L.splits, L.m, out);
    UOTK_LAUNCHED(ctx);
  }
  return UOTK_OK;
}

}  // namespace uotk

// ---------------------------------------------------------------------------
// Direct kernel summation without any allocation (uotk_kernel_sum_noalloc).
//
// For callers that must not allocate device memory at call time.  Examples
// are a service that reserves all of its memory when it starts and treats
// any later cudaMalloc as an error, or code that runs where an allocation
// would synchronise the device or could fail under memory pressure.  The
// scratch these calls need (packed points, split partial sums, validation
// counters) lives in one file-scope device array, reserved when the library
// is loaded on a device and kept until the process exits.
// ---------------------------------------------------------------------------
namespace uotk {
namespace {

constexpr long long NOALLOC_MAX_POINTS = 65536;  // per cloud (sources, targets)
constexpr int NOALLOC_MAX_SPLITS = 8;
constexpr size_t NOALLOC_SRC_BYTES =
    (size_t)(NOALLOC_MAX_POINTS + DIRECT_TILE) * sizeof(float4);            // 1 MiB + 4 KiB
constexpr size_t NOALLOC_TGT_BYTES = (size_t)NOALLOC_MAX_POINTS * sizeof(float4);  // 1 MiB
constexpr size_t NOALLOC_PART_BYTES =
    (size_t)NOALLOC_MAX_SPLITS * NOALLOC_MAX_POINTS * sizeof(float);        // 2 MiB
constexpr size_t NOALLOC_FLAG_BYTES = 256;
constexpr size_t NOALLOC_BYTES =
    NOALLOC_SRC_BYTES + NOALLOC_TGT_BYTES + NOALLOC_PART_BYTES + NOALLOC_FLAG_BYTES;

// The scratch itself.  In host code `noalloc_scratch` names a host-side
// stand-in, not the device memory: its device address is looked up once per
// device with cudaGetSymbolAddress and passed to the kernels.
static __device__ __align__(256) unsigned char noalloc_scratch[NOALLOC_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex noalloc_mutex;
unsigned char* noalloc_ptr[NOALLOC_MAX_DEVICES] = {};

// Device address of the scratch on the current device (set-up on first use).
uotk_status noalloc_scratch_on(int dev, unsigned char** out) {
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return UOTK_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(noalloc_mutex);
  if (!noalloc_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return UOTK_ERR_CUDA;
    }
    noalloc_ptr[dev] = static_cast<unsigned char*>(p);
  }
  *out = noalloc_ptr[dev];
  return UOTK_OK;
}

}  // namespace


// ---------------------------------------------------------------------------
// Several right-hand sides over the same pairs (the coordinate sums of the
// gradients): out_k[j] = sum_i w_k[i] exp(-|s_i - t_j|^2/eps), k < K <= 4,
// Gaussian, d <= 3.  The distance and the exponential of a pair are computed
// once for all K sums: 7 + K FP32 operations per pair instead of 8 K.
// ---------------------------------------------------------------------------
namespace {

constexpr int MULTI_R = 2;   // targets per thread

// w4[i] = {b_0[i], .., b_3[i]} * f_i, f_i = exp(lam pot_i - shift) (pot != NULL;
// shift from its ordered-int64 slot) or 1; zero beyond n.
__global__ void k_pack_w4(const float* __restrict__ w0, const float* __restrict__ w1,
                          const float* __restrict__ w2, const float* __restrict__ w3,
                          const double* __restrict__ pot, double lam,
                          const long long* __restrict__ shift_slot, long long n,
                          long long n_pad, float4* __restrict__ out) {
  const double shift = pot ? ordered_to_dbl(*shift_slot) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
       i += (long long)gridDim.x * blockDim.x) {
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i < n) {
      const float f = pot ? exp_shifted(lam * pot[i] - shift) : 1.f;
      v.x = w0 ? w0[i] * f : 0.f;
      v.y = w1 ? w1[i] * f : 0.f;
      v.z = w2 ? w2[i] * f : 0.f;
      v.w = w3 ? w3[i] * f : 0.f;
    }
    out[i] = v;
  }
}

// Sources: positions (the packed source tiles; their weight lane is ignored)
// and weights {w_0..w_3}, both staged per tile by bulk copies into a 3-stage
// ring; partial sums to part[(k splits + split) m + j].
template <int D, int K>
__global__ void __launch_bounds__(DIRECT_THREADS)
    k_direct_multi(const float4* __restrict__ src, const float4* __restrict__ wsrc,
                   long long tiles, int tiles_per_split, const float4* __restrict__ tgt,
                   long long m, float neg_c, int splits, float* __restrict__ part,
                   long long* __restrict__ flags) {
  constexpr int R = MULTI_R;
  __shared__ __align__(128) float4 sp[STAGES][DIRECT_TILE];
  __shared__ __align__(128) float4 sw[STAGES][DIRECT_TILE];
  __shared__ __align__(8) unsigned long long bar[STAGES];
  const int tid = threadIdx.x;
  const long long t_begin = (long long)blockIdx.y * tiles_per_split;
  const long long t_end = min(t_begin + (long long)tiles_per_split, tiles);
  const int count = t_end > t_begin ? (int)(t_end - t_begin) : 0;
  const long long tb = (long long)blockIdx.x * (DIRECT_THREADS * R) + tid;
  float tx[R], ty[R], tz[R], hi[R][K], lo[R][K];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long j = tb + (long long)r * DIRECT_THREADS;
    const float4 p = j < m ? tgt[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    tx[r] = p.x; ty[r] = p.y; tz[r] = p.z;
#pragma unroll
    for (int k = 0; k < K; ++k) { hi[r][k] = 0.f; lo[r][k] = 0.f; }
  }
  constexpr unsigned BYTES = DIRECT_TILE * sizeof(float4);
  if (tid == 0) {
#pragma unroll
    for (int s = 0; s < STAGES; ++s) mbar_init(&bar[s], 1);
    mbar_fence_init();
  }
  __syncthreads();
  if (tid == 0) {
    for (int s = 0; s < STAGES && s < count; ++s) {
      mbar_expect(&bar[s], 2 * BYTES);
      bulk_copy(sp[s], src + (t_begin + s) * DIRECT_TILE, BYTES, &bar[s]);
      bulk_copy(sw[s], wsrc + (t_begin + s) * DIRECT_TILE, BYTES, &bar[s]);
    }
  }
  for (int kk = 0; kk < count; ++kk) {
    const int s = kk % STAGES;
    const bool ok = mbar_wait(&bar[s], (unsigned)(kk / STAGES) & 1u);
    if (__syncthreads_or(!ok)) {
      if (tid == 0) {
        flag_add(&flags[FLAG_TIMEOUT], 1LL);
        for (int q = kk; q < count && q < kk + STAGES; ++q)
          mbar_wait(&bar[q % STAGES], (unsigned)(q / STAGES) & 1u);
      }
      return;
    }
#pragma unroll 1
    for (int j0 = 0; j0 < DIRECT_TILE; j0 += 32) {
      float acc[R][K];
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < K; ++k) acc[r][k] = 0.f;
#pragma unroll 4
      for (int j = j0; j < j0 + 32; ++j) {
        const float4 q = sp[s][j];
        const float4 w4 = sw[s][j];
        const float wv[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const float dx = tx[r] - q.x;
          float r2 = dx * dx;
          if (D > 1) { const float dy = ty[r] - q.y; r2 = fmaf(dy, dy, r2); }
          if (D > 2) { const float dz = tz[r] - q.z; r2 = fmaf(dz, dz, r2); }
          const float e = ex2_approx(r2 * neg_c);
#pragma unroll
          for (int k = 0; k < K; ++k) acc[r][k] = fmaf(wv[k], e, acc[r][k]);
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int k = 0; k < K; ++k) neumaier(hi[r][k], lo[r][k], acc[r][k]);
    }
    __syncthreads();
    if (tid == 0 && kk + STAGES < count) {
      mbar_expect(&bar[s], 2 * BYTES);
      bulk_copy(sp[s], src + (t_begin + kk + STAGES) * DIRECT_TILE, BYTES, &bar[s]);
      bulk_copy(sw[s], wsrc + (t_begin + kk + STAGES) * DIRECT_TILE, BYTES, &bar[s]);
    }
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long j = tb + (long long)r * DIRECT_THREADS;
    if (j < m)
#pragma unroll
      for (int k = 0; k < K; ++k)
        part[((long long)k * splits + blockIdx.y) * m + j] = hi[r][k] + lo[r][k];
  }
}

// out_k[j] = sum over splits of part[(k splits + split) m + j], added in FP64 in split order.
__global__ void k_reduce_multi(const float* __restrict__ part, int splits, long long m, int K,
                               float* __restrict__ o0, float* __restrict__ o1,
                               float* __restrict__ o2, float* __restrict__ o3) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < (long long)K * m;
       i += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(i / m);
    const long long j = i - (long long)k * m;
    double acc = 0.0;
    for (int q = 0; q < splits; ++q) acc += (double)part[((long long)k * splits + q) * m + j];
    float* o = k == 0 ? o0 : (k == 1 ? o1 : (k == 2 ? o2 : o3));
    o[j] = (float)acc;
  }
}

}  // namespace

size_t direct_multi_bytes(const uotk_ctx* ctx, int d, int64_t n, int64_t m) {
  const DirectLayout L = direct_layout(ctx, d, n, m, MULTI_R);
  const size_t w4 = (size_t)(L.tiles * DIRECT_TILE > 0 ? L.tiles * DIRECT_TILE : 1) * sizeof(float4);
  return w4 + 256 + (size_t)4 * L.splits * (m > 0 ? m : 1) * sizeof(float) + 256;
}

uotk_status direct_run_multi(uotk_ctx* ctx, cudaStream_t s, int d, int64_t n, int64_t m,
                             const void* src_packed, const void* tgt_packed, int K,
                             const float* const* w, const double* pot, double lam,
                             const long long* shift_slot, void* scratch, double eps,
                             float* const* out) {
  if (m == 0) return UOTK_OK;
  if (d > 3 || K < 1 || K > 4) return set_error(ctx, UOTK_ERR_INTERNAL, "direct_run_multi: d %d K %d", d, K);
  if (n == 0) {
    for (int k = 0; k < K; ++k) UOTK_CUDA(ctx, cudaMemsetAsync(out[k], 0, sizeof(float) * m, s));
    return UOTK_OK;
  }
  const DirectLayout L = direct_layout(ctx, d, n, m, MULTI_R);
  const int64_t n_pad = L.tiles * DIRECT_TILE;
  Carver cv(reinterpret_cast<char*>(scratch));
  float4* w4 = cv.take<float4>(n_pad);
  float* part = cv.take<float>((size_t)4 * L.splits * m);
  const float* wk[4] = {nullptr, nullptr, nullptr, nullptr};
  for (int k = 0; k < K; ++k) wk[k] = w[k];
  {
    UOTK_PROF(ctx, s, "weights");
    k_pack_w4<<<grid_for(ctx, n_pad, 256), 256, 0, s>>>(wk[0], wk[1], wk[2], wk[3], pot, lam,
                                                        shift_slot, n, n_pad, w4);
    UOTK_LAUNCHED(ctx);
  }
  const float neg_c = (float)(-1.4426950408889634 / eps);
  const dim3 grid(L.blocks_x, L.splits);
  const float4* src = reinterpret_cast<const float4*>(src_packed);
  const float4* tgt = reinterpret_cast<const float4*>(tgt_packed);
  {
    UOTK_PROF(ctx, s, "direct_multi");
#define UOTK_MULTI_CASE(DD, KK)                                                              \
  if (d == DD && K == KK)                                                                    \
    k_direct_multi<DD, KK><<<grid, DIRECT_THREADS, 0, s>>>(src, w4, L.tiles, L.tiles_per_split, \
                                                           tgt, m, neg_c, L.splits, part,     \
                                                           ctx->dflags);
    UOTK_MULTI_CASE(1, 2) UOTK_MULTI_CASE(2, 2) UOTK_MULTI_CASE(2, 3)
    UOTK_MULTI_CASE(3, 2) UOTK_MULTI_CASE(3, 3) UOTK_MULTI_CASE(3, 4)
    UOTK_MULTI_CASE(1, 3) UOTK_MULTI_CASE(1, 4) UOTK_MULTI_CASE(2, 4)
    UOTK_MULTI_CASE(1, 1) UOTK_MULTI_CASE(2, 1) UOTK_MULTI_CASE(3, 1)
#undef UOTK_MULTI_CASE
  }
  UOTK_LAUNCHED(ctx);
  {
    UOTK_PROF(ctx, s, "split_reduce");
    k_reduce_multi<<<grid_for(ctx, (int64_t)K * m, 256), 256, 0, s>>>(
        part, L.splits, m, K, out[0], K > 1 ? out[1] : nullptr, K > 2 ? out[2] : nullptr,
        K > 3 ? out[3] : nullptr);
    UOTK_LAUNCHED(ctx);
  }
  return UOTK_OK;
}

}  // namespace uotk

extern "C" uotk_status uotk_kernel_sum_noalloc(void* stream, int d, const float* src, int64_t n,
                                               const float* w, const float* tgt, int64_t m,
                                               float* out, double eps) {
  using namespace uotk;
  if (d < 1 || d > 3) return UOTK_ERR_UNSUPPORTED;
  if (n < 0 || m < 0 || !(eps > 0.0) || !isfinite(eps)) return UOTK_ERR_INVALID;
  if (n > NOALLOC_MAX_POINTS || m > NOALLOC_MAX_POINTS) return UOTK_ERR_UNSUPPORTED;
  if ((n > 0 && (!src || !w)) || (m > 0 && (!tgt || !out))) return UOTK_ERR_INVALID;
  if (m == 0) return UOTK_OK;
  cudaStream_t s = (cudaStream_t)stream;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return UOTK_ERR_CUDA;
  }
  if (n == 0) {
    if (cudaMemsetAsync(out, 0, sizeof(float) * m, s) != cudaSuccess) return UOTK_ERR_CUDA;
    return UOTK_OK;
  }
  unsigned char* base = nullptr;
  const uotk_status st0 = noalloc_scratch_on(dev, &base);
  if (st0 != UOTK_OK) return st0;
  float4* psrc = reinterpret_cast<float4*>(base);
  float4* ptgt = reinterpret_cast<float4*>(base + NOALLOC_SRC_BYTES);
  float* part = reinterpret_cast<float*>(base + NOALLOC_SRC_BYTES + NOALLOC_TGT_BYTES);
  long long* flags =
      reinterpret_cast<long long*>(base + NOALLOC_SRC_BYTES + NOALLOC_TGT_BYTES + NOALLOC_PART_BYTES);
  // the same launch shape as the context path, with at most NOALLOC_MAX_SPLITS splits
  const int R = 1;
  const int blocks_x = (int)((m + DIRECT_THREADS - 1) / DIRECT_THREADS);
  const long long tiles = (n + DIRECT_TILE - 1) / DIRECT_TILE;
  long long splits = (32LL * sms + blocks_x - 1) / blocks_x;
  const long long max_splits = tiles / 2 > 0 ? tiles / 2 : 1;
  if (splits > max_splits) splits = max_splits;
  if (splits > NOALLOC_MAX_SPLITS) splits = NOALLOC_MAX_SPLITS;
  if (splits < 1) splits = 1;
  const int tps = (int)((tiles + splits - 1) / splits);
  splits = (tiles + tps - 1) / tps;
  // the validation counters start at zero on every call
  if (cudaMemsetAsync(flags, 0, NOALLOC_FLAG_BYTES, s) != cudaSuccess) return UOTK_ERR_CUDA;
  const long long n_pad = tiles * DIRECT_TILE;
  const int gp = (int)((n_pad + 255) / 256 < 8LL * sms ? (n_pad + 255) / 256 : 8LL * sms);
  k_pack<<<gp, 256, 0, s>>>(src, w, n, n_pad, d, 4, 1, psrc, flags);
  const int gt = (int)((m + 255) / 256 < 8LL * sms ? (m + 255) / 256 : 8LL * sms);
  k_pack<<<gt, 256, 0, s>>>(tgt, nullptr, m, m, d, 4, 1, ptgt, flags);
  const float neg_c = (float)(-1.4426950408889634 / eps);
  float* dst = splits > 1 ? part : out;
  const dim3 grid(blocks_x, (unsigned)splits);
  if (d == 1)
    k_direct_small<1, R><<<grid, DIRECT_THREADS, 0, s>>>(psrc, tiles, tps, ptgt, m, neg_c, dst, flags);
  else if (d == 2)
    k_direct_small<2, R><<<grid, DIRECT_THREADS, 0, s>>>(psrc, tiles, tps, ptgt, m, neg_c, dst, flags);
  else
    k_direct_small<3, R><<<grid, DIRECT_THREADS, 0, s>>>(psrc, tiles, tps, ptgt, m, neg_c, dst, flags);
  if (splits > 1) k_reduce_splits<<<gt, 256, 0, s>>>(part, (int)splits, m, out);
  if (cudaGetLastError() != cudaSuccess) return UOTK_ERR_CUDA;
  long long h[4] = {0, 0, 0, 0};
  if (cudaMemcpyAsync(h, flags, sizeof(h), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    return UOTK_ERR_CUDA;
  }
  if (h[FLAG_NONFINITE]) return UOTK_ERR_NONFINITE;
  if (h[FLAG_NEG_WEIGHT]) return UOTK_ERR_INVALID;
  if (h[FLAG_TIMEOUT]) return UOTK_ERR_TIMEOUT;
  return UOTK_OK;
}
