// The CTA body of the exact FP32 direct kernel sum (Alg. 1 matrix-vector
// product), shared by the single-problem kernels (ksum_direct.cu) and the
// batched solver (batch.cu).  See ksum_direct.cu for the design.
#pragma once

#include "uotk_internal.cuh"

namespace uotk {
namespace {

constexpr int STAGES = 3;

// Kernel value of a pair from its squared distance r2 (Table tab:0):
//   KIND 0 Gauss   2^{c0 r2}            c0 = -log2(e)/eps
//   KIND 1 Laplace 2^{c0 sqrt(r2)}      c0 = -log2(e)/ell
//   KIND 2 IMQ     1/sqrt(r2 + c1)      c1 = c^2
//   KIND 3 energy  -sqrt(r2)
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <int KIND>
__device__ __forceinline__ float kpair(float r2, float c0, float c1) {
  if (KIND == 0) return ex2_approx(r2 * c0);
  if (KIND == 1) return ex2_approx(sqrt_approx(r2) * c0);
  if (KIND == 2) return rsqrt_approx(r2 + c1);
  return -sqrt_approx(r2);
}

__device__ __forceinline__ void neumaier(float& hi, float& lo, float v) {
  const float t = hi + v;
  lo += (fabsf(hi) >= fabsf(v)) ? ((hi - t) + v) : ((v - t) + hi);
  hi = t;
}

// Body of the direct sum for one CTA: DIRECT_THREADS*R targets starting at
// target tb0 (of m) against `count` source tiles from tile t_begin of src,
// row sums written to o[j] (j < m).  Also used by the batched solver.
template <int D, int R, int KIND>
__device__ __forceinline__ void direct_body(const float4* __restrict__ src, long long t_begin,
                                            int count, const float4* __restrict__ tgt,
                                            long long m, long long tb0, float neg_c, float c1,
                                            float* __restrict__ o,
                                            long long* __restrict__ flags) {
  __shared__ __align__(128) float4 sm[STAGES][DIRECT_TILE];
  __shared__ __align__(8) unsigned long long bar[STAGES];
  const int tid = threadIdx.x;
  const long long tb = tb0 + tid;

  float tx[R], ty[R], tz[R], hi[R], lo[R];
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long j = tb + (long long)r * DIRECT_THREADS;
    const float4 p = j < m ? tgt[j] : make_float4(0.f, 0.f, 0.f, 0.f);
    tx[r] = p.x; ty[r] = p.y; tz[r] = p.z;
    hi[r] = 0.f; lo[r] = 0.f;
  }
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
      // A copy never completed: record it, wait (bounded) for the copies this
      // CTA still has in flight so none lands after exit, and leave.
      if (tid == 0) {
        flag_add(&flags[FLAG_TIMEOUT], 1LL);
        for (int q = k; q < count && q < k + STAGES; ++q)
          mbar_wait(&bar[q % STAGES], (unsigned)(q / STAGES) & 1u);
      }
      return;
    }
    const float4* T = sm[s];
#pragma unroll 1
    for (int j0 = 0; j0 < DIRECT_TILE; j0 += 32) {
      float acc[R];
      if constexpr (KIND == 0 && R % 2 == 0) {
        // Gaussian with an even number of targets per thread: the same IEEE
        // operations on target pairs in packed FP32x2 (half the issue slots)
        constexpr int R2 = R / 2;
        unsigned long long px[R2], py[R2], pz[R2], a2[R2];
        const unsigned long long c2 = f2_pack(neg_c, neg_c);
#pragma unroll
        for (int h = 0; h < R2; ++h) {
          px[h] = f2_pack(tx[2 * h], tx[2 * h + 1]);
          py[h] = f2_pack(ty[2 * h], ty[2 * h + 1]);
          pz[h] = f2_pack(tz[2 * h], tz[2 * h + 1]);
          a2[h] = 0ull;
        }
#pragma unroll 8
        for (int j = j0; j < j0 + 32; ++j) {
          const float4 q = T[j];
          const unsigned long long qx = f2_pack(q.x, q.x), qw = f2_pack(q.w, q.w);
#pragma unroll
          for (int h = 0; h < R2; ++h) {
            const unsigned long long dx = f2_sub(px[h], qx);
            unsigned long long r2 = f2_mul(dx, dx);
            if (D > 1) {
              const unsigned long long dy = f2_sub(py[h], f2_pack(q.y, q.y));
              r2 = f2_fma(dy, dy, r2);
            }
            if (D > 2) {
              const unsigned long long dz = f2_sub(pz[h], f2_pack(q.z, q.z));
              r2 = f2_fma(dz, dz, r2);
            }
            float e0, e1;
            f2_unpack(f2_mul(r2, c2), e0, e1);
            a2[h] = f2_fma(qw, f2_pack(ex2_approx(e0), ex2_approx(e1)), a2[h]);
          }
        }
#pragma unroll
        for (int h = 0; h < R2; ++h) f2_unpack(a2[h], acc[2 * h], acc[2 * h + 1]);
      } else {
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = 0.f;
#pragma unroll 8
        for (int j = j0; j < j0 + 32; ++j) {
          const float4 q = T[j];
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const float dx = tx[r] - q.x;
            float r2 = dx * dx;
            if (D > 1) { const float dy = ty[r] - q.y; r2 = fmaf(dy, dy, r2); }
            if (D > 2) { const float dz = tz[r] - q.z; r2 = fmaf(dz, dz, r2); }
            acc[r] = fmaf(q.w, kpair<KIND>(r2, neg_c, c1), acc[r]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) neumaier(hi[r], lo[r], acc[r]);
    }
    __syncthreads();
    if (tid == 0 && k + STAGES < count)
      { mbar_expect(&bar[s], BYTES); bulk_copy(sm[s], src + (t_begin + k + STAGES) * DIRECT_TILE, BYTES, &bar[s]); }
  }

#pragma unroll
  for (int r = 0; r < R; ++r) {
    const long long j = tb + (long long)r * DIRECT_THREADS;
    if (j < m) o[j] = hi[r] + lo[r];
  }
}


}  // namespace
}  // namespace uotk
