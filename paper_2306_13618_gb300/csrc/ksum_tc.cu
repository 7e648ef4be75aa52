// Direct kernel summation with the cross term on the 5th-generation tensor
// cores (tcgen05):
//
//   out_i = sum_j w_j 2^{-c ||x_i - y_j||^2},   c = log2(e)/eps,
//   ||x_i - y_j||^2 = |x_i|^2 + |y_j|^2 - 2 x_i . y_j,
//
// the exact matrix-vector product of Alg. 1 for high-dimensional clouds.  For
// d >= ~16 the squared distance, not the exponential, dominates the FP32 form
// (d FMAs per pair); here S = X Y^T is a dense contraction and runs on
// tcgen05.mma (kind::f16, BF16 inputs, FP32 accumulators in tensor memory),
// while the norms, the exponential and the weighted row sums stay in FP32 on
// the CUDA cores, fused behind the MMA.
//
// Precision.  Points are centred on the middle of the joint bounding box and
// rounded to BF16 as v = hi + lo (both BF16, lo the rounded remainder).
//   * BF16 form: S = hi_x . hi_y, one product (about 3 significant digits).
//   * BF16x3 form: S = hi.hi + hi.lo + lo.hi, three products accumulated in
//     FP32, the cross term to about 2^-17 relative (near FP32).
// The norms |x|^2, |y|^2 are FP32 from the FP32 centred coordinates.
//
// Layout.  Each cloud is packed once into tiles of 128 points; a tile holds,
// per 64-coordinate chunk, a block of hi and a block of lo values, each block
// 128 rows x 128 bytes in the 128-byte-swizzled K-major layout the MMA reads
// (16-byte chunk g of row r stored at chunk g ^ (r mod 8)).  Blocks are
// 16 KB, contiguous, and move global -> shared with 1-D bulk copies.
//
// CTA (640 threads, one per SM, all 512 tensor-memory columns):
//   warp 0, one lane: producer -- the CTA's 128-target tile once, then source
//     tiles through a ring of shared-memory stages (mbarrier transaction counts);
//   warp 1: allocates tensor memory; one lane issues the MMAs of each source
//     tile into one of 4 accumulator stages of 128 columns, and commits them to
//     the stage's barriers;
//   warp 2, one lane: copies the {b_j, w_j} pairs of each source tile into a
//     4-entry shared ring, one entry per accumulator stage;
//   warps 4-19: four epilogue warpgroups, warpgroup g taking source tiles
//     k = g mod 4; thread (warp, lane) owns target row 32 (warp mod 4) + lane,
//     reads its 128 accumulator columns with tcgen05.ld, and adds
//     w_j 2^{2c S + b_j + a_i} (b_j = -c |y_j|^2, a_i = -c |x_i|^2) into a
//     compensated FP32 pair.  Four warps per SM sub-partition hide the
//     tensor-memory and MUFU latencies.
// Every wait is bounded; a timeout raises the context's TIMEOUT flag, and the
// CTA drains its copies and MMAs before it frees tensor memory and exits.
#include <cuda_bf16.h>
#include <math.h>

#include <memory>

#include "engine.cuh"
#include "tcgen05.cuh"

namespace uotk {

namespace {

constexpr int TC_ROWS = 128;                 // targets per CTA (MMA M) = sources per tile (MMA N)
constexpr int TC_BLOCK = TC_ROWS * 128;      // bytes of one 128 x 64 BF16 block
constexpr int TC_ACC = 4;                    // accumulator stages (4 x 128 columns)
constexpr int TC_EPI_GROUPS = 4;            // epilogue warpgroups
constexpr int TC_THREADS = 128 + 128 * TC_EPI_GROUPS;
constexpr int TC_MISC = 12288;               // barriers, flags, weight ring, hand-over buffer
constexpr int TC_MIN_SMEM = 120 * 1024;      // forces one CTA per SM

__host__ __device__ constexpr int tc_ka(bool split, int dc) { return split ? 2 * dc : dc; }
// Source ring: slots of T = 1 or 2 source tiles (T = 2: one MMA of N = 256
// covers both, reading the target tile from shared memory half as often), as
// many slots as fit next to the target tile in ~200 KB, at most 8 (a deep ring
// hides the latency of streaming source tiles from L2).
__host__ __device__ constexpr int tc_tiles_per_slot(bool pair) { return pair ? 2 : 1; }
__host__ __device__ constexpr int tc_stages(bool split, int dc, bool pair) {
  return (200 * 1024 - tc_ka(split, dc) * TC_BLOCK) /
                     (tc_tiles_per_slot(pair) * tc_ka(split, dc) * TC_BLOCK) > 8
             ? 8
             : (200 * 1024 - tc_ka(split, dc) * TC_BLOCK) /
                   (tc_tiles_per_slot(pair) * tc_ka(split, dc) * TC_BLOCK);
}
__host__ __device__ constexpr size_t tc_smem_bytes(bool split, int dc, bool pair) {
  return (size_t)tc_ka(split, dc) * TC_BLOCK *
             (1 + (size_t)tc_tiles_per_slot(pair) * tc_stages(split, dc, pair)) +
         TC_MISC + 1024;
}
// Pairing needs at least two slots.
__host__ __device__ constexpr bool tc_can_pair(bool split, int dc) {
  return tc_stages(split, dc, true) >= 2;
}

// ---- tcgen05 instruction descriptor of this kernel ----
// Instruction descriptor: D FP32, A and B BF16, both K-major, M = 128, N = n.
__host__ __device__ constexpr unsigned tc_idesc(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((unsigned)(n >> 3) << 17) |
         ((unsigned)(TC_ROWS >> 4) << 24);
}
__device__ __forceinline__ void tc_neumaier(float& hi, float& lo, float v) {
  const float t = hi + v;
  lo += (fabsf(hi) >= fabsf(v)) ? ((hi - t) + v) : ((v - t) + hi);
  hi = t;
}

// Weighted exponential sum of 16 accumulator columns of one row:
//   sum_j w_j 2^{2c S_j + b_j + aa}   (FAST: without aa, applied to the row sum).
// Columns go in pairs through packed FP32 instructions; bw holds, per pair of
// columns, {b_j, b_j+1, w_j, w_j+1}.
template <bool FAST>
__device__ __forceinline__ float tc_chunk(const unsigned (&v)[16], const ulonglong2* bw,
                                          unsigned long long two_c2, unsigned long long aa2) {
  unsigned long long acc = 0ull;
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    const ulonglong2 q = bw[j >> 1];  // shared-memory broadcast
    unsigned long long e =
        f2_fma(f2_pack(__uint_as_float(v[j]), __uint_as_float(v[j + 1])), two_c2, q.x);
    if (!FAST) e = f2_add(e, aa2);
    float e0, e1;
    f2_unpack(e, e0, e1);
    acc = f2_fma(q.y, f2_pack(ex2_approx(e0), ex2_approx(e1)), acc);
  }
  float s0, s1;
  f2_unpack(acc, s0, s1);
  return s0 + s1;
}

// Online log-sum-exp form of tc_chunk (log domain): the terms are
//   e_j = 2c S_j + b_j + lw_j   (log2 units; lw_j = log2 w_j in the weight lane),
// and (M, hi + lo) is updated so that the row's running sum of 2^{e_j} equals
// 2^M (hi + lo).  No term has to be representable as an FP32 number.
__device__ __forceinline__ void tc_chunk_lse(const unsigned (&v)[16], const ulonglong2* bw,
                                             unsigned long long two_c2, float& M, float& hi,
                                             float& lo) {
  float e[16];
  float cm = -INFINITY;
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    const ulonglong2 q = bw[j >> 1];
    const unsigned long long t = f2_add(
        f2_fma(f2_pack(__uint_as_float(v[j]), __uint_as_float(v[j + 1])), two_c2, q.x), q.y);
    f2_unpack(t, e[j], e[j + 1]);
    cm = fmaxf(cm, fmaxf(e[j], e[j + 1]));
  }
  if (cm == -INFINITY) return;  // every weight of the chunk is zero
  if (cm > M) {
    const float f = ex2_approx(M - cm);  // 0 while M is still -inf
    hi *= f;
    lo *= f;
    M = cm;
  }
  const unsigned long long m2 = f2_pack(M, M);
  unsigned long long acc = 0ull;
#pragma unroll
  for (int j = 0; j < 16; j += 2) {
    float d0, d1;
    f2_unpack(f2_sub(f2_pack(e[j], e[j + 1]), m2), d0, d1);
    acc = f2_add(acc, f2_pack(ex2_approx(d0), ex2_approx(d1)));
  }
  float s0, s1;
  f2_unpack(acc, s0, s1);
  tc_neumaier(hi, lo, s0 + s1);
}

// One CTA: 128 targets (blockIdx.x) against the source tiles of split
// blockIdx.y.  tiles: [tile][2*DC blocks][16 KB], block 2c = hi, 2c+1 = lo of
// coordinate chunk c.  bw: per pair of sources {b_j, b_j+1, w_j, w_j+1} with
// b = -c |y|^2, zero past the last source.
// out: [splits][m] (split partial sums) or [m].
// FAST: the row factor 2^{-c |x|^2} is applied to the finished row sum instead
// of to every term (one FP32 add less per pair).  The host selects it only when
// c R^2 <= 64, R the largest centred norm, so that no term 2^{c(|x|^2 - ||x-y||^2)}
// can overflow.
// LSE: the log-domain form; weights are log2 w_j, each row keeps a running
// maximum M and the sum relative to it, and out holds {M + aa, S} per row
// (float2) with log2 t_i = M + aa + log2 S.
template <bool SPLIT, int DC, bool FAST, bool PAIR, bool LSE = false>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_direct_tc(const unsigned char* __restrict__ src_tiles, const float* __restrict__ src_bw,
                long long src_tiles_total, int tiles_per_split,
                const unsigned char* __restrict__ tgt_tiles, const float* __restrict__ tgt_n2,
                long long m, float two_c, float neg_c, float* __restrict__ out,
                long long* __restrict__ flags) {
  constexpr int KBT = 2 * DC;               // blocks per tile in global memory
  constexpr int KA = tc_ka(SPLIT, DC);      // blocks per tile in shared memory
  constexpr int T = tc_tiles_per_slot(PAIR);        // source tiles per ring slot
  constexpr int S = tc_stages(SPLIT, DC, PAIR);     // ring slots
  constexpr unsigned STAGE_BYTES = (unsigned)KA * TC_BLOCK;  // one tile, all blocks
  constexpr unsigned SLOT_BYTES = (unsigned)T * STAGE_BYTES;
  static_assert(S >= 2, "at least two source slots");

  extern __shared__ unsigned char tc_raw[];
  const unsigned raw = smem_addr(tc_raw);
  unsigned char* sA = tc_raw + ((1024u - (raw & 1023u)) & 1023u);
  unsigned char* sB = sA + STAGE_BYTES;
  unsigned char* misc = sB + (size_t)S * SLOT_BYTES;
  unsigned long long* a_full = reinterpret_cast<unsigned long long*>(misc);
  unsigned long long* b_full = a_full + 1;
  unsigned long long* b_empty = b_full + S;
  unsigned long long* t_full = b_empty + S;
  unsigned long long* t_empty = t_full + TC_ACC;
  unsigned long long* done = t_empty + TC_ACC;
  unsigned long long* w_full = done + 1;                  // [TC_ACC] weight ring entries landed
  unsigned* tmem_slot = reinterpret_cast<unsigned*>(misc + 256);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(misc + 260);
  // Weight ring: the {b_j, w_j} pairs of the source tile in accumulator stage a
  // (1 KB each), filled by warp 2 once the epilogue has released stage a.
  float* wring = reinterpret_cast<float*>(misc + 1024);  // [TC_ACC][2 * TC_ROWS]
  // [groups - 1][2][128] compensated row sums handed to warpgroup 0
  float* hand = reinterpret_cast<float*>(misc + 1024 + TC_ACC * TC_ROWS * sizeof(float2));

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long t_begin = (long long)blockIdx.y * tiles_per_split;
  const long long t_end = min(t_begin + (long long)tiles_per_split, src_tiles_total);
  const int count = t_end > t_begin ? (int)(t_end - t_begin) : 0;
  const int groups = (count + T - 1) / T;  // ring fills; group r holds tiles rT .. rT + T - 1

  if (threadIdx.x == 0) {
    mbar_init(a_full, 1);
    for (int s = 0; s < S; ++s) { mbar_init(&b_full[s], 1); mbar_init(&b_empty[s], 1); }
    for (int a = 0; a < TC_ACC; ++a) { mbar_init(&t_full[a], 1); mbar_init(&t_empty[a], 128); }
    mbar_init(done, 1);
    for (int a = 0; a < TC_ACC; ++a) mbar_init(&w_full[a], 1);
    *abort_flag = 0;
    mbar_fence_init();
  }
  if (warp == 1) {
    __syncwarp();
    tc_alloc(tmem_slot, 512);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const unsigned tmem = *tmem_slot;
  float hi = 0.f, lo = 0.f;  // epilogue: compensated row sum
  float M = -INFINITY;        // log domain: the row's running maximum exponent

  if (warp == 0 && lane == 0) {
    // ---- producer ----
    int fills[S];
#pragma unroll
    for (int s = 0; s < S; ++s) fills[s] = 0;
    static_assert(S <= 8, "barrier region holds at most 8 stages");
    mbar_expect(a_full, STAGE_BYTES);
    for (int b = 0; b < KA; ++b) {
      const int kb = SPLIT ? b : 2 * b;
      bulk_copy(sA + (size_t)b * TC_BLOCK,
                tgt_tiles + ((size_t)blockIdx.x * KBT + kb) * TC_BLOCK, TC_BLOCK, a_full);
    }
    for (int r = 0; r < groups; ++r) {
      const int s = r % S, u = r / S;
      if (u > 0 && !mbar_wait(&b_empty[s], (unsigned)(u - 1) & 1u)) {
        *abort_flag = 1;
        flag_add(&flags[FLAG_TIMEOUT], 1LL);
        break;
      }
      if (*abort_flag) break;
      const int nt = min(T, count - r * T);
      mbar_expect(&b_full[s], (unsigned)nt * STAGE_BYTES);
      // slot layout: block b of tile t at b*T*16K + t*16K, so that the T tiles
      // of one block form T*128 consecutive rows
      for (int t = 0; t < nt; ++t) {
        const size_t tile = (size_t)(t_begin + r * T + t);
        for (int b = 0; b < KA; ++b) {
          const int kb = SPLIT ? b : 2 * b;
          bulk_copy(sB + (size_t)s * SLOT_BYTES + ((size_t)b * T + t) * TC_BLOCK,
                    src_tiles + (tile * KBT + kb) * TC_BLOCK, TC_BLOCK, &b_full[s]);
        }
      }
      fills[s]++;
    }
    // Drain: every copy this thread started has landed before the CTA exits.
    mbar_wait(a_full, 0u);
#pragma unroll
    for (int s = 0; s < S; ++s)
      if (fills[s]) mbar_wait(&b_full[s], (unsigned)(fills[s] - 1) & 1u);
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer ----
    int issued = 0;
    bool ok = mbar_wait(a_full, 0u);
    if (!ok) { *abort_flag = 1; flag_add(&flags[FLAG_TIMEOUT], 1LL); }
    const unsigned a0 = smem_addr(sA);
    for (int r = 0; ok && r < groups; ++r) {
      const int s = r % S, us = r / S;
      const int nt = min(T, count - r * T);
      bool got = mbar_wait(&b_full[s], (unsigned)us & 1u);
      for (int t = 0; got && t < nt; ++t) {
        const int k = r * T + t, ua = k / TC_ACC;
        if (ua > 0) got = mbar_wait(&t_empty[k % TC_ACC], (unsigned)(ua - 1) & 1u);
      }
      if (!got) {
        *abort_flag = 1;
        flag_add(&flags[FLAG_TIMEOUT], 1LL);
        break;
      }
      if (*abort_flag) break;
      tc_fence_after();
      // the group's tiles land in consecutive accumulator stages (T = 2: stages
      // 0,1 or 2,3, i.e. 256 consecutive columns)
      const unsigned d_tmem = tmem + (unsigned)(((r * T) % TC_ACC) * TC_ROWS);
      const unsigned idesc = tc_idesc(nt * TC_ROWS);
      const unsigned b0 = smem_addr(sB + (size_t)s * SLOT_BYTES);
      unsigned q = 0;
#pragma unroll
      for (int c = 0; c < DC; ++c) {
#pragma unroll
        for (int p = 0; p < (SPLIT ? 3 : 1); ++p) {
          // products hi.hi, hi.lo, lo.hi (blocks 2c = hi, 2c + 1 = lo)
          const int ba = SPLIT ? 2 * c + (p == 2 ? 1 : 0) : c;
          const int bb = SPLIT ? 2 * c + (p == 1 ? 1 : 0) : c;
#pragma unroll
          for (int ks = 0; ks < 4; ++ks, ++q)
            tc_mma(d_tmem, tc_desc(a0 + (unsigned)(ba * TC_BLOCK + ks * 32)),
                   tc_desc(b0 + (unsigned)(bb * T * TC_BLOCK + ks * 32)), idesc,
                   q > 0 ? 1u : 0u);
        }
      }
      tc_commit(&b_empty[s]);
      for (int t = 0; t < nt; ++t) tc_commit(&t_full[(r * T + t) % TC_ACC]);
      issued++;
    }
    // Drain: no MMA may still be running when tensor memory is freed.
    if (issued) {
      tc_commit(done);
      mbar_wait(done, 0u);
    }
  } else if (warp == 2 && lane == 0) {
    // ---- weight producer ----
    int fills[TC_ACC] = {0, 0, 0, 0};
    for (int k = 0; k < count; ++k) {
      const int a = k % TC_ACC, ua = k / TC_ACC;
      if (ua > 0 && !mbar_wait(&t_empty[a], (unsigned)(ua - 1) & 1u)) {
        *abort_flag = 1;
        flag_add(&flags[FLAG_TIMEOUT], 1LL);
        break;
      }
      if (*abort_flag) break;
      mbar_expect(&w_full[a], 2 * TC_ROWS * sizeof(float));
      bulk_copy(wring + a * 2 * TC_ROWS, src_bw + (t_begin + k) * 2 * TC_ROWS, TC_ROWS * sizeof(float2),
                &w_full[a]);
      fills[a]++;
    }
#pragma unroll
    for (int a = 0; a < TC_ACC; ++a)
      if (fills[a]) mbar_wait(&w_full[a], (unsigned)(fills[a] - 1) & 1u);
  } else if (warp >= 4) {
    // ---- epilogue ----
    const int g = (warp - 4) >> 2;  // warpgroup: source tiles k = g, g + groups, ...
    const int quad = warp & 3;      // tensor-memory lanes 32 quad .. 32 quad + 31
    const int row = quad * 32 + lane;
    const long long i = (long long)blockIdx.x * TC_ROWS + row;
    const float aa = i < m ? neg_c * tgt_n2[i] : 0.f;
    const unsigned long long aa2 = f2_pack(aa, aa), two_c2 = f2_pack(two_c, two_c);
    for (int k = g; k < count; k += TC_EPI_GROUPS) {
      const int a = k % TC_ACC, ua = k / TC_ACC;
      bool ok = mbar_wait(&t_full[a], (unsigned)ua & 1u) && mbar_wait(&w_full[a], (unsigned)ua & 1u);
      ok = __all_sync(0xffffffffu, ok) && !__any_sync(0xffffffffu, *abort_flag != 0);
      if (!ok) {
        if (lane == 0) {
          *abort_flag = 1;
          flag_add(&flags[FLAG_TIMEOUT], 1LL);
        }
        break;
      }
      tc_fence_after();
      const ulonglong2* bw = reinterpret_cast<const ulonglong2*>(wring + a * 2 * TC_ROWS);
      const unsigned tb = tmem + ((unsigned)(quad * 32) << 16) + (unsigned)(a * TC_ROWS);
      // columns in chunks of 16, the load of the next chunk in flight while
      // the current one is summed
      unsigned v0[16], v1[16];
      tc_ld16(tb, v0);
      tc_wait16(v0);
#pragma unroll
      for (int c0 = 0; c0 < TC_ROWS; c0 += 32) {
        tc_ld16(tb + (unsigned)(c0 + 16), v1);
        if constexpr (LSE)
          tc_chunk_lse(v0, bw + (c0 >> 1), two_c2, M, hi, lo);
        else
          tc_neumaier(hi, lo, tc_chunk<FAST>(v0, bw + (c0 >> 1), two_c2, aa2));
        tc_wait16(v1);
        if (c0 + 32 < TC_ROWS) tc_ld16(tb + (unsigned)(c0 + 32), v0);
        if constexpr (LSE)
          tc_chunk_lse(v1, bw + ((c0 + 16) >> 1), two_c2, M, hi, lo);
        else
          tc_neumaier(hi, lo, tc_chunk<FAST>(v1, bw + ((c0 + 16) >> 1), two_c2, aa2));
        if (c0 + 32 < TC_ROWS) tc_wait16(v0);
      }
      tc_fence_before();
      mbar_arrive(&t_empty[a]);
    }
    if (g > 0) {
      // log domain: {M, S}; otherwise the compensated pair {hi, lo}
      hand[(g - 1) * 2 * TC_ROWS + row] = LSE ? M : hi;
      hand[(g - 1) * 2 * TC_ROWS + TC_ROWS + row] = LSE ? hi + lo : lo;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp >= 4 && warp < 8) {
    // warpgroup 0 adds the other warpgroups' pairs for the same row
    const int row = (warp & 3) * 32 + lane;
    const long long i = (long long)blockIdx.x * TC_ROWS + row;
    if constexpr (LSE) {
#pragma unroll
      for (int q = 0; q < TC_EPI_GROUPS - 1; ++q) {
        const float Mq = hand[q * 2 * TC_ROWS + row], Sq = hand[q * 2 * TC_ROWS + TC_ROWS + row];
        if (Mq == -INFINITY) continue;
        if (Mq > M) {
          const float f = ex2_approx(M - Mq);
          hi *= f;
          lo *= f;
          M = Mq;
        }
        tc_neumaier(hi, lo, Sq * ex2_approx(Mq - M));
      }
      if (i < m) {
        const float aa = neg_c * tgt_n2[i];
        reinterpret_cast<float2*>(out)[(long long)blockIdx.y * m + i] =
            make_float2(M == -INFINITY ? -INFINITY : M + aa, hi + lo);
      }
    }
#pragma unroll
    for (int q = 0; q < (LSE ? 0 : TC_EPI_GROUPS - 1); ++q) {
      tc_neumaier(hi, lo, hand[q * 2 * TC_ROWS + row]);
      tc_neumaier(hi, lo, hand[q * 2 * TC_ROWS + TC_ROWS + row]);
    }
    if (!LSE && i < m) {
      float v = hi + lo;
      if (FAST) {
        // v * 2^{aa}, aa = -c |x_i|^2 <= 0, without flushing a small result
        const float aa = neg_c * tgt_n2[i];
        const float k = floorf(aa);
        v = ldexpf(v * exp2f(aa - k), (int)k);
      }
      out[(long long)blockIdx.y * m + i] = v;
    }
  }
  if (warp == 1) {
    __syncwarp();
    tc_fence_after();
    tc_dealloc(tmem, 512);
  }
}

// ---- packing ----
// Per-dimension maximum of v and of -v over a cloud (ordered encodings in
// slots[0..d) and slots[d..2d)).  The grid stride is a multiple of d, so each
// thread stays on one coordinate.
__global__ void k_tc_minmax(const float* __restrict__ p, long long count, int d,
                            long long* __restrict__ slots) {
  __shared__ long long smx[128], smn[128];
  for (int c = threadIdx.x; c < d; c += blockDim.x) { smx[c] = ORDERED_NEG_INF; smn[c] = ORDERED_NEG_INF; }
  __syncthreads();
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long first = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (first < count) {
    double mx = -INFINITY, mn = -INFINITY;
    for (long long q = first; q < count; q += stride) {
      const double v = (double)p[q];
      mx = fmax(mx, v);
      mn = fmax(mn, -v);
    }
    atomicMax(&smx[first % d], dbl_to_ordered(mx));
    atomicMax(&smn[first % d], dbl_to_ordered(mn));
  }
  __syncthreads();
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    if (smx[c] != ORDERED_NEG_INF) atomicMax(&slots[c], smx[c]);
    if (smn[c] != ORDERED_NEG_INF) atomicMax(&slots[d + c], smn[c]);
  }
}

// Box centre per coordinate, and in r2[0] the squared distance from the centre
// to the farthest corner (an upper bound of |p - centre|^2).  One block.
__global__ void k_tc_center(const long long* __restrict__ slots, int d, float* __restrict__ center,
                            double* __restrict__ r2) {
  __shared__ double part[128];
  double acc = 0.0;
  for (int c = threadIdx.x; c < d; c += blockDim.x) {
    const double hi = ordered_to_dbl(slots[c]), lo = -ordered_to_dbl(slots[d + c]);
    const bool ok = isfinite(hi) && isfinite(lo);
    center[c] = ok ? (float)(0.5 * (hi + lo)) : 0.f;
    const double hw = ok ? 0.5 * (hi - lo) : 0.0;
    acc += hw * hw;
  }
  part[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)blockDim.x; ++k) t += part[k];
    r2[0] = t;
  }
}

__global__ void k_tc_fill_slots(long long* slots, int count) {
  for (int c = threadIdx.x; c < count; c += blockDim.x) slots[c] = ORDERED_NEG_INF;
}

// BF16 hi/lo blocks of the centred coordinates: one thread per (point, 8
// coordinates).  Points i >= n are zero rows.
__global__ void k_tc_pack(const float* __restrict__ pts, long long n, long long n_pad, int d,
                          int dc, const float* __restrict__ center,
                          unsigned char* __restrict__ tiles) {
  const long long units = n_pad * 8 * dc;
  for (long long u = blockIdx.x * (long long)blockDim.x + threadIdx.x; u < units;
       u += (long long)gridDim.x * blockDim.x) {
    const long long i = u / (8 * dc);
    const int q = (int)(u % (8 * dc));
    const int c = q >> 3, g = q & 7;
    unsigned hw[4], lw[4];
#pragma unroll
    for (int e = 0; e < 8; e += 2) {
      float v[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int t = 64 * c + 8 * g + e + h;
        v[h] = (i < n && t < d) ? __fsub_rn(pts[i * d + t], center[t]) : 0.f;
      }
      const __nv_bfloat16 h0 = __float2bfloat16_rn(v[0]), h1 = __float2bfloat16_rn(v[1]);
      const __nv_bfloat16 l0 = __float2bfloat16_rn(__fsub_rn(v[0], __bfloat162float(h0)));
      const __nv_bfloat16 l1 = __float2bfloat16_rn(__fsub_rn(v[1], __bfloat162float(h1)));
      hw[e >> 1] = (unsigned)__bfloat16_as_ushort(h0) | ((unsigned)__bfloat16_as_ushort(h1) << 16);
      lw[e >> 1] = (unsigned)__bfloat16_as_ushort(l0) | ((unsigned)__bfloat16_as_ushort(l1) << 16);
    }
    const long long tile = i / TC_ROWS;
    const int r = (int)(i % TC_ROWS);
    const size_t off = (size_t)(r >> 3) * 1024 + (size_t)(r & 7) * 128 + (size_t)((g ^ (r & 7)) * 16);
    unsigned char* hb = tiles + ((size_t)tile * 2 * dc + 2 * c) * TC_BLOCK + off;
    *reinterpret_cast<uint4*>(hb) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
    *reinterpret_cast<uint4*>(hb + TC_BLOCK) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
  }
}

// Squared norms of the centred FP32 points (0 past n), the source entries
// {b_j, b_j+1, w_j, w_j+1} per pair of points (b = -c |p|^2; b = w = 0 past n),
// and validation counters of the weights.
__global__ void k_tc_norms(const float* __restrict__ pts, const float* __restrict__ w, long long n,
                           long long n_pad, int d, const float* __restrict__ center, float neg_c,
                           float* __restrict__ n2, float* __restrict__ bw,
                           long long* __restrict__ flags) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long start = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const long long iters = (n_pad + stride - 1) / stride;
  for (long long it = 0; it < iters; ++it) {
    const long long i = start + it * stride;
    bool neg = false, bad = false;
    if (i < n_pad) {
      double s = 0.0;
      float wi = 0.f;
      if (i < n) {
        for (int t = 0; t < d; ++t) {
          const float v = __fsub_rn(pts[i * d + t], center[t]);
          bad |= !isfinite(pts[i * d + t]);
          s = fma((double)v, (double)v, s);
        }
        if (w) {
          wi = w[i];
          neg = wi < 0.f;
          bad |= !isfinite(wi);
        }
      }
      n2[i] = (float)s;
      bw[(i >> 1) * 4 + (i & 1)] = neg_c * (float)s;  // per source pair {b, b', w, w'}
      bw[(i >> 1) * 4 + 2 + (i & 1)] = wi;
    }
    const unsigned bn = __ballot_sync(0xffffffffu, neg);
    const unsigned bf = __ballot_sync(0xffffffffu, bad);
    if ((threadIdx.x & 31) == 0) {
      if (bn) flag_add(&flags[FLAG_NEG_WEIGHT], (long long)__popc(bn));
      if (bf) flag_add(&flags[FLAG_NONFINITE], (long long)__popc(bf));
    }
  }
}

// w_j = base_j * exp(lam*pot_j - shift) (pot NULL: base_j; base NULL: 1), 0
// past n; LOG: log2 w_j instead (-inf past n and for zero weights), the FP64
// exponent taken to log2 units before the one rounding to FP32.
template <bool LOG>
__global__ void k_tc_set_weights(float* __restrict__ bw, long long n, long long n_pad,
                                 const float* __restrict__ base, const double* __restrict__ pot,
                                 double lam, const long long* __restrict__ shift_slot) {
  const double shift = pot ? ordered_to_dbl(*shift_slot) : 0.0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n_pad;
       i += (long long)gridDim.x * blockDim.x) {
    float v;
    if (LOG) {
      if (i < n) {
        const double e = pot ? (lam * pot[i] - shift) * 1.4426950408889634 : 0.0;
        const float bl = base ? log2f(base[i]) : 0.f;
        v = (float)((double)bl + e);
      } else {
        v = -INFINITY;
      }
    } else {
      v = 0.f;
      if (i < n) {
        v = pot ? exp_shifted(lam * pot[i] - shift) : 1.f;
        if (base) v *= base[i];
      }
    }
    bw[(i >> 1) * 4 + 2 + (i & 1)] = v;
  }
}

// Log-sum-exp of the split partials {M, S}: out = {max M, sum S 2^{M_k - max}}.
__global__ void k_tc_reduce_lse(const float2* __restrict__ part, int splits, long long m,
                                float2* __restrict__ out) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
       j += (long long)gridDim.x * blockDim.x) {
    float mx = -INFINITY;
    for (int k = 0; k < splits; ++k) mx = fmaxf(mx, part[(long long)k * m + j].x);
    double s = 0.0;
    if (mx != -INFINITY)
      for (int k = 0; k < splits; ++k) {
        const float2 p = part[(long long)k * m + j];
        if (p.x != -INFINITY) s += (double)p.y * (double)exp2f(p.x - mx);
      }
    out[j] = make_float2(mx, (float)s);
  }
}

__global__ void k_tc_reduce(const float* __restrict__ part, int splits, long long m,
                            float* __restrict__ out) {
  for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
       j += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < splits; ++k) s += (double)part[(long long)k * m + j];
    out[j] = (float)s;
  }
}

// A packed cloud: tiles, squared norms, source pairs.
struct TcCloud {
  int64_t n = 0, tiles = 0;
  unsigned char* tile_data = nullptr;  // [tiles][2 dc][16 KB]
  float* n2 = nullptr;                 // [tiles * 128]
  float* bw = nullptr;                 // [tiles * 64][4]: per source pair {b, b', w, w'}
};

int64_t tc_tiles(int64_t n) { return (n + TC_ROWS - 1) / TC_ROWS; }

void tc_carve_cloud(Carver& cv, int dc, int64_t n, TcCloud& C) {
  C.n = n;
  C.tiles = tc_tiles(n);
  const int64_t t = C.tiles > 0 ? C.tiles : 1;
  C.tile_data = cv.take<unsigned char>((size_t)t * 2 * dc * TC_BLOCK);
  C.n2 = cv.take<float>((size_t)t * TC_ROWS);
  C.bw = cv.take<float>((size_t)t * 2 * TC_ROWS);
}

// Source splits for a (sources -> targets) pair: enough CTAs for about two
// per SM when the targets alone give fewer.
struct TcSplit {
  int splits = 1;
  int tiles_per_split = 0;
};
TcSplit tc_split(const uotk_ctx* ctx, int64_t src_tiles, int64_t tgt_tiles) {
  TcSplit L;
  if (src_tiles == 0 || tgt_tiles == 0) return L;
  int64_t want = (2 * (int64_t)ctx->num_sms + tgt_tiles - 1) / tgt_tiles;
  want = want < 1 ? 1 : (want > src_tiles ? src_tiles : want);
  want = want > 64 ? 64 : want;
  L.tiles_per_split = (int)((src_tiles + want - 1) / want);
  L.splits = (int)((src_tiles + L.tiles_per_split - 1) / L.tiles_per_split);
  return L;
}

template <bool SPLIT, int DC, bool FAST, bool LSE = false>
uotk_status tc_launch(uotk_ctx* ctx, cudaStream_t s, const TcCloud& src, const TcCloud& tgt,
                      const TcSplit& L, double eps, float* dst) {
  constexpr bool PAIR = tc_can_pair(SPLIT, DC);
  constexpr size_t smem0 = tc_smem_bytes(SPLIT, DC, PAIR);
  constexpr size_t smem = smem0 > (size_t)TC_MIN_SMEM ? smem0 : (size_t)TC_MIN_SMEM;
  UOTK_CUDA(ctx, smem_attr(s, k_direct_tc<SPLIT, DC, FAST, PAIR, LSE>, smem));
  const double c = 1.4426950408889634 / eps;
  const dim3 grid((unsigned)tgt.tiles, (unsigned)L.splits);
  k_direct_tc<SPLIT, DC, FAST, PAIR, LSE><<<grid, TC_THREADS, smem, s>>>(
      src.tile_data, src.bw, src.tiles, L.tiles_per_split, tgt.tile_data, tgt.n2, tgt.n,
      (float)(2.0 * c), (float)(-c), dst, ctx->dflags);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

// out[i] = sum_j w_j exp(-||tgt_i - src_j||^2/eps), w in src.bw.
uotk_status tc_run(uotk_ctx* ctx, cudaStream_t s, bool split, int dc, bool fast,
                   const TcCloud& src, const TcCloud& tgt, double eps, float* part, float* out) {
  if (tgt.n == 0) return UOTK_OK;
  if (src.n == 0) {
    UOTK_CUDA(ctx, cudaMemsetAsync(out, 0, sizeof(float) * tgt.n, s));
    return UOTK_OK;
  }
  const TcSplit L = tc_split(ctx, src.tiles, tgt.tiles);
  float* dst = L.splits > 1 ? part : out;
  {
    UOTK_PROF(ctx, s, "direct_tc");
    uotk_status st;
#define UOTK_TC_CASE(SP, DCC, FA) \
  if (split == SP && dc == DCC && fast == FA) st = tc_launch<SP, DCC, FA>(ctx, s, src, tgt, L, eps, dst);
    st = UOTK_ERR_INTERNAL;
    UOTK_TC_CASE(true, 1, true) UOTK_TC_CASE(true, 1, false) UOTK_TC_CASE(true, 2, true)
    UOTK_TC_CASE(true, 2, false) UOTK_TC_CASE(false, 1, true) UOTK_TC_CASE(false, 1, false)
    UOTK_TC_CASE(false, 2, true) UOTK_TC_CASE(false, 2, false)
#undef UOTK_TC_CASE
    UOTK_TRY(st);
  }
  if (L.splits > 1) {
    UOTK_PROF(ctx, s, "split_reduce");
    k_tc_reduce<<<grid_for(ctx, tgt.n, 256), 256, 0, s>>>(part, L.splits, tgt.n, out);
    UOTK_LAUNCHED(ctx);
  }
  return UOTK_OK;
}

// Log domain: out[i] = {M_i, S_i} with log2 sum_j w_j exp(-||tgt_i - src_j||^2/eps)
// = M_i + log2 S_i, log2 w in src.bw; part holds splits * m float2.
uotk_status tc_run_lse(uotk_ctx* ctx, cudaStream_t s, bool split, int dc, const TcCloud& src,
                       const TcCloud& tgt, double eps, float2* part, float2* out) {
  if (tgt.n == 0) return UOTK_OK;
  if (src.n == 0) return set_error(ctx, UOTK_ERR_INVALID, "log-domain sum with no sources");
  const TcSplit L = tc_split(ctx, src.tiles, tgt.tiles);
  float* dst = reinterpret_cast<float*>(L.splits > 1 ? part : out);
  {
    UOTK_PROF(ctx, s, "direct_tc_lse");
    uotk_status st = UOTK_ERR_INTERNAL;
#define UOTK_TC_LSE_CASE(SP, DCC) \
  if (split == SP && dc == DCC) st = tc_launch<SP, DCC, true, true>(ctx, s, src, tgt, L, eps, dst);
    UOTK_TC_LSE_CASE(true, 1) UOTK_TC_LSE_CASE(true, 2) UOTK_TC_LSE_CASE(false, 1)
    UOTK_TC_LSE_CASE(false, 2)
#undef UOTK_TC_LSE_CASE
    UOTK_TRY(st);
  }
  if (L.splits > 1) {
    UOTK_PROF(ctx, s, "split_reduce");
    k_tc_reduce_lse<<<grid_for(ctx, tgt.n, 256), 256, 0, s>>>(part, L.splits, tgt.n, out);
    UOTK_LAUNCHED(ctx);
  }
  return UOTK_OK;
}

// ---------------------------------------------------------------------------
// Engine: both clouds packed once; every half-step rewrites the source weights
// and runs the tensor-core summation.
// ---------------------------------------------------------------------------
struct TcEngine : Engine {
  uotk_ctx* ctx = nullptr;
  int d = 0, dc = 1;
  bool split = true;
  bool fast = false;  // c R^2 <= 64: row factor applied after the sum
  int64_t n = 0, m = 0;
  const float* a = nullptr;
  const float* b = nullptr;
  double eps = 1.0;
  TcCloud X, Y;
  float* part = nullptr;
  float* center = nullptr;
  long long* slots = nullptr;
  double* r2 = nullptr;

  static void carve(const uotk_ctx* ctx, const EngineSpec& sp, Carver& cv, TcEngine* e) {
    const int dc = (sp.d + 63) / 64;
    TcCloud X, Y;
    tc_carve_cloud(cv, dc, sp.n, X);
    tc_carve_cloud(cv, dc, sp.m, Y);
    size_t part = 1;
    const int64_t pairs[4][2] = {{Y.tiles, X.tiles}, {X.tiles, Y.tiles}, {X.tiles, X.tiles},
                                 {Y.tiles, Y.tiles}};
    const int64_t tgt_n[4] = {sp.n, sp.m, sp.n, sp.m};
    for (int k = 0; k < 4; ++k) {
      const TcSplit L = tc_split(ctx, pairs[k][0], pairs[k][1]);
      if (L.splits > 1) {
        const size_t need = (size_t)L.splits * (size_t)tgt_n[k];
        part = need > part ? need : part;
      }
    }
    float* pp = cv.take<float>(2 * part);  // FP32 sums, or {M, S} pairs of the log domain
    float* ctr = cv.take<float>(128);
    long long* sl = cv.take<long long>(256);
    double* r2 = cv.take<double>(1);
    if (e) {
      e->r2 = r2;
      e->dc = dc;
      e->X = X;
      e->Y = Y;
      e->part = pp;
      e->center = ctr;
      e->slots = sl;
    }
  }

  uotk_status set_weights(cudaStream_t s, TcCloud& C, const float* base, const double* pot,
                          double lam, const long long* shift_slot, bool log2w = false) {
    if (C.n == 0) return UOTK_OK;
    UOTK_PROF(ctx, s, "weights");
    const long long n_pad = C.tiles * TC_ROWS;
    if (log2w)
      k_tc_set_weights<true><<<grid_for(ctx, n_pad, 256, 4), 256, 0, s>>>(C.bw, C.n, n_pad, base,
                                                                          pot, lam, shift_slot);
    else
      k_tc_set_weights<false><<<grid_for(ctx, n_pad, 256, 4), 256, 0, s>>>(C.bw, C.n, n_pad, base,
                                                                           pot, lam, shift_slot);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  }

  uotk_status half(cudaStream_t s, int side, const float* base, const double* pot, double lam,
                   const long long* shift_slot, float* out) override {
    TcCloud& src = side == 0 ? Y : X;
    const TcCloud& tgt = side == 0 ? X : Y;
    UOTK_TRY(set_weights(s, src, base, pot, lam, shift_slot));
    return tc_run(ctx, s, split, dc, fast, src, tgt, eps, part, out);
  }
  uotk_status half_log(cudaStream_t s, int side, const float* base, const double* pot,
                       double lam, const long long* shift_slot, float2* out) override {
    TcCloud& src = side == 0 ? Y : X;
    const TcCloud& tgt = side == 0 ? X : Y;
    UOTK_TRY(set_weights(s, src, base, pot, lam, shift_slot, true));
    return tc_run_lse(ctx, s, split, dc, src, tgt, eps, reinterpret_cast<float2*>(part), out);
  }
  uotk_status plain(cudaStream_t s, int src, int tgt, const float* w, float* out) override {
    TcCloud& S = src == 0 ? X : Y;
    UOTK_TRY(set_weights(s, S, w, nullptr, 0.0, nullptr));
    return tc_run(ctx, s, split, dc, fast, S, tgt == 0 ? X : Y, eps, part, out);
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

int gcd_int(int a, int b) { return b == 0 ? a : gcd_int(b, a % b); }

uotk_status tc_minmax(uotk_ctx* ctx, cudaStream_t s, const float* p, int64_t n, int d,
                      long long* slots) {
  if (n == 0) return UOTK_OK;
  const long long count = (long long)n * d;
  const int step = d / gcd_int(d, 256);  // blocks per multiple of d threads
  int blocks = grid_for(ctx, count, 256, 2);
  blocks = ((blocks + step - 1) / step) * step;
  k_tc_minmax<<<blocks, 256, 0, s>>>(p, count, d, slots);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status tc_pack(uotk_ctx* ctx, cudaStream_t s, const float* pts, const float* w, int d,
                    int dc, const float* center, double eps, TcCloud& C) {
  if (C.tiles == 0) return UOTK_OK;
  const long long n_pad = C.tiles * TC_ROWS;
  k_tc_pack<<<grid_for(ctx, n_pad * 8 * dc, 256, 4), 256, 0, s>>>(pts, C.n, n_pad, d, dc, center,
                                                                   C.tile_data);
  UOTK_LAUNCHED(ctx);
  k_tc_norms<<<grid_for(ctx, n_pad, 256, 4), 256, 0, s>>>(
      pts, w, C.n, n_pad, d, center, (float)(-1.4426950408889634 / eps), C.n2, C.bw, ctx->dflags);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

}  // namespace

size_t tc_engine_bytes(uotk_ctx* ctx, const EngineSpec& sp) {
  Carver cv(nullptr);
  TcEngine::carve(ctx, sp, cv, nullptr);
  return cv.off;
}

uotk_status tc_engine_create(uotk_ctx* ctx, cudaStream_t s, const EngineSpec& sp, Carver& cv,
                             Engine** out) {
  std::unique_ptr<TcEngine> e(new TcEngine());
  e->ctx = ctx;
  e->d = sp.d;
  e->n = sp.n;
  e->m = sp.m;
  e->a = sp.a;
  e->b = sp.b;
  e->eps = sp.eps;
  e->split = sp.method == UOTK_DIRECT_BF16X3;
  TcEngine::carve(ctx, sp, cv, e.get());
  {
    UOTK_PROF(ctx, s, "pack");
    k_tc_fill_slots<<<1, 256, 0, s>>>(e->slots, 2 * sp.d);
    UOTK_LAUNCHED(ctx);
    UOTK_TRY(tc_minmax(ctx, s, sp.x, sp.n, sp.d, e->slots));
    UOTK_TRY(tc_minmax(ctx, s, sp.y, sp.m, sp.d, e->slots));
    k_tc_center<<<1, 128, 0, s>>>(e->slots, sp.d, e->center, e->r2);
    UOTK_LAUNCHED(ctx);
    UOTK_CUDA(ctx, cudaMemcpyAsync(ctx->host + 24, e->r2, sizeof(double), cudaMemcpyDeviceToHost, s));
    UOTK_CUDA(ctx, cudaStreamSynchronize(s));
    const double r2 = ctx->host[24] * 1.0001;  // margin for the FP32 rounding of the centre
    e->fast = r2 * 1.4426950408889634 / sp.eps <= 64.0;
    UOTK_TRY(tc_pack(ctx, s, sp.x, sp.a, sp.d, e->dc, e->center, sp.eps, e->X));
    UOTK_TRY(tc_pack(ctx, s, sp.y, sp.b, sp.d, e->dc, e->center, sp.eps, e->Y));
  }
  *out = e.release();
  return UOTK_OK;
}

}  // namespace uotk
