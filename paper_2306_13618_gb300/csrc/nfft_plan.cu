// NFFT plan and point preprocessing (Sec. 4): torus scaling, the Kaiser-Bessel
// window and its Fourier coefficients, the Gaussian's Fourier coefficients
// b_k, binning of the points by grid tile, and the per-point window weights.
#include <math.h>

#include "nfft.cuh"

namespace uotk {

namespace {

// I_0(x) = sum_j ((x/2)^j / j!)^2, summed in FP64 until the terms vanish.
double bessel_i0(double x) {
  const double q = 0.25 * x * x;
  double term = 1.0, sum = 1.0;
  for (int j = 1; j < 500; ++j) {
    term *= q / ((double)j * (double)j);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  return sum;
}

// Upper bound of the Kaiser-Bessel window error for cut-off m and oversampling
// sigma (the standard bound of the NFFT literature), relative to sum |w|.
double kb_error_bound(int m, double sigma) {
  const double r = sqrt(1.0 - 1.0 / sigma);
  return 4.0 * M_PI * (sqrt((double)m) + m) * sqrt(r) * exp(-2.0 * M_PI * m * r);
}

__global__ void k_bbox(const float* __restrict__ p, long long n, int d, long long* __restrict__ slots) {
  float mx[3] = {-INFINITY, -INFINITY, -INFINITY}, mn[3] = {INFINITY, INFINITY, INFINITY};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    for (int t = 0; t < d; ++t) {
      const float v = p[i * d + t];
      mx[t] = fmaxf(mx[t], v);
      mn[t] = fminf(mn[t], v);
    }
  for (int t = 0; t < d; ++t) {
    double a = mx[t], b = -(double)mn[t];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a = fmax(a, __shfl_xor_sync(0xffffffffu, a, o));
      b = fmax(b, __shfl_xor_sync(0xffffffffu, b, o));
    }
    if ((threadIdx.x & 31) == 0) {
      atomicMax(&slots[t], dbl_to_ordered(a));
      atomicMax(&slots[3 + t], dbl_to_ordered(b));
    }
  }
}

__global__ void k_bbox_reset(long long* slots) {
  if (threadIdx.x < 6) slots[threadIdx.x] = ORDERED_NEG_INF;
}

struct CellRule {
  float c[3];
  float inv_h;
  int n, d;
};

// Cell and fraction of one point by the FP32 rule of the header, one IEEE
// rounding per operation (no contraction).
__device__ __forceinline__ void cell_of(const float* __restrict__ p, const CellRule& R, int cell[3],
                                        float frac[3]) {
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const float x = t < R.d ? p[t] : R.c[t];
    float v = __fsub_rn(x, R.c[t]);
    v = __fmul_rn(v, R.inv_h);
    v = __fadd_rn(v, 0.5f);
    v = __fmul_rn(v, (float)R.n);
    const float fl = floorf(v);
    frac[t] = __fsub_rn(v, fl);
    int ci = (int)fl % R.n;
    cell[t] = ci < 0 ? ci + R.n : ci;
  }
}

__global__ void k_cells(const float* __restrict__ pts, long long n, CellRule R,
                        int* __restrict__ out) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    float f[3];
    cell_of(pts + i * R.d, R, c, f);
    out[3 * i] = c[0];
    out[3 * i + 1] = c[1];
    out[3 * i + 2] = c[2];
  }
}

// Cell key: tile-major, then z, y, x inside the tile, so that the points of a
// tile, and inside it the points of a cell, are contiguous after sorting.
__device__ __forceinline__ int cell_key(const int c[3], int tiles1) {
  const int tile = ((c[2] / NFFT_TILE) * tiles1 + c[1] / NFFT_TILE) * tiles1 + c[0] / NFFT_TILE;
  const int local = ((c[2] % NFFT_TILE) * NFFT_TILE + c[1] % NFFT_TILE) * NFFT_TILE + c[0] % NFFT_TILE;
  return tile * (NFFT_TILE * NFFT_TILE * NFFT_TILE) + local;
}

__global__ void k_bin_count(const float* __restrict__ pts, long long n, CellRule R, int tiles1,
                            int4* __restrict__ tmp_cell, int* __restrict__ tmp_key,
                            int* __restrict__ count) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    int c[3];
    float f[3];
    cell_of(pts + i * R.d, R, c, f);
    const int key = cell_key(c, tiles1);
    tmp_key[i] = key;
    tmp_cell[i] = make_int4(c[0] | (c[1] << 10) | (c[2] << 20), __float_as_int(f[0]),
                            __float_as_int(f[1]), __float_as_int(f[2]));
    atomicAdd(&count[key], 1);
  }
}

// Exclusive scan of the n^3 cell counts: blocks of 2048 (eight per thread),
// block sums scanned by one block, then added back.  Counts are zeroed as they
// are read (they become the scatter cursors).
constexpr int SCAN_BLOCK = 2048;

__global__ void __launch_bounds__(256) k_scan_local(int* __restrict__ count, long long total,
                                                    int* __restrict__ start,
                                                    int* __restrict__ block_sums) {
  // 256 threads x 8 consecutive entries: serial sums per thread, a shuffle scan
  // of the thread totals per warp, then of the eight warp totals
  constexpr int PER = SCAN_BLOCK / 256;
  __shared__ int wsum[8];
  const long long base = (long long)blockIdx.x * SCAN_BLOCK + (long long)threadIdx.x * PER;
  int v[PER];
  int run = 0;
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const long long i = base + k;
    v[k] = 0;
    if (i < total) {
      v[k] = count[i];
      count[i] = 0;
    }
    run += v[k];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = run;  // inclusive scan of the thread totals in the warp
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    int w = lane < 8 ? wsum[lane] : 0;
#pragma unroll
    for (int o = 1; o < 8; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, w, o);
      if (lane >= o) w += t;
    }
    if (lane < 8) wsum[lane] = w;  // inclusive warp prefix
  }
  __syncthreads();
  int off = inc - run + (warp ? wsum[warp - 1] : 0);  // exclusive prefix of this thread
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const long long i = base + k;
    if (i < total) start[i] = off;
    off += v[k];
  }
  if (threadIdx.x == 0) block_sums[blockIdx.x] = wsum[7];
}

__global__ void __launch_bounds__(1024) k_scan_top(int* __restrict__ block_sums, int nb) {
  __shared__ int sh[1024];
  __shared__ int carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < nb; base += 1024) {
    const int i = base + threadIdx.x;
    const int v = i < nb ? block_sums[i] : 0;
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const int a = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
      __syncthreads();
      sh[threadIdx.x] += a;
      __syncthreads();
    }
    if (i < nb) block_sums[i] = carry + sh[threadIdx.x] - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry += sh[1023];
    __syncthreads();
  }
  if (threadIdx.x == 0) block_sums[nb] = carry;
}

__global__ void k_scan_add(int* __restrict__ start, long long total,
                           const int* __restrict__ block_sums, int nb) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x)
    start[i] += block_sums[i / SCAN_BLOCK];
  if (blockIdx.x == 0 && threadIdx.x == 0) start[total] = block_sums[nb];
}

__global__ void k_tile_counts(const int* __restrict__ cell_start, int tiles,
                              int* __restrict__ count) {
  constexpr int T3 = NFFT_TILE * NFFT_TILE * NFFT_TILE;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x)
    count[t] = cell_start[(long long)(t + 1) * T3] - cell_start[(long long)t * T3];
}

// 1 where a cell holds points (from the scanned counts), for the cell ranks.
__global__ void k_occ_flags(const int* __restrict__ cell_start, long long cells,
                            int* __restrict__ flag) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < cells;
       c += (long long)gridDim.x * blockDim.x)
    flag[c] = cell_start[c + 1] > cell_start[c];
}

// Cost of sorted point p of a tile with occupied-tile rank r (see nfft.cuh):
// p + cell_cost (occupied cells up to p's cell) + tile_cost (r + 1).
__device__ __forceinline__ long long point_cost(int p, int cells_upto, int r, int cell_cost,
                                                int tile_cost) {
  return (long long)p + (long long)cell_cost * cells_upto + (long long)tile_cost * (r + 1);
}

// Single block.  Pass 1: exclusive scans of the points per tile (tile_start)
// and of the occupied tiles (tile_rank), then the cost per chunk of the spread
// and of the gather: Q = max(min chunk, ceil(total cost / chunks)).  Pass 2:
// the work units per tile, one per chunk its cost range meets, scanned (tus_a,
// tus_b, totals num_a, num_b).
__global__ void k_bin_scan(const int* __restrict__ count, const int* __restrict__ cell_rank,
                           int tiles, int chunks_a, int chunks_b,
                           int* __restrict__ tile_start, int* __restrict__ tile_rank,
                           long long* __restrict__ chunk_q, int* __restrict__ tus_a,
                           int* __restrict__ num_a, int* __restrict__ tus_b,
                           int* __restrict__ num_b) {
  constexpr int T3 = NFFT_TILE * NFFT_TILE * NFFT_TILE;
  __shared__ int sa[1024], sb[1024];
  __shared__ int carry_a, carry_b;
  __shared__ long long qa, qb;
  if (threadIdx.x == 0) { carry_a = 0; carry_b = 0; }
  __syncthreads();
  for (int pass = 0; pass < 2; ++pass) {
    for (int base = 0; base < tiles; base += 1024) {
      const int i = base + threadIdx.x;
      int ca = 0, cb = 0;
      if (i < tiles) {
        if (pass == 0) {
          ca = count[i];
          cb = ca > 0;
        } else {
          const int b = tile_start[i], e = tile_start[i + 1];
          if (e > b) {
            // occupied cells up to the tile's first and last occupied cell
            const int c0 = cell_rank[(long long)i * T3] + 1, c1 = cell_rank[(long long)(i + 1) * T3];
            const int r = tile_rank[i];
            ca = (int)(point_cost(e - 1, c1, r, NFFT_SPREAD_CELL_COST, NFFT_SPREAD_TILE_COST) / qa -
                       point_cost(b, c0, r, NFFT_SPREAD_CELL_COST, NFFT_SPREAD_TILE_COST) / qa) + 1;
            cb = (int)(point_cost(e - 1, c1, r, NFFT_GATHER_CELL_COST, NFFT_GATHER_TILE_COST) / qb -
                       point_cost(b, c0, r, NFFT_GATHER_CELL_COST, NFFT_GATHER_TILE_COST) / qb) + 1;
          }
        }
      }
      sa[threadIdx.x] = ca;
      sb[threadIdx.x] = cb;
      __syncthreads();
      for (int o = 1; o < 1024; o <<= 1) {
        const int y = threadIdx.x >= o ? sa[threadIdx.x - o] : 0;
        const int z = threadIdx.x >= o ? sb[threadIdx.x - o] : 0;
        __syncthreads();
        sa[threadIdx.x] += y;
        sb[threadIdx.x] += z;
        __syncthreads();
      }
      if (i < tiles) {
        if (pass == 0) {
          tile_start[i] = carry_a + sa[threadIdx.x] - ca;
          tile_rank[i] = carry_b + sb[threadIdx.x] - cb;
        } else {
          tus_a[i] = carry_a + sa[threadIdx.x] - ca;
          tus_b[i] = carry_b + sb[threadIdx.x] - cb;
        }
      }
      __syncthreads();
      if (threadIdx.x == 1023) {
        carry_a += sa[1023];
        carry_b += sb[1023];
      }
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      if (pass == 0) {
        const int n = carry_a, occ = carry_b, cells = cell_rank[(long long)tiles * T3];
        tile_start[tiles] = carry_a;
        tile_rank[tiles] = carry_b;
        // total cost: one past the last point's
        const long long ta = point_cost(n, cells, occ - 1, NFFT_SPREAD_CELL_COST,
                                        NFFT_SPREAD_TILE_COST);
        const long long tb = point_cost(n, cells, occ - 1, NFFT_GATHER_CELL_COST,
                                        NFFT_GATHER_TILE_COST);
        qa = max((long long)NFFT_SPREAD_MIN_CHUNK, (ta + chunks_a - 1) / chunks_a);
        qb = max((long long)NFFT_GATHER_MIN_CHUNK, (tb + chunks_b - 1) / chunks_b);
        chunk_q[0] = qa;
        chunk_q[1] = qb;
        carry_a = 0;
        carry_b = 0;
      } else {
        tus_a[tiles] = carry_a;
        tus_b[tiles] = carry_b;
        *num_a = carry_a;
        *num_b = carry_b;
      }
    }
    __syncthreads();
  }
}

// Stable LSD radix sort of the cell keys, 8-bit digits: the points of one cell
// keep their caller order, so the sorted order (and every FP32 sum taken in it)
// is the same on every run.  A CTA owns RS_TILE consecutive elements; its
// per-digit counts go digit-major into hist[digit * blocks + cta], whose
// exclusive scan gives each (digit, CTA) its first output position.
constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;

__global__ void __launch_bounds__(RS_THREADS)
    k_rs_hist(const int* __restrict__ keys, long long n, int shift, int blocks,
              int* __restrict__ hist) {
  __shared__ int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const long long b0 = (long long)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = b0 + (long long)r * RS_THREADS + threadIdx.x;
    if (i < n) atomicAdd(&h[(keys[i] >> shift) & 255], 1);  // integer counts: order-free
  }
  __syncthreads();
  hist[threadIdx.x * blocks + blockIdx.x] = h[threadIdx.x];
}

// Element i of the CTA's tile goes to start[digit][cta] + (number of earlier
// elements of the tile with the same digit): earlier iterations of the tile
// loop (base), earlier warps of this iteration (cnt), earlier lanes of this
// warp (match mask).
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scatter(const int* __restrict__ kin, const int* __restrict__ vin, long long n, int shift,
                 int blocks, const int* __restrict__ start, int* __restrict__ kout,
                 int* __restrict__ vout) {
  constexpr int NW = RS_THREADS / 32;
  __shared__ int base[256];
  __shared__ int cnt[NW][256];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  base[threadIdx.x] = start[threadIdx.x * blocks + blockIdx.x];
  for (int k = threadIdx.x; k < NW * 256; k += RS_THREADS) (&cnt[0][0])[k] = 0;
  __syncthreads();
  const long long b0 = (long long)blockIdx.x * RS_TILE;
  for (int r = 0; r < RS_ITEMS; ++r) {
    const long long i = b0 + (long long)r * RS_THREADS + threadIdx.x;
    const bool valid = i < n;
    const int key = valid ? kin[i] : 0;
    // lanes past the end take distinct out-of-range digits: no peers, no counts
    const int dg = valid ? (key >> shift) & 255 : 256 + lane;
    const unsigned peers = __match_any_sync(0xffffffffu, dg);
    const int rank = __popc(peers & ((1u << lane) - 1u));
    const bool leader = rank == 0;
    if (valid && leader) cnt[w][dg] = __popc(peers);
    __syncthreads();
    int pos = 0;
    if (valid) {
      pos = base[dg] + rank;
      for (int w2 = 0; w2 < w; ++w2) pos += cnt[w2][dg];
    }
    __syncthreads();
    if (valid && leader) {
      atomicAdd(&base[dg], __popc(peers));  // integer: order-free
      cnt[w][dg] = 0;
    }
    if (valid) {
      kout[pos] = key;
      vout[pos] = vin ? vin[i] : (int)i;
    }
    __syncthreads();
  }
}

// Sorted position -> packed cell, key and caller index.
__global__ void k_bin_place(const int4* __restrict__ tmp_cell, const int* __restrict__ order,
                            long long n, int4* __restrict__ cell, int* __restrict__ ckey,
                            int* __restrict__ perm) {
  for (long long p = blockIdx.x * (long long)blockDim.x + threadIdx.x; p < n;
       p += (long long)gridDim.x * blockDim.x) {
    const int i = order[p];
    const int4 c = tmp_cell[i];
    cell[p] = c;
    ckey[p] = c.x;
    perm[p] = i;
  }
}

// Cost of sorted point p from its cell key (the point costs of nfft.cuh).
__device__ __forceinline__ long long sorted_point_cost(int p, const int* __restrict__ ckey,
                                                       const int* __restrict__ cell_rank,
                                                       const int* __restrict__ tile_rank,
                                                       int tiles1, int cell_cost, int tile_cost) {
  const int k = ckey[p];
  const int c[3] = {k & 1023, (k >> 10) & 1023, k >> 20};
  const int cell = cell_key(c, tiles1);
  return point_cost(p, cell_rank[cell] + 1, tile_rank[cell / (NFFT_TILE * NFFT_TILE * NFFT_TILE)],
                    cell_cost, tile_cost);
}

// first[c] = the first sorted point whose cost reaches c q (n if none),
// c = 0 .. chunks, by bisection (the costs increase along the sorted points).
__global__ void k_chunk_first(const int* __restrict__ ckey, const int* __restrict__ cell_rank,
                              const int* __restrict__ tile_rank, int n, int tiles1,
                              const long long* __restrict__ chunk_q, int which, int cell_cost,
                              int tile_cost, int chunks, int* __restrict__ first) {
  const long long q = chunk_q[which];
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= chunks; c += gridDim.x * blockDim.x) {
    int lo = 0, hi = n;
    while (lo < hi) {
      const int mid = lo + ((hi - lo) >> 1);
      if (sorted_point_cost(mid, ckey, cell_rank, tile_rank, tiles1, cell_cost, tile_cost) <
          (long long)c * q)
        lo = mid + 1;
      else
        hi = mid;
    }
    first[c] = lo;
  }
}

// The work units of each tile: its sorted points [b, e) cut at the first
// points of the chunks that start inside it; chunk(b) .. chunk(e - 1) are the
// tile's chunks (no chunk is skipped inside a tile: consecutive points differ
// in cost by at most 1 + cell cost < q).  unit_chunk gets each unit's chunk.
__global__ void k_make_units(const int* __restrict__ tile_start,
                             const int* __restrict__ tile_rank, const int* __restrict__ cell_rank,
                             const int* __restrict__ ckey, const int* __restrict__ tile_unit_start,
                             int tiles, int tiles1, const long long* __restrict__ chunk_q,
                             int which, int cell_cost, int tile_cost,
                             const int* __restrict__ first, int* __restrict__ unit_tile,
                             int* __restrict__ unit_begin, int* __restrict__ unit_count,
                             int* __restrict__ unit_chunk) {
  const long long q = chunk_q[which];
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
    const int b = tile_start[t], e = tile_start[t + 1];
    if (e <= b) continue;
    const int c0 = (int)(sorted_point_cost(b, ckey, cell_rank, tile_rank, tiles1, cell_cost,
                                           tile_cost) / q);
    const int c1 = (int)(sorted_point_cost(e - 1, ckey, cell_rank, tile_rank, tiles1, cell_cost,
                                           tile_cost) / q);
    int u = tile_unit_start[t], p = b;
    for (int c = c0; c <= c1; ++c, ++u) {
      const int end = c < c1 ? first[c + 1] : e;
      unit_tile[u] = t;
      unit_begin[u] = p;
      unit_count[u] = end - p;
      unit_chunk[u] = c;
      p = end;
    }
  }
}

// chunk_unit_start[c] = the first unit of chunk c or later (units are in
// chunk order), c = 0 .. chunks; chunks past the last unit start at num.
__global__ void k_chunk_starts(const int* __restrict__ unit_chunk, const int* __restrict__ num,
                               int chunks, int* __restrict__ chunk_unit_start) {
  const int nu = *num;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c <= chunks; c += gridDim.x * blockDim.x) {
    int lo = 0, hi = nu;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (unit_chunk[mid] < c) lo = mid + 1;
      else hi = mid;
    }
    chunk_unit_start[c] = lo;
  }
}

// Normalised Kaiser-Bessel window at distance v (grid units, |v| < m):
// phi(v)/phi(0) = (m/s) e^{b(s-m)} (1 - e^{-2bs}) / (1 - e^{-2bm}),  s = sqrt(m^2 - v^2).
__device__ __forceinline__ float kb_window(float v, int m, float b) {
  const float mf = (float)m;
  const float s2 = fmaxf(mf * mf - v * v, 0.f);
  const float s = sqrtf(s2);
  const float den = -expm1f(-2.f * b * mf);
  if (s < 1e-4f) return mf * 2.f * b * expf(-b * mf) / den;
  return mf * expf(b * (s - mf)) * (-expm1f(-2.f * b * s)) / (s * den);
}

// Window tables.  A CTA takes WIN_PTS consecutive sorted points, thread (q, t)
// evaluates the 2m values of point q along axis t into a shared-memory copy
// of the CTA's rows (with their padding), and the CTA then writes its rows,
// which are contiguous in the table, with 16-byte stores.
constexpr int WIN_PTS = 64;
constexpr int WIN_SMEM_F = WIN_PTS * 48;  // rows of the largest stride (m = 8): 48 floats a point

// Gather layout (nfft.cuh): point q's row, phi_x halves, phi_y, phi_z.
__global__ void __launch_bounds__(3 * WIN_PTS)
    k_windows(const int4* __restrict__ cell, long long n, int m, float b,
              float* __restrict__ win) {
  __shared__ __align__(16) float buf[WIN_SMEM_F];
  const int ws = nfft_win_stride(m), hp = nfft_win_half(m);
  const int yo = nfft_win_yoff(m), zo = nfft_win_zoff(m);
  for (long long q0 = (long long)blockIdx.x * WIN_PTS; q0 < n; q0 += (long long)gridDim.x * WIN_PTS) {
    const int np = (int)min((long long)WIN_PTS, n - q0);
    for (int i = threadIdx.x; i < np * ws; i += blockDim.x) buf[i] = 0.f;
    __syncthreads();
    const int qi = threadIdx.x / 3, t = threadIdx.x - 3 * qi;
    if (qi < np) {
      const int4 c = cell[q0 + qi];
      const float f = __int_as_float(t == 0 ? c.y : (t == 1 ? c.z : c.w));
      float* row = buf + qi * ws;
      for (int k = 0; k < 2 * m; ++k) {
        const int r = t == 0 ? (k < m ? k : hp + k - m) : (t == 1 ? yo : zo) + k;
        row[r] = kb_window(f + (float)(m - 1 - k), m, b);
      }
    }
    __syncthreads();
    float4* dst = reinterpret_cast<float4*>(win + q0 * ws);
    const float4* src = reinterpret_cast<const float4*>(buf);
    for (int i = threadIdx.x; i < np * ws / 4; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
}

// Pair layout (nfft.cuh): row p holds, for every window value, the pair
// (point 2p, point 2p + 1); a missing second point (odd n) gets zeros.
__global__ void __launch_bounds__(3 * WIN_PTS)
    k_windows_pair(const int4* __restrict__ cell, long long n, int m, float b,
                   float* __restrict__ win) {
  __shared__ __align__(16) float buf[WIN_SMEM_F];
  const int ws = nfft_winp_stride(m), hp = nfft_winp_half(m);
  const int yo = nfft_winp_yoff(m), zo = nfft_winp_zoff(m);
  const long long n2 = (n + 1) & ~1LL;
  for (long long q0 = (long long)blockIdx.x * WIN_PTS; q0 < n2; q0 += (long long)gridDim.x * WIN_PTS) {
    const int np = (int)min((long long)WIN_PTS, n2 - q0);  // even
    for (int i = threadIdx.x; i < np / 2 * ws; i += blockDim.x) buf[i] = 0.f;
    __syncthreads();
    const int qi = threadIdx.x / 3, t = threadIdx.x - 3 * qi;
    if (qi < np && q0 + qi < n) {
      const int4 c = cell[q0 + qi];
      const float f = __int_as_float(t == 0 ? c.y : (t == 1 ? c.z : c.w));
      float* row = buf + (qi >> 1) * ws + (qi & 1);
      for (int k = 0; k < 2 * m; ++k) {
        const int r = t == 0 ? (k / m) * hp + 2 * (k % m) : (t == 1 ? yo : zo) + 2 * k;
        row[r] = kb_window(f + (float)(m - 1 - k), m, b);
      }
    }
    __syncthreads();
    float4* dst = reinterpret_cast<float4*>(win + (q0 >> 1) * ws);
    const float4* src = reinterpret_cast<const float4*>(buf);
    for (int i = threadIdx.x; i < np / 2 * ws / 4; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  }
}

}  // namespace

int nfft_max_units(const NfftParams& P, int64_t n, int chunks) {
  const int64_t tiles = (int64_t)P.tiles1 * P.tiles1 * P.tiles1;
  return (int)(chunks + (n < tiles ? n : tiles));
}

uotk_status nfft_make_params(uotk_ctx* ctx, int d, const float lo[3], const float hi[3],
                             double eps, const uotk_sum_opts* opts, NfftParams* P) {
  P->d = d;
  P->kernel = opts ? opts->kernel : UOTK_KERNEL_GAUSS;
  const bool reg = P->kernel != UOTK_KERNEL_GAUSS;
  P->n = (opts && opts->grid) ? opts->grid : (reg ? 256 : 128);
  P->N = (opts && opts->bandwidth) ? opts->bandwidth : P->n / 2;
  P->eps = eps;
  const double sigma = (double)P->n / P->N;
  P->b = (float)(M_PI * (2.0 - 1.0 / sigma));
  double L = 0.0, D2 = 0.0;
  for (int t = 0; t < 3; ++t) {
    if (t < d) {
      P->c[t] = (float)(0.5 * ((double)lo[t] + (double)hi[t]));
      L = fmax(L, (double)hi[t] - (double)lo[t]);
      D2 += ((double)hi[t] - (double)lo[t]) * ((double)hi[t] - (double)lo[t]);
    } else {
      P->c[t] = 0.f;
    }
  }
  if (!isfinite(L)) return set_error(ctx, UOTK_ERR_NONFINITE, "NFFT plan: non-finite coordinates");
  const double target = (opts && opts->target_err > 0) ? opts->target_err : 1e-6;
  if (reg) {
    // Sec. 4.2: every difference must stay where K_R = K or the near field
    // corrects it, |x - y| <= (1/2 - eps_B) h; eps_I = eps_B = p/N.
    if (P->n < 2 * P->N)
      return set_error(ctx, UOTK_ERR_INVALID,
                       "NFFT: the non-Gaussian kernels need oversampling grid >= 2 bandwidth");
    P->reg_p = (opts && opts->reg_degree) ? opts->reg_degree : 4;
    P->reg_target = (opts && opts->target_err > 0) ? opts->target_err : 1e-3;
    if (P->reg_p < 2 || P->reg_p > 12)
      return set_error(ctx, UOTK_ERR_INVALID, "NFFT: regularisation degree %d not in [2, 12]",
                       P->reg_p);
    P->eps_i = (double)P->reg_p / P->N;
    if (P->eps_i > 0.125)
      return set_error(ctx, UOTK_ERR_INVALID,
                       "NFFT: regularisation width p/N = %d/%d above 1/8; raise the bandwidth",
                       P->reg_p, P->N);
    const double diam = sqrt(D2);
    const double hmin = diam / (0.5 - P->eps_i);
    if (opts && opts->period > 0) {
      P->h = opts->period;
      if (P->h < hmin * (1.0 + 1e-6))
        return set_error(ctx, UOTK_ERR_INVALID,
                         "NFFT: period %g below %g = diameter / (1/2 - eps_B) of the points",
                         P->h, hmin);
    } else {
      P->h = hmin > 0.0 ? hmin * (1.0 + 1e-6) : 1.0;
    }
  } else if (opts && opts->period > 0) {
    P->h = opts->period;
  } else {
    // Balance the periodisation error exp(-(h-L)^2/eps) against the Fourier
    // truncation error exp(-pi^2 eps N^2 / (4 h^2)): h (h - L) = pi eps N / 2.
    P->h = 0.5 * (L + sqrt(L * L + 2.0 * M_PI * eps * P->N));
    const double e1 = (P->h - L) * (P->h - L) / eps;
    if (exp(-e1) > 0.1 * target)
      return set_error(ctx, UOTK_ERR_UNSUPPORTED,
                       "NFFT: bandwidth %d too small for eps %g over a point spread of %g "
                       "(estimated error %.1e > target %.1e); raise grid/bandwidth", P->N, eps, L,
                       exp(-e1), target);
  }
  // the kernels scale by the FP32 value inv_h; h is its exact reciprocal, so the
  // Fourier coefficients b_k describe the scaling actually applied
  P->inv_h = (float)(1.0 / P->h);
  P->h = 1.0 / (double)P->inv_h;
  if (opts && opts->cutoff) {
    P->m = opts->cutoff;
  } else {
    P->m = 8;
    for (int m = 6; m <= 8; ++m)
      if (kb_error_bound(m, sigma) <= target) { P->m = m; break; }
  }
  if (2 * P->m > P->n) return set_error(ctx, UOTK_ERR_INVALID, "NFFT: 2m > grid");
  P->tiles1 = P->n / NFFT_TILE;
  P->E = NFFT_TILE + 2 * P->m - 1;
  return UOTK_OK;
}

void nfft_deconv_rows(const NfftParams& P, double* rows) {
  const double b = M_PI * (2.0 - (double)P.N / P.n);
  const double m = P.m;
  const double sh = sinh(b * m);
  for (int t = 0; t < 3; ++t)
    for (int i = 0; i < P.N; ++i) {
      const double k = i - P.N / 2;
      const double arg = b * b - pow(2.0 * M_PI * k / P.n, 2);
      const double nph = bessel_i0(m * sqrt(arg > 0 ? arg : 0.0)) * M_PI * m / sh;
      rows[t * P.N + i] = (t < P.d || i == P.N / 2) ? 1.0 / (nph * nph) : 0.0;
    }
}

void nfft_scale_table(const NfftParams& P, float* table) {
  // scale_k = b_k / prod_t (n phihat_s(k_t))^2 is separable: row t holds
  // g_t(k) = sqrt(pi eps)/h exp(-pi^2 eps k^2/h^2) / (n phihat_s(k))^2 for a real
  // dimension, and [k == 0] / (n phihat_s(0))^2 for an embedded one (constant 1).
  // n phihat_s(k) = I_0(m sqrt(b^2 - (2 pi k/n)^2)) * pi m / sinh(b m).
  const double b = M_PI * (2.0 - (double)P.N / P.n);
  const double m = P.m;
  const double sh = sinh(b * m);
  for (int t = 0; t < 3; ++t)
    for (int i = 0; i < P.N; ++i) {
      const double k = i - P.N / 2;
      const double arg = b * b - pow(2.0 * M_PI * k / P.n, 2);
      const double nph = bessel_i0(m * sqrt(arg > 0 ? arg : 0.0)) * M_PI * m / sh;
      double g;
      if (t < P.d)
        g = sqrt(M_PI * P.eps) / P.h * exp(-M_PI * M_PI * P.eps * k * k / (P.h * P.h)) / (nph * nph);
      else
        g = (i == P.N / 2) ? 1.0 / (nph * nph) : 0.0;
      table[t * P.N + i] = (float)g;
    }
}

uotk_status nfft_bbox(uotk_ctx* ctx, cudaStream_t s, int d, const float* a, int64_t na,
                      const float* b, int64_t nb, float lo[3], float hi[3]) {
  long long* slots = ctx->dflags + FLAG_BBOX;
  k_bbox_reset<<<1, 32, 0, s>>>(slots);
  UOTK_LAUNCHED(ctx);
  if (na > 0) {
    k_bbox<<<grid_for(ctx, na, 256, 4), 256, 0, s>>>(a, na, d, slots);
    UOTK_LAUNCHED(ctx);
  }
  if (nb > 0) {
    k_bbox<<<grid_for(ctx, nb, 256, 4), 256, 0, s>>>(b, nb, d, slots);
    UOTK_LAUNCHED(ctx);
  }
  long long* h = reinterpret_cast<long long*>(ctx->host + 96);
  UOTK_CUDA(ctx, cudaMemcpyAsync(h, slots, 6 * sizeof(long long), cudaMemcpyDeviceToHost, s));
  UOTK_CUDA(ctx, cudaStreamSynchronize(s));
  for (int t = 0; t < 3; ++t) {
    if (t < d) {
      hi[t] = (float)ordered_to_dbl(h[t]);
      lo[t] = (float)(-ordered_to_dbl(h[3 + t]));
    } else {
      hi[t] = lo[t] = 0.f;
    }
  }
  return UOTK_OK;
}

size_t nfft_points_bytes(const NfftParams& P, int64_t n) {
  Carver cv(nullptr);
  NfftPoints S;
  nfft_points_carve(cv, P, n, S);
  return cv.off;
}

void nfft_points_carve(Carver& cv, const NfftParams& P, int64_t n, NfftPoints& S) {
  const int tiles = P.tiles1 * P.tiles1 * P.tiles1;
  const int64_t nn = n > 0 ? n : 1;
  S.n = n;
  S.c_spread = nfft_spread_slots(P.m);
  S.c_gather = nfft_gather_slots(P.m);
  S.max_units = nfft_max_units(P, n, S.c_spread);
  S.g_max_units = nfft_max_units(P, n, S.c_gather);
  S.cell = cv.take<int4>(nn);
  S.ckey = cv.take<int>(nn + 4);
  S.win = cv.take<float>((size_t)nn * nfft_win_stride(P.m));
  S.winp = cv.take<float>((size_t)((nn + 1) / 2) * nfft_winp_stride(P.m));
  S.perm = cv.take<int>(nn);
  S.tile_start = cv.take<int>(tiles + 1);
  S.tile_rank = cv.take<int>(tiles + 1);
  S.chunk_q = cv.take<long long>(2);
  S.tile_unit_start = cv.take<int>(tiles + 1);
  S.unit_tile = cv.take<int>(S.max_units + 1);
  S.unit_begin = cv.take<int>(S.max_units + 1);
  S.unit_count = cv.take<int>(S.max_units + 1);
  S.unit_box = cv.take<int>(S.max_units + 1);
  S.num_units = cv.take<int>(1);
  S.unit_chunk = cv.take<int>(S.max_units + 1);
  S.chunk_unit_start = cv.take<int>(S.c_spread + 1);
  S.g_tile_unit_start = cv.take<int>(tiles + 1);
  S.g_unit_chunk = cv.take<int>(S.g_max_units + 1);
  S.g_chunk_unit_start = cv.take<int>(S.c_gather + 1);
  S.g_unit_tile = cv.take<int>(S.g_max_units + 1);
  S.g_unit_begin = cv.take<int>(S.g_max_units + 1);
  S.g_unit_count = cv.take<int>(S.g_max_units + 1);
  S.g_num_units = cv.take<int>(1);
  S.scratch = cv.take<int>(tiles);
  const long long n3 = (long long)P.n * P.n * P.n;
  S.cell_count = cv.take<int>(n3);
  S.cell_start = cv.take<int>(n3 + 1);
  S.cell_rank = cv.take<int>(n3 + 1);
  S.block_sums = cv.take<int>(n3 / 2048 + 2);
  // temporaries of the build: caller-order cells and the radix sort buffers
  const int64_t rb = (nn + RS_TILE - 1) / RS_TILE;
  S.tmp_cell = cv.take<int4>(nn);
  for (int k = 0; k < 2; ++k) {
    S.rs_key[k] = cv.take<int>(nn);
    S.rs_val[k] = cv.take<int>(nn);
  }
  S.rs_hist = cv.take<int>(256 * rb + 1);
  S.rs_start = cv.take<int>(256 * rb + 1);
  S.rs_bsum = cv.take<int>((256 * rb) / SCAN_BLOCK + 2);
}

uotk_status nfft_points_build(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                              const float* pts, int64_t n, NfftPoints& S) {
  const int tiles = P.tiles1 * P.tiles1 * P.tiles1;
  const long long n3 = (long long)P.n * P.n * P.n;
  const int nb = (int)((n3 + SCAN_BLOCK - 1) / SCAN_BLOCK);
  CellRule R{{P.c[0], P.c[1], P.c[2]}, P.inv_h, P.n, P.d};
  {
    UOTK_PROF(ctx, s, "bin");
    UOTK_CUDA(ctx, cudaMemsetAsync(S.cell_count, 0, sizeof(int) * n3, s));
    if (n > 0) {
      k_bin_count<<<grid_for(ctx, n, 256), 256, 0, s>>>(pts, n, R, P.tiles1, S.tmp_cell,
                                                         S.rs_key[0], S.cell_count);
      UOTK_LAUNCHED(ctx);
    }
    k_scan_local<<<nb, 256, 0, s>>>(S.cell_count, n3, S.cell_start, S.block_sums);
    UOTK_LAUNCHED(ctx);
    k_scan_top<<<1, 1024, 0, s>>>(S.block_sums, nb);
    UOTK_LAUNCHED(ctx);
    k_scan_add<<<grid_for(ctx, n3, 256), 256, 0, s>>>(S.cell_start, n3, S.block_sums, nb);
    UOTK_LAUNCHED(ctx);
    k_tile_counts<<<grid_for(ctx, tiles, 256), 256, 0, s>>>(S.cell_start, tiles, S.scratch);
    UOTK_LAUNCHED(ctx);
    // occupied-cell ranks (the counts are not needed any more: flags in place)
    k_occ_flags<<<grid_for(ctx, n3, 256), 256, 0, s>>>(S.cell_start, n3, S.cell_count);
    UOTK_LAUNCHED(ctx);
    k_scan_local<<<nb, 256, 0, s>>>(S.cell_count, n3, S.cell_rank, S.block_sums);
    UOTK_LAUNCHED(ctx);
    k_scan_top<<<1, 1024, 0, s>>>(S.block_sums, nb);
    UOTK_LAUNCHED(ctx);
    k_scan_add<<<grid_for(ctx, n3, 256), 256, 0, s>>>(S.cell_rank, n3, S.block_sums, nb);
    UOTK_LAUNCHED(ctx);
    k_bin_scan<<<1, 1024, 0, s>>>(S.scratch, S.cell_rank, tiles, S.c_spread, S.c_gather,
                                  S.tile_start, S.tile_rank, S.chunk_q, S.tile_unit_start,
                                  S.num_units, S.g_tile_unit_start, S.g_num_units);
    UOTK_LAUNCHED(ctx);
    if (n > 0) {
      // stable sort by cell key: ceil(bits / 8) passes over the key's bits
      int bits = 0;
      while ((1LL << bits) < n3) ++bits;
      const int rb = (int)((n + RS_TILE - 1) / RS_TILE);
      const long long hn = 256LL * rb;
      const int hb = (int)((hn + SCAN_BLOCK - 1) / SCAN_BLOCK);
      int cur = 0;
      for (int shift = 0; shift < bits; shift += 8, cur ^= 1) {
        k_rs_hist<<<rb, RS_THREADS, 0, s>>>(S.rs_key[cur], n, shift, rb, S.rs_hist);
        UOTK_LAUNCHED(ctx);
        k_scan_local<<<hb, 256, 0, s>>>(S.rs_hist, hn, S.rs_start, S.rs_bsum);
        UOTK_LAUNCHED(ctx);
        k_scan_top<<<1, 1024, 0, s>>>(S.rs_bsum, hb);
        UOTK_LAUNCHED(ctx);
        k_scan_add<<<grid_for(ctx, hn, 256), 256, 0, s>>>(S.rs_start, hn, S.rs_bsum, hb);
        UOTK_LAUNCHED(ctx);
        k_rs_scatter<<<rb, RS_THREADS, 0, s>>>(S.rs_key[cur], shift == 0 ? nullptr : S.rs_val[cur],
                                               n, shift, rb, S.rs_start, S.rs_key[cur ^ 1],
                                               S.rs_val[cur ^ 1]);
        UOTK_LAUNCHED(ctx);
      }
      k_bin_place<<<grid_for(ctx, n, 256), 256, 0, s>>>(S.tmp_cell, S.rs_val[cur], n, S.cell,
                                                         S.ckey, S.perm);
      UOTK_LAUNCHED(ctx);
    }
    // the chunks' first points (in the unit-start arrays, overwritten below)
    k_chunk_first<<<grid_for(ctx, S.c_spread + 1, 128), 128, 0, s>>>(
        S.ckey, S.cell_rank, S.tile_rank, (int)n, P.tiles1, S.chunk_q, 0, NFFT_SPREAD_CELL_COST,
        NFFT_SPREAD_TILE_COST, S.c_spread, S.chunk_unit_start);
    UOTK_LAUNCHED(ctx);
    k_chunk_first<<<grid_for(ctx, S.c_gather + 1, 128), 128, 0, s>>>(
        S.ckey, S.cell_rank, S.tile_rank, (int)n, P.tiles1, S.chunk_q, 1, NFFT_GATHER_CELL_COST,
        NFFT_GATHER_TILE_COST, S.c_gather, S.g_chunk_unit_start);
    UOTK_LAUNCHED(ctx);
    k_make_units<<<grid_for(ctx, tiles, 128), 128, 0, s>>>(
        S.tile_start, S.tile_rank, S.cell_rank, S.ckey, S.tile_unit_start, tiles, P.tiles1,
        S.chunk_q, 0, NFFT_SPREAD_CELL_COST, NFFT_SPREAD_TILE_COST, S.chunk_unit_start,
        S.unit_tile, S.unit_begin, S.unit_count, S.unit_chunk);
    UOTK_LAUNCHED(ctx);
    k_make_units<<<grid_for(ctx, tiles, 128), 128, 0, s>>>(
        S.tile_start, S.tile_rank, S.cell_rank, S.ckey, S.g_tile_unit_start, tiles, P.tiles1,
        S.chunk_q, 1, NFFT_GATHER_CELL_COST, NFFT_GATHER_TILE_COST, S.g_chunk_unit_start,
        S.g_unit_tile, S.g_unit_begin, S.g_unit_count, S.g_unit_chunk);
    UOTK_LAUNCHED(ctx);
    k_chunk_starts<<<grid_for(ctx, S.c_spread + 1, 256), 256, 0, s>>>(
        S.unit_chunk, S.num_units, S.c_spread, S.chunk_unit_start);
    UOTK_LAUNCHED(ctx);
    k_chunk_starts<<<grid_for(ctx, S.c_gather + 1, 256), 256, 0, s>>>(
        S.g_unit_chunk, S.g_num_units, S.c_gather, S.g_chunk_unit_start);
    UOTK_LAUNCHED(ctx);
  }
  S.win_ready = false;
  S.winp_ready = false;
  return UOTK_OK;
}

uotk_status nfft_points_windows(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                                const NfftPoints& S, bool pair) {
  const int64_t n = S.n;
  if (n == 0 || (pair ? S.winp_ready : S.win_ready)) return UOTK_OK;
  UOTK_PROF(ctx, s, "window");
  if (pair) {
    k_windows_pair<<<grid_for(ctx, (n + 1) / 2 * 6, 3 * WIN_PTS), 3 * WIN_PTS, 0, s>>>(
        S.cell, n, P.m, P.b, S.winp);
    S.winp_ready = true;
  } else {
    k_windows<<<grid_for(ctx, 3 * n, 3 * WIN_PTS), 3 * WIN_PTS, 0, s>>>(S.cell, n, P.m, P.b,
                                                                        S.win);
    S.win_ready = true;
  }
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status op_nfft_cells(uotk_ctx* ctx, cudaStream_t s, const uotk_nfft_plan_info* plan,
                          const float* pts, int64_t n, int32_t* cells) {
  if (n == 0) return UOTK_OK;
  CellRule R{{plan->center[0], plan->center[1], plan->center[2]}, plan->inv_h, plan->grid, plan->d};
  k_cells<<<grid_for(ctx, n, 256), 256, 0, s>>>(pts, n, R, cells);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

}  // namespace uotk
