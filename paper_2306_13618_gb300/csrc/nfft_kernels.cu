// NFFT stage kernels (Sec. 4, Eq. 1724): spread (adjoint NFFT step 1), the
// grid convolution (FFT, multiply by b_k and the double deconvolution,
// inverse FFT) and gather (NFFT final step).
//
// Spread.  Points are sorted by tile (16^3 cells).  A work unit is (tile, up to
// NFFT_UNIT_POINTS points); its CTA accumulates the windows of its points into
// an E^3 shared-memory block (E = 16 + 2m - 1, the tile plus the window halo)
// and writes the block out whole.  A fold kernel then adds, for every grid
// node, the blocks that cover it in unit order -- a fixed order, so the grid
// does not depend on scheduling between units.
// Gather.  The CTA of a unit stages the E^3 block of the grid around its tile
// in shared memory; a warp evaluates one target: lanes split the (2m)^2 (y, x)
// pairs of the footprint, loop over the 2m z-planes, and reduce by shuffles.
// FFT.  Radix-2 decimation-in-time on lines of n <= 256 complex values in
// shared memory (bit-reversed load, log2 n butterfly stages), 16 lines per CTA,
// lines adjacent in memory so every load and store is coalesced; passes along
// x, y, z.  The z pass multiplies by scale_k (zero outside I_N^3) between its
// forward and inverse transforms.
#include <math.h>

#include "nfft.cuh"

namespace uotk {

namespace {

constexpr int FFT_LINES = 16;
constexpr int FFT_THREADS = 256;

// ---------------------------------------------------------------- spread ----
constexpr int CH = 64;  // points staged in shared memory per chunk

// M floats of a window row from shared memory (8-byte vector loads when M is even).
template <int M>
__device__ __forceinline__ void load_row(const float* p, float* r) {
  if (M % 2 == 0) {
#pragma unroll
    for (int j = 0; j < M; j += 2) {
      const float2 v = *reinterpret_cast<const float2*>(p + j);
      r[j] = v.x;
      r[j + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < M; ++j) r[j] = p[j];
  }
}

// One CTA per work unit.  Thread (row r = (kz, ky), half) owns the M nodes
// kx in [half*M, half*M + M) of footprint row (kz, ky).  The points of one grid
// cell share the footprint: their rank-1 window products are accumulated in
// registers, then added to the block once; a barrier separates the additions of
// consecutive cells, so no two threads ever update a node at the same time.
template <int M>
__global__ void __launch_bounds__(8 * M * M)
    k_spread(const int4* __restrict__ cell, const float* __restrict__ win,
             const int* __restrict__ unit_tile, const int* __restrict__ unit_begin,
             const int* __restrict__ unit_count, const int* __restrict__ num_units, int tiles1,
             const float* __restrict__ base, const double* __restrict__ pot, double lam,
             const long long* __restrict__ shift_slot, float* __restrict__ part) {
  constexpr int W2 = 2 * M, E = NFFT_TILE + 2 * M - 1, E3 = E * E * E, WIN = 3 * W2;
  constexpr int NT = 8 * M * M;
  extern __shared__ float smem[];
  float* blk = smem;
  float* swin = blk + E3 + (E3 & 1);  // 8-byte aligned
  float* sw = swin + CH * WIN;
  int* skey = reinterpret_cast<int*>(sw + CH);
  const int u = blockIdx.x;
  if (u >= *num_units) return;
  for (int i = threadIdx.x; i < E3; i += NT) blk[i] = 0.f;
  const int tile = unit_tile[u];
  const int tx0 = (tile % tiles1) * NFFT_TILE;
  const int ty0 = ((tile / tiles1) % tiles1) * NFFT_TILE;
  const int tz0 = (tile / (tiles1 * tiles1)) * NFFT_TILE;
  const int r = threadIdx.x >> 1, half = threadIdx.x & 1;
  const int kz = r / W2, ky = r - kz * W2, kx0 = half * M;
  const double shift = pot ? ordered_to_dbl(*shift_slot) : 0.0;
  const int b0 = unit_begin[u], cnt = unit_count[u];
  for (int c0 = 0; c0 < cnt; c0 += CH) {
    const int cn = min(CH, cnt - c0);
    __syncthreads();
    const float* gw = win + (size_t)(b0 + c0) * WIN;
    for (int i = threadIdx.x; i < cn * WIN; i += NT) swin[i] = gw[i];
    for (int i = threadIdx.x; i < cn; i += NT) {
      const int q = b0 + c0 + i;
      const float bq = base ? base[q] : 1.f;
      sw[i] = pot ? bq * exp_shifted(lam * pot[q] - shift) : bq;
      skey[i] = cell[q].x;
    }
    __syncthreads();
    int p = 0;
    while (p < cn) {
      const int key = skey[p];
      float acc[M];
#pragma unroll
      for (int j = 0; j < M; ++j) acc[j] = 0.f;
      int q = p;
      for (; q < cn && skey[q] == key; ++q) {
        const float* wq = swin + q * WIN;
        const float a = sw[q] * wq[2 * W2 + kz] * wq[W2 + ky];
        float fx[M];
        load_row<M>(wq + kx0, fx);
#pragma unroll
        for (int j = 0; j < M; ++j) acc[j] = fmaf(a, fx[j], acc[j]);
      }
      const int bx = (key & 1023) - tx0, by = ((key >> 10) & 1023) - ty0, bz = (key >> 20) - tz0;
      float* dst = blk + ((bz + kz) * E + by + ky) * E + bx + kx0;
#pragma unroll
      for (int j = 0; j < M; ++j) dst[j] += acc[j];
      __syncthreads();
      p = q;
    }
  }
  __syncthreads();
  float* out = part + (size_t)u * E3;
  for (int i = threadIdx.x; i < E3; i += NT) out[i] = blk[i];
}

// Grid node g (per dimension) is covered by the block of tile t at local index
// l = g - t*T + m - 1 (mod n), when l lies in [0, E).  General form (aliases
// when E > n) and the direct form for n >= 2E.
__device__ __forceinline__ int covers(int g, int n, int tiles1, int m, int E, int* tl, int* ll) {
  int k = 0;
  if (n >= 2 * E) {
    const int top = (g + m - 1) >= 0 ? (g + m - 1) / NFFT_TILE : -1;
    for (int t = top; k < 8; --t) {
      const int l = g + m - 1 - t * NFFT_TILE;
      if (l >= E) break;
      tl[k] = ((t % tiles1) + tiles1) % tiles1;
      ll[k] = l;
      ++k;
    }
    return k;
  }
  for (int t = 0; t < tiles1 && k < 8; ++t) {
    int l = g - t * NFFT_TILE + m - 1;
    l %= n;
    if (l < 0) l += n;
    for (; l < E && k < 8; l += n) { tl[k] = t; ll[k] = l; ++k; }
  }
  return k;
}

__global__ void k_fold(const float* __restrict__ part, const int* __restrict__ tile_unit_start,
                       int n, int tiles1, int m, int E, float* __restrict__ grid) {
  const long long total = (long long)n * n * n;
  const long long E2 = (long long)E * E, E3 = E2 * E;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int gx = (int)(i % n), gy = (int)((i / n) % n), gz = (int)(i / ((long long)n * n));
    int txl[8], lxl[8], tyl[8], lyl[8], tzl[8], lzl[8];
    const int nx = covers(gx, n, tiles1, m, E, txl, lxl);
    const int ny = covers(gy, n, tiles1, m, E, tyl, lyl);
    const int nz = covers(gz, n, tiles1, m, E, tzl, lzl);
    float acc = 0.f;
    for (int a = 0; a < nz; ++a)
      for (int b = 0; b < ny; ++b)
        for (int c = 0; c < nx; ++c) {
          const int tile = (tzl[a] * tiles1 + tyl[b]) * tiles1 + txl[c];
          const long long loc = ((long long)lzl[a] * E + lyl[b]) * E + lxl[c];
          for (int u = tile_unit_start[tile]; u < tile_unit_start[tile + 1]; ++u)
            acc += part[(long long)u * E3 + loc];
        }
    grid[i] = acc;
  }
}

// Fold for grids of at least 3 tiles per dimension: one CTA per output tile
// (T^3 threads, one node each).  The blocks that can cover the tile are those
// of the 27 neighbouring tiles (E - m + 1 <= 2T and T + m - 1 < 2T for T = 8,
// m <= 8); each node adds the covering block values unit by unit, neighbours
// in a fixed order.
__global__ void __launch_bounds__(NFFT_TILE * NFFT_TILE * NFFT_TILE)
    k_fold_tiles(const float* __restrict__ part, const int* __restrict__ tile_unit_start, int n,
                 int tiles1, int m, int E, float* __restrict__ grid) {
  const int t = blockIdx.x;
  const int tx = t % tiles1, ty = (t / tiles1) % tiles1, tz = t / (tiles1 * tiles1);
  const int lx = threadIdx.x % NFFT_TILE, ly = (threadIdx.x / NFFT_TILE) % NFFT_TILE,
            lz = threadIdx.x / (NFFT_TILE * NFFT_TILE);
  const long long E3 = (long long)E * E * E;
  float acc = 0.f;
  for (int dz = -1; dz <= 1; ++dz) {
    const int bz = lz - dz * NFFT_TILE + m - 1;
    if (bz < 0 || bz >= E) continue;
    const int nz = (tz + dz + tiles1) % tiles1;
    for (int dy = -1; dy <= 1; ++dy) {
      const int by = ly - dy * NFFT_TILE + m - 1;
      if (by < 0 || by >= E) continue;
      const int ny = (ty + dy + tiles1) % tiles1;
      for (int dx = -1; dx <= 1; ++dx) {
        const int bx = lx - dx * NFFT_TILE + m - 1;
        if (bx < 0 || bx >= E) continue;
        const int nx = (tx + dx + tiles1) % tiles1;
        const int nt = (nz * tiles1 + ny) * tiles1 + nx;
        const long long loc = ((long long)bz * E + by) * E + bx;
        for (int u = tile_unit_start[nt]; u < tile_unit_start[nt + 1]; ++u)
          acc += part[(long long)u * E3 + loc];
      }
    }
  }
  const int gx = tx * NFFT_TILE + lx, gy = ty * NFFT_TILE + ly, gz = tz * NFFT_TILE + lz;
  grid[((long long)gz * n + gy) * n + gx] = acc;
}

// ------------------------------------------------------------------ FFT ----
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// In-place radix-2 DIT on FFT_LINES lines of length n held in bit-reversed
// order in `buf` ([line][n]); tw[j] = exp(-2 pi i j / n), j < n/2; dir = +1
// uses the conjugate twiddles (inverse, unnormalised).
__device__ void fft_lines_smem(float2* buf, const float2* tw, int n, int logn, int dir) {
  const int half_total = FFT_LINES * (n >> 1);
  for (int s = 1; s <= logn; ++s) {
    const int half = 1 << (s - 1);
    const int tstep = n >> s;
    for (int b = threadIdx.x; b < half_total; b += blockDim.x) {
      const int line = b / (n >> 1);
      const int j = b - line * (n >> 1);
      const int grp = j >> (s - 1);
      const int pos = j & (half - 1);
      const int i0 = line * n + grp * 2 * half + pos;
      const int i1 = i0 + half;
      float2 w = tw[pos * tstep];
      if (dir > 0) w.y = -w.y;
      const float2 t = cmul(w, buf[i1]);
      const float2 a = buf[i0];
      buf[i0] = make_float2(a.x + t.x, a.y + t.y);
      buf[i1] = make_float2(a.x - t.x, a.y - t.y);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void load_twiddles(float2* tw, int n) {
  for (int j = threadIdx.x; j < n / 2; j += blockDim.x) {
    float sn, cs;
    sincospif(-2.0f * (float)j / (float)n, &sn, &cs);
    tw[j] = make_float2(cs, sn);
  }
}

// Line geometry: axis 0 = x (lines are rows), 1 = y, 2 = z.  Line L, element e.
__device__ __forceinline__ long long line_addr(int axis, int n, long long L, int e) {
  const long long n2 = (long long)n * n;
  if (axis == 0) return L * n + e;
  if (axis == 1) return (L / n) * n2 + (long long)e * n + (L % n);
  return (long long)e * n2 + L;
}

// One FFT pass along `axis`.  mode 0: real in -> complex out (forward);
// mode 1: complex -> complex; mode 2: complex in -> real part out (inverse);
// mode 3: z pass: forward, multiply by scale_k on I_N^3, inverse.
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_pass(const float* __restrict__ rin, const float2* __restrict__ cin,
               float* __restrict__ rout, float2* __restrict__ cout, int n, int logn, int axis,
               int mode, int dir, const float* __restrict__ scale, int N) {
  extern __shared__ float2 sh[];
  float2* tw = sh;
  float2* buf = sh + n / 2;
  load_twiddles(tw, n);
  const long long L0 = (long long)blockIdx.x * FFT_LINES;
  for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
    // consecutive threads take consecutive lines for y/z passes (coalesced),
    // consecutive elements for x passes
    int line, e;
    if (axis == 0) { line = i / n; e = i - line * n; }
    else { e = i / FFT_LINES; line = i - e * FFT_LINES; }
    const long long a = line_addr(axis, n, L0 + line, e);
    const float2 v = mode == 0 ? make_float2(rin[a], 0.f) : cin[a];
    buf[line * n + (__brev(e) >> (32 - logn))] = v;
  }
  __syncthreads();
  fft_lines_smem(buf, tw, n, logn, mode == 3 ? -1 : dir);
  if (mode == 3) {
    // multiply by scale_k: line L = y*n + x carries (kx, ky); element = kz
    for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
      const int line = i / n, e = i - line * n;
      const long long L = L0 + line;
      const int x = (int)(L % n), y = (int)(L / n);
      const int kx = x < n / 2 ? x : x - n, ky = y < n / 2 ? y : y - n, kz = e < n / 2 ? e : e - n;
      float f = 0.f;
      if (kx >= -N / 2 && kx < N / 2 && ky >= -N / 2 && ky < N / 2 && kz >= -N / 2 && kz < N / 2)
        f = scale[kx + N / 2] * scale[N + ky + N / 2] * scale[2 * N + kz + N / 2];
      const float2 v = buf[i];
      buf[i] = make_float2(v.x * f, v.y * f);
    }
    __syncthreads();
    // bit-reverse in place for the inverse transform
    for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
      const int line = i / n, e = i - line * n;
      const int r = __brev(e) >> (32 - logn);
      if (r > e) {
        const float2 t = buf[line * n + e];
        buf[line * n + e] = buf[line * n + r];
        buf[line * n + r] = t;
      }
    }
    __syncthreads();
    fft_lines_smem(buf, tw, n, logn, +1);
  }
  for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
    int line, e;
    if (axis == 0) { line = i / n; e = i - line * n; }
    else { e = i / FFT_LINES; line = i - e * FFT_LINES; }
    const long long a = line_addr(axis, n, L0 + line, e);
    const float2 v = buf[line * n + e];
    if (mode == 2) rout[a] = v.x;
    else cout[a] = v;
  }
}

// ---------------------------------------------------------------- gather ----
// One CTA per work unit: the E^3 block of the grid around the tile is staged
// in shared memory, then each warp evaluates one target at a time.
template <int M>
__global__ void __launch_bounds__(256)
    k_gather(const int4* __restrict__ cell, const float* __restrict__ win,
             const int* __restrict__ unit_tile, const int* __restrict__ unit_begin,
             const int* __restrict__ unit_count, const int* __restrict__ num_units, int n,
             int tiles1, const float* __restrict__ grid, float* __restrict__ out) {
  constexpr int W2 = 2 * M, E = NFFT_TILE + 2 * M - 1, E2 = E * E, E3 = E2 * E, WIN = 3 * W2;
  constexpr int NIT = (W2 * W2 + 31) / 32;
  // Footprint values of the current cell kept in registers while a warp's
  // consecutive targets share that cell (targets are sorted by cell).
  constexpr bool CACHE = NIT * W2 <= 64;
  extern __shared__ float smem[];
  float* blk = smem;
  float* swin = blk + E3 + (E3 & 1);
  int* skey = reinterpret_cast<int*>(swin + CH * WIN);
  const int u = blockIdx.x;
  if (u >= *num_units) return;
  const int tile = unit_tile[u];
  const int tx0 = (tile % tiles1) * NFFT_TILE;
  const int ty0 = ((tile / tiles1) % tiles1) * NFFT_TILE;
  const int tz0 = (tile / (tiles1 * tiles1)) * NFFT_TILE;
  for (int i = threadIdx.x; i < E3; i += blockDim.x) {
    const int lz = i / E2, ly = (i / E) % E, lx = i % E;
    int gz = (tz0 - M + 1 + lz) % n, gy = (ty0 - M + 1 + ly) % n, gx = (tx0 - M + 1 + lx) % n;
    gz += gz < 0 ? n : 0;
    gy += gy < 0 ? n : 0;
    gx += gx < 0 ? n : 0;
    blk[i] = grid[((long long)gz * n + gy) * n + gx];
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int off[NIT], kxs[NIT], kys[NIT];
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int c = lane + 32 * it;
    kxs[it] = c % W2;
    kys[it] = c / W2;
    off[it] = c < W2 * W2 ? kys[it] * E + kxs[it] : -1;
  }
  float hc[CACHE ? NIT * W2 : 1];
  int cached = -1;
  const int b0 = unit_begin[u], cnt = unit_count[u];
  for (int c0 = 0; c0 < cnt; c0 += CH) {
    const int cn = min(CH, cnt - c0);
    __syncthreads();
    const float* gw = win + (size_t)(b0 + c0) * WIN;
    for (int i = threadIdx.x; i < cn * WIN; i += blockDim.x) swin[i] = gw[i];
    for (int i = threadIdx.x; i < cn; i += blockDim.x) skey[i] = cell[b0 + c0 + i].x;
    __syncthreads();
    for (int p = warp; p < cn; p += nwarps) {
      const int key = skey[p];
      const int bx = (key & 1023) - tx0, by = ((key >> 10) & 1023) - ty0, bz = (key >> 20) - tz0;
      const float* wq = swin + p * WIN;
      const float* src = blk + (bz * E + by) * E + bx;
      float fz[W2];
#pragma unroll
      for (int k = 0; k < W2; ++k) fz[k] = wq[2 * W2 + k];
      float acc = 0.f;
      if (CACHE) {
        if (key != cached) {
#pragma unroll
          for (int it = 0; it < NIT; ++it)
#pragma unroll
            for (int k = 0; k < W2; ++k)
              hc[CACHE ? it * W2 + k : 0] = off[it] >= 0 ? src[k * E2 + off[it]] : 0.f;
          cached = key;
        }
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
          float s = 0.f;
#pragma unroll
          for (int k = 0; k < W2; ++k) s = fmaf(fz[k], hc[CACHE ? it * W2 + k : 0], s);
          const float pxy = off[it] >= 0 ? wq[kxs[it]] * wq[W2 + kys[it]] : 0.f;
          acc = fmaf(pxy, s, acc);
        }
      } else {
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
          if (off[it] >= 0) {
            const float pxy = wq[kxs[it]] * wq[W2 + kys[it]];
            const float* col = src + off[it];
            float s = 0.f;
#pragma unroll
            for (int k = 0; k < W2; ++k) s = fmaf(fz[k], col[k * E2], s);
            acc = fmaf(pxy, s, acc);
          }
        }
      }
      acc = warp_sum(acc);
      if (lane == 0) out[b0 + c0 + p] = acc;
    }
  }
}

template <int M>
size_t spread_smem() {
  constexpr int E = NFFT_TILE + 2 * M - 1, E3 = E * E * E;
  return sizeof(float) * (E3 + 1 + CH * 6 * M + 2 * CH);
}

template <int M>
uotk_status launch_spread(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                          const NfftPoints& S, const SpreadWeights& w, float* part) {
  const size_t smem = spread_smem<M>();
  UOTK_CUDA(ctx, cudaFuncSetAttribute(k_spread<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  k_spread<M><<<S.max_units, 8 * M * M, smem, s>>>(S.cell, S.win, S.unit_tile, S.unit_begin,
                                                   S.unit_count, S.num_units, P.tiles1, w.base,
                                                   w.pot, w.lam, w.shift_slot, part);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

template <int M>
uotk_status launch_gather(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                          const NfftPoints& S, const float* grid, float* out) {
  const size_t smem = spread_smem<M>();
  UOTK_CUDA(ctx, cudaFuncSetAttribute(k_gather<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  k_gather<M><<<S.max_units, 256, smem, s>>>(S.cell, S.win, S.unit_tile, S.unit_begin,
                                             S.unit_count, S.num_units, P.n, P.tiles1, grid, out);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

}  // namespace

#define UOTK_M_SWITCH(m, CALL)                 \
  switch (m) {                                 \
    case 2: return CALL(2);                    \
    case 3: return CALL(3);                    \
    case 4: return CALL(4);                    \
    case 5: return CALL(5);                    \
    case 6: return CALL(6);                    \
    case 7: return CALL(7);                    \
    case 8: return CALL(8);                    \
    default: return set_error(ctx, UOTK_ERR_INVALID, "cut-off %d outside [2, 8]", m); \
  }

static uotk_status spread_units(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                                const NfftPoints& S, const SpreadWeights& w, float* part) {
#define UOTK_SPREAD_CALL(M) launch_spread<M>(ctx, s, P, S, w, part)
  UOTK_M_SWITCH(P.m, UOTK_SPREAD_CALL)
#undef UOTK_SPREAD_CALL
}

static uotk_status gather_units(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                                const NfftPoints& S, const float* grid, float* out) {
#define UOTK_GATHER_CALL(M) launch_gather<M>(ctx, s, P, S, grid, out)
  UOTK_M_SWITCH(P.m, UOTK_GATHER_CALL)
#undef UOTK_GATHER_CALL
}

uotk_status nfft_spread(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& S,
                        const SpreadWeights& w, NfftWork& W, float* grid_out) {
  if (S.n > 0) {
    UOTK_PROF(ctx, s, "spread");
    UOTK_TRY(spread_units(ctx, s, P, S, w, W.part));
  }
  {
    UOTK_PROF(ctx, s, "fold");
    const long long total = (long long)P.n * P.n * P.n;
    if (S.n > 0 && P.tiles1 >= 3) {
      k_fold_tiles<<<P.tiles1 * P.tiles1 * P.tiles1, NFFT_TILE * NFFT_TILE * NFFT_TILE, 0, s>>>(
          W.part, S.tile_unit_start, P.n, P.tiles1, P.m, P.E, grid_out);
      UOTK_LAUNCHED(ctx);
    } else if (S.n > 0) {
      k_fold<<<grid_for(ctx, total, 256, 8), 256, 0, s>>>(W.part, S.tile_unit_start, P.n, P.tiles1,
                                                          P.m, P.E, grid_out);
      UOTK_LAUNCHED(ctx);
    } else {
      UOTK_CUDA(ctx, cudaMemsetAsync(grid_out, 0, sizeof(float) * total, s));
    }
  }
  return UOTK_OK;
}

uotk_status nfft_convolve(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, NfftWork& W,
                          const float* grid_in, float* grid_out) {
  const int n = P.n;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  const int blocks = n * n / FFT_LINES;
  const size_t smem = sizeof(float2) * (n / 2 + FFT_LINES * n);
  UOTK_PROF(ctx, s, "fft");
  // forward x (real -> complex), forward y, z (forward, scale, inverse), inverse y, inverse x
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(grid_in, nullptr, nullptr, W.cgrid, n, logn, 0, 0,
                                               -1, nullptr, P.N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 1, 1,
                                               -1, nullptr, P.N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 2, 3,
                                               -1, W.scale, P.N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 1, 1,
                                               +1, nullptr, P.N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, grid_out, nullptr, n, logn, 0, 2,
                                               +1, nullptr, P.N);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status nfft_gather(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& S,
                        const float* grid, float* out_sorted) {
  if (S.n == 0) return UOTK_OK;
  UOTK_PROF(ctx, s, "gather");
  return gather_units(ctx, s, P, S, grid, out_sorted);
}

size_t nfft_work_bytes(const NfftParams& P, int max_src_units) {
  Carver cv(nullptr);
  NfftWork W;
  nfft_work_carve(cv, P, max_src_units, W);
  return cv.off;
}

void nfft_work_carve(Carver& cv, const NfftParams& P, int max_src_units, NfftWork& W) {
  const size_t n3 = (size_t)P.n * P.n * P.n;
  W.part = cv.take<float>((size_t)(max_src_units > 0 ? max_src_units : 1) * P.E * P.E * P.E);
  W.grid = cv.take<float>(n3);
  W.cgrid = cv.take<float2>(n3);
  W.scale = cv.take<float>(3 * P.N);
}

}  // namespace uotk
