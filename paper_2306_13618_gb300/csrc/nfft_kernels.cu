// NFFT stage kernels (Sec. 4, Eq. 1724): spread (adjoint NFFT step 1), the
// grid convolution (FFT, multiply by b_k and the double deconvolution,
// inverse FFT) and gather (NFFT final step).
//
// Work units.  Points are sorted by grid cell, cells tile by tile (8^3 cells
// per tile).  A unit is (tile, up to NFFT_UNIT_POINTS points); its CTA owns the
// E^3 block of grid nodes the tile's windows reach (E = 8 + 2m - 1).  Chunks
// of NFFT_CHUNK points -- window table rows, packed cells, weights -- are
// staged in shared memory by double-buffered 1-D bulk copies (TMA) completing
// on mbarriers, so the copy of chunk k+1 overlaps the arithmetic of chunk k.
// Spread.  Thread (row (kz, ky), half) owns the m nodes kx in [half m, half m
// + m) of footprint row (kz, ky).  The points of one cell share the footprint:
// their rank-1 window products w phi_z phi_y phi_x accumulate in registers and
// are added to the shared block once per cell, a barrier separating the
// additions of consecutive cells (no shared-memory atomics).  The finished
// block is added into the grid with global reductions, skipping zeros.
// Gather.  The CTA stages the E^3 grid block around its tile; each warp
// evaluates one target at a time: lanes split the (2m)^2 (y, x) pairs of the
// footprint, each lane contracting its z-columns with phi_z; consecutive
// targets of one cell reuse the footprint held in registers.
#include <math.h>

#include "nfft.cuh"

namespace uotk {

namespace {

constexpr int CH = NFFT_CHUNK;
constexpr int STAGES = 2;

template <int M>
struct Geo {
  static constexpr int W2 = 2 * M;
  static constexpr int E = NFFT_TILE + 2 * M - 1;
  static constexpr int E2 = E * E;
  static constexpr int E3 = E2 * E;
  static constexpr int E3P = (E3 + 3) & ~3;           // block floats, 16-byte multiple
  static constexpr int WS = nfft_win_stride(M);      // floats per window-table row
  static constexpr int STAGE_F = CH * WS + 2 * (CH + 4);  // floats per staging buffer
};

// Issue the bulk copies of chunk `k` of a unit into staging buffer `st`:
// the window rows (16-byte aligned by construction), and the packed cells and
// weights from the 16-byte-aligned element at or below the chunk start, whose
// offset `off` (0..3) the consumer adds back.
template <int M>
__device__ __forceinline__ void stage_chunk(float* st, unsigned long long* bar, const float* win,
                                            const int* ckey, const float* wts, int q0, int cn) {
  using G = Geo<M>;
  const int off = q0 & 3;
  const unsigned wbytes = (unsigned)(cn * G::WS * 4);
  const unsigned kbytes = (unsigned)(((cn + off + 3) & ~3) * 4);
  mbar_expect(bar, wbytes + (wts ? 2 * kbytes : kbytes));
  bulk_copy(st, win + (size_t)q0 * G::WS, wbytes, bar);
  bulk_copy(st + CH * G::WS, ckey + (q0 - off), kbytes, bar);
  if (wts) bulk_copy(st + CH * G::WS + CH + 4, wts + (q0 - off), kbytes, bar);
}

// Bounded wait for a staging buffer; on time-out every thread learns it, the
// copies still in flight are waited for (bounded) and the CTA leaves.
__device__ __forceinline__ bool stage_ready(unsigned long long* bars, int k, int nchunks,
                                            long long* flags) {
  const bool ok = mbar_wait(&bars[k % STAGES], (unsigned)(k / STAGES) & 1u);
  if (__syncthreads_or(!ok)) {
    if (threadIdx.x == 0) {
      flag_add(&flags[FLAG_TIMEOUT], 1LL);
      for (int q = k; q < nchunks && q < k + STAGES; ++q)
        mbar_wait(&bars[q % STAGES], (unsigned)(q / STAGES) & 1u);
    }
    return false;
  }
  return true;
}

__device__ __forceinline__ void tile_origin(int tile, int tiles1, int& x, int& y, int& z) {
  x = (tile % tiles1) * NFFT_TILE;
  y = ((tile / tiles1) % tiles1) * NFFT_TILE;
  z = (tile / (tiles1 * tiles1)) * NFFT_TILE;
}

// M floats of a window row from shared memory (8-byte loads when M is even).
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

// ---------------------------------------------------------------- spread ----
template <int M>
__global__ void __launch_bounds__(8 * M * M)
    k_spread(const float* __restrict__ win, const int* __restrict__ ckey,
             const float* __restrict__ wts, const int* __restrict__ unit_tile,
             const int* __restrict__ unit_begin, const int* __restrict__ unit_count,
             const int* __restrict__ num_units, int n, int tiles1, float* __restrict__ grid,
             long long* __restrict__ flags) {
  using G = Geo<M>;
  constexpr int W2 = G::W2, E = G::E, E3 = G::E3, WS = G::WS, NT = 8 * M * M;
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) unsigned long long bars[STAGES];
  float* blk = smem;
  float* stage0 = smem + G::E3P;
  const int u = blockIdx.x;
  if (u >= *num_units) return;
  const int b0 = unit_begin[u], cnt = unit_count[u];
  const int nchunks = (cnt + CH - 1) / CH;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
    for (int k = 0; k < STAGES && k < nchunks; ++k)
      stage_chunk<M>(stage0 + k * G::STAGE_F, &bars[k], win, ckey, wts, b0 + k * CH,
                     min(CH, cnt - k * CH));
  }
  for (int i = threadIdx.x; i < E3; i += NT) blk[i] = 0.f;
  __syncthreads();  // barriers initialised and block zeroed before anyone waits or adds
  int tx0, ty0, tz0;
  tile_origin(unit_tile[u], tiles1, tx0, ty0, tz0);
  const int r = threadIdx.x >> 1, half = threadIdx.x & 1;
  const int kz = r / W2, ky = r - kz * W2, kx0 = half * M;
  for (int k = 0; k < nchunks; ++k) {
    if (!stage_ready(bars, k, nchunks, flags)) return;
    const int q0 = b0 + k * CH, cn = min(CH, cnt - k * CH), off = q0 & 3;
    const float* sw = stage0 + (k % STAGES) * G::STAGE_F;
    const int* skey = reinterpret_cast<const int*>(sw + CH * WS) + off;
    const float* swt = sw + CH * WS + CH + 4 + off;
    int p = 0;
    while (p < cn) {
      const int key = skey[p];
      float acc[M];
#pragma unroll
      for (int j = 0; j < M; ++j) acc[j] = 0.f;
      int q = p;
      for (; q < cn && skey[q] == key; ++q) {
        const float* wq = sw + q * WS;
        const float a = swt[q] * wq[2 * W2 + kz] * wq[W2 + ky];
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
    if (threadIdx.x == 0 && k + STAGES < nchunks)
      stage_chunk<M>(stage0 + (k % STAGES) * G::STAGE_F, &bars[k % STAGES], win, ckey, wts,
                     b0 + (k + STAGES) * CH, min(CH, cnt - (k + STAGES) * CH));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < E3; i += NT) {
    const float v = blk[i];
    if (v == 0.f) continue;
    const int lz = i / G::E2, ly = (i / E) % E, lx = i % E;
    int gz = (tz0 - M + 1 + lz) % n, gy = (ty0 - M + 1 + ly) % n, gx = (tx0 - M + 1 + lx) % n;
    gz += gz < 0 ? n : 0;
    gy += gy < 0 ? n : 0;
    gx += gx < 0 ? n : 0;
    atomicAdd(&grid[((long long)gz * n + gy) * n + gx], v);
  }
}

// Spread weights in sorted order: w_q = base_q exp(lam pot_q - shift).
__global__ void k_point_weights(const float* __restrict__ base, const double* __restrict__ pot,
                                double lam, const long long* __restrict__ shift_slot, long long n,
                                float* __restrict__ out) {
  const double shift = ordered_to_dbl(*shift_slot);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n + 4;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = i < n ? (base ? base[i] : 1.f) * exp_shifted(lam * pot[i] - shift) : 0.f;
}

// ------------------------------------------------------------------ FFT ----
// Radix-2 decimation in time on lines held in shared memory in bit-reversed
// order: line l, element e at buf[l * lstride + e * estride].  tw[j] =
// exp(-2 pi i j/n), j < n/2; dir = +1 takes the conjugate twiddles (inverse,
// unnormalised).  Called by all threads of the CTA; ends with a barrier.
constexpr int FFT_LINES = 16;
constexpr int FFT_THREADS = 256;
constexpr int SLAB_THREADS = 512;
constexpr int SLAB_ROWS = 16;

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ void fft_smem(float2* buf, int lines, int lstride, int estride, const float2* tw, int n,
                         int logn, int dir) {
  const int hn = n >> 1;
  const int total = lines * hn;
  for (int st = 1; st <= logn; ++st) {
    const int half = 1 << (st - 1);
    const int tstep = n >> st;
    for (int b = threadIdx.x; b < total; b += blockDim.x) {
      const int line = b / hn;
      const int j = b - line * hn;
      const int grp = j >> (st - 1);
      const int pos = j & (half - 1);
      const int e0 = grp * 2 * half + pos;
      float2* p0 = buf + line * lstride + e0 * estride;
      float2* p1 = p0 + half * estride;
      float2 w = tw[pos * tstep];
      if (dir > 0) w.y = -w.y;
      const float2 t = cmul(w, *p1);
      const float2 a = *p0;
      *p0 = make_float2(a.x + t.x, a.y + t.y);
      *p1 = make_float2(a.x - t.x, a.y - t.y);
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

__device__ __forceinline__ int bitrev(int e, int logn) { return (int)(__brev((unsigned)e) >> (32 - logn)); }
// FFT index of the k' th kept frequency, k = k' - N/2 in I_N.
__device__ __forceinline__ int kept_index(int kp, int N, int n) {
  const int k = kp - N / 2;
  return k < 0 ? k + n : k;
}

// Forward transform of one z-slab: x then y, both pruned to I_N.
// in: real grid [z][y][x];  out: A[z][ky'][kx'] complex, n x N x N.
__global__ void __launch_bounds__(SLAB_THREADS)
    k_fft_slab_fwd(const float* __restrict__ g, float2* __restrict__ A, int n, int logn, int N) {
  extern __shared__ __align__(16) float2 fsh[];
  float2* tw = fsh;
  float2* col = fsh + n / 2;            // [n (y, bit-reversed)][N (kx')]
  float2* rows = col + (size_t)n * N;   // [SLAB_ROWS][n]
  load_twiddles(tw, n);
  const int z = blockIdx.x;
  const float* gz = g + (size_t)z * n * n;
  for (int r0 = 0; r0 < n; r0 += SLAB_ROWS) {
    for (int i = threadIdx.x; i < SLAB_ROWS * n; i += blockDim.x) {
      const int r = i / n, x = i - r * n;
      rows[r * n + bitrev(x, logn)] = make_float2(gz[(size_t)(r0 + r) * n + x], 0.f);
    }
    __syncthreads();
    fft_smem(rows, SLAB_ROWS, n, 1, tw, n, logn, -1);
    for (int i = threadIdx.x; i < SLAB_ROWS * N; i += blockDim.x) {
      const int r = i / N, kp = i - r * N;
      col[bitrev(r0 + r, logn) * N + kp] = rows[r * n + kept_index(kp, N, n)];
    }
    __syncthreads();
  }
  fft_smem(col, N, 1, N, tw, n, logn, -1);
  float2* Az = A + (size_t)z * N * N;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    const int kyp = i / N, kxp = i - kyp * N;
    Az[i] = col[kept_index(kyp, N, n) * N + kxp];
  }
}

// z lines: forward FFT, keep I_N and multiply by scale_k, inverse FFT.
// In place on A[z][ky'][kx'] (n x N x N); FFT_LINES adjacent kx' per CTA.
__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_zlines(float2* __restrict__ A, int n, int logn, int N, const float* __restrict__ scale) {
  extern __shared__ __align__(16) float2 fsh[];
  float2* tw = fsh;
  float2* a = fsh + n / 2;                // [FFT_LINES][n]
  float2* b = a + FFT_LINES * n;          // [FFT_LINES][n]
  load_twiddles(tw, n);
  const int line0 = blockIdx.x * FFT_LINES;  // line = ky' * N + kx'
  const size_t zs = (size_t)N * N;
  for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
    const int z = i / FFT_LINES, l = i - z * FFT_LINES;
    a[l * n + bitrev(z, logn)] = A[(size_t)z * zs + line0 + l];
  }
  __syncthreads();
  fft_smem(a, FFT_LINES, n, 1, tw, n, logn, -1);
  for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
    const int l = i / n, e = i - l * n;
    const int line = line0 + l;
    const int kyp = line / N, kxp = line - kyp * N;
    const int kz = e < n / 2 ? e : e - n;
    float2 v = make_float2(0.f, 0.f);
    if (kz >= -N / 2 && kz < N / 2) {
      const float f = scale[kxp] * scale[N + kyp] * scale[2 * N + kz + N / 2];
      const float2 u = a[l * n + e];
      v = make_float2(u.x * f, u.y * f);
    }
    b[l * n + bitrev(e, logn)] = v;
  }
  __syncthreads();
  fft_smem(b, FFT_LINES, n, 1, tw, n, logn, +1);
  for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
    const int z = i / FFT_LINES, l = i - z * FFT_LINES;
    A[(size_t)z * zs + line0 + l] = b[l * n + z];
  }
}

// Inverse transform of one z-slab: y then x from the I_N^2 coefficients,
// real part out.  in: A[z][ky'][kx'];  out: real grid [z][y][x].
__global__ void __launch_bounds__(SLAB_THREADS)
    k_fft_slab_inv(const float2* __restrict__ A, float* __restrict__ g, int n, int logn, int N) {
  extern __shared__ __align__(16) float2 fsh[];
  float2* tw = fsh;
  float2* col = fsh + n / 2;
  float2* rows = col + (size_t)n * N;
  load_twiddles(tw, n);
  const int z = blockIdx.x;
  const float2* Az = A + (size_t)z * N * N;
  for (int i = threadIdx.x; i < n * N; i += blockDim.x) col[i] = make_float2(0.f, 0.f);
  __syncthreads();
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) {
    const int kyp = i / N, kxp = i - kyp * N;
    col[bitrev(kept_index(kyp, N, n), logn) * N + kxp] = Az[i];
  }
  __syncthreads();
  fft_smem(col, N, 1, N, tw, n, logn, +1);
  float* gz = g + (size_t)z * n * n;
  for (int r0 = 0; r0 < n; r0 += SLAB_ROWS) {
    for (int i = threadIdx.x; i < SLAB_ROWS * n; i += blockDim.x) rows[i] = make_float2(0.f, 0.f);
    __syncthreads();
    for (int i = threadIdx.x; i < SLAB_ROWS * N; i += blockDim.x) {
      const int r = i / N, kp = i - r * N;
      rows[r * n + bitrev(kept_index(kp, N, n), logn)] = col[(r0 + r) * N + kp];
    }
    __syncthreads();
    fft_smem(rows, SLAB_ROWS, n, 1, tw, n, logn, +1);
    for (int i = threadIdx.x; i < SLAB_ROWS * n; i += blockDim.x) {
      const int r = i / n, x = i - r * n;
      gz[(size_t)(r0 + r) * n + x] = rows[i].x;
    }
    __syncthreads();
  }
}

// Unpruned passes for large grids (n > 128): one FFT pass along `axis` on
// FFT_LINES lines adjacent in memory.  mode 0: real in -> complex out;
// mode 1: complex -> complex; mode 2: complex in -> real part out; mode 3:
// z pass: forward, multiply by scale_k on I_N^3, inverse.
__device__ __forceinline__ long long line_addr(int axis, int n, long long L, int e) {
  const long long n2 = (long long)n * n;
  if (axis == 0) return L * n + e;
  if (axis == 1) return (L / n) * n2 + (long long)e * n + (L % n);
  return (long long)e * n2 + L;
}

__global__ void __launch_bounds__(FFT_THREADS)
    k_fft_pass(const float* __restrict__ rin, const float2* __restrict__ cin,
               float* __restrict__ rout, float2* __restrict__ cout, int n, int logn, int axis,
               int mode, int dir, const float* __restrict__ scale, int N) {
  extern __shared__ __align__(16) float2 fsh[];
  float2* tw = fsh;
  float2* buf = fsh + n / 2;
  load_twiddles(tw, n);
  const long long L0 = (long long)blockIdx.x * FFT_LINES;
  for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
    int line, e;
    if (axis == 0) { line = i / n; e = i - line * n; }
    else { e = i / FFT_LINES; line = i - e * FFT_LINES; }
    const long long ad = line_addr(axis, n, L0 + line, e);
    const float2 v = mode == 0 ? make_float2(rin[ad], 0.f) : cin[ad];
    buf[line * n + bitrev(e, logn)] = v;
  }
  __syncthreads();
  fft_smem(buf, FFT_LINES, n, 1, tw, n, logn, mode == 3 ? -1 : dir);
  if (mode == 3) {
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
    for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
      const int line = i / n, e = i - line * n;
      const int r = bitrev(e, logn);
      if (r > e) {
        const float2 t = buf[line * n + e];
        buf[line * n + e] = buf[line * n + r];
        buf[line * n + r] = t;
      }
    }
    __syncthreads();
    fft_smem(buf, FFT_LINES, n, 1, tw, n, logn, +1);
  }
  for (int i = threadIdx.x; i < FFT_LINES * n; i += blockDim.x) {
    int line, e;
    if (axis == 0) { line = i / n; e = i - line * n; }
    else { e = i / FFT_LINES; line = i - e * FFT_LINES; }
    const long long ad = line_addr(axis, n, L0 + line, e);
    const float2 v = buf[line * n + e];
    if (mode == 2) rout[ad] = v.x;
    else cout[ad] = v;
  }
}

// ---------------------------------------------------------------- gather ----
template <int M>
__global__ void __launch_bounds__(256)
    k_gather(const float* __restrict__ win, const int* __restrict__ ckey,
             const int* __restrict__ unit_tile, const int* __restrict__ unit_begin,
             const int* __restrict__ unit_count, const int* __restrict__ num_units, int n,
             int tiles1, const float* __restrict__ grid, float* __restrict__ out,
             long long* __restrict__ flags) {
  using G = Geo<M>;
  constexpr int W2 = G::W2, E = G::E, E2 = G::E2, E3 = G::E3, WS = G::WS;
  constexpr int NIT = (W2 * W2 + 31) / 32;
  // Footprint of the current cell kept in registers while a warp's consecutive
  // targets share that cell.
  constexpr bool CACHE = NIT * W2 <= 64;
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) unsigned long long bars[STAGES];
  float* blk = smem;
  float* stage0 = smem + G::E3P;
  const int u = blockIdx.x;
  if (u >= *num_units) return;
  const int b0 = unit_begin[u], cnt = unit_count[u];
  const int nchunks = (cnt + CH - 1) / CH;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    mbar_fence_init();
    for (int k = 0; k < STAGES && k < nchunks; ++k)
      stage_chunk<M>(stage0 + k * G::STAGE_F, &bars[k], win, ckey, nullptr, b0 + k * CH,
                     min(CH, cnt - k * CH));
  }
  int tx0, ty0, tz0;
  tile_origin(unit_tile[u], tiles1, tx0, ty0, tz0);
  for (int i = threadIdx.x; i < E3; i += blockDim.x) {
    const int lz = i / E2, ly = (i / E) % E, lx = i % E;
    int gz = (tz0 - M + 1 + lz) % n, gy = (ty0 - M + 1 + ly) % n, gx = (tx0 - M + 1 + lx) % n;
    gz += gz < 0 ? n : 0;
    gy += gy < 0 ? n : 0;
    gx += gx < 0 ? n : 0;
    blk[i] = grid[((long long)gz * n + gy) * n + gx];
  }
  __syncthreads();  // barriers initialised and block staged before anyone waits or reads
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
  for (int k = 0; k < nchunks; ++k) {
    if (!stage_ready(bars, k, nchunks, flags)) return;
    const int q0 = b0 + k * CH, cn = min(CH, cnt - k * CH), koff = q0 & 3;
    const float* sw = stage0 + (k % STAGES) * G::STAGE_F;
    const int* skey = reinterpret_cast<const int*>(sw + CH * WS) + koff;
    for (int p = warp; p < cn; p += nwarps) {
      const int key = skey[p];
      const int bx = (key & 1023) - tx0, by = ((key >> 10) & 1023) - ty0, bz = (key >> 20) - tz0;
      const float* wq = sw + p * WS;
      const float* src = blk + (bz * E + by) * E + bx;
      float fz[W2];
#pragma unroll
      for (int kk = 0; kk < W2; ++kk) fz[kk] = wq[2 * W2 + kk];
      float acc = 0.f;
      if (CACHE) {
        if (key != cached) {
#pragma unroll
          for (int it = 0; it < NIT; ++it)
#pragma unroll
            for (int kk = 0; kk < W2; ++kk)
              hc[CACHE ? it * W2 + kk : 0] = off[it] >= 0 ? src[kk * E2 + off[it]] : 0.f;
          cached = key;
        }
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
          float s = 0.f;
#pragma unroll
          for (int kk = 0; kk < W2; ++kk) s = fmaf(fz[kk], hc[CACHE ? it * W2 + kk : 0], s);
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
            for (int kk = 0; kk < W2; ++kk) s = fmaf(fz[kk], col[kk * E2], s);
            acc = fmaf(pxy, s, acc);
          }
        }
      }
      acc = warp_sum(acc);
      if (lane == 0) out[q0 + p] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0 && k + STAGES < nchunks)
      stage_chunk<M>(stage0 + (k % STAGES) * G::STAGE_F, &bars[k % STAGES], win, ckey, nullptr,
                     b0 + (k + STAGES) * CH, min(CH, cnt - (k + STAGES) * CH));
  }
}

template <int M>
size_t unit_smem() {
  using G = Geo<M>;
  return sizeof(float) * (G::E3P + STAGES * G::STAGE_F);
}

template <int M>
uotk_status launch_spread(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                          const NfftPoints& S, const float* wts, float* grid) {
  const size_t smem = unit_smem<M>();
  UOTK_CUDA(ctx, cudaFuncSetAttribute(k_spread<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  k_spread<M><<<S.max_units, 8 * M * M, smem, s>>>(S.win, S.ckey, wts, S.unit_tile, S.unit_begin,
                                                   S.unit_count, S.num_units, P.n, P.tiles1, grid,
                                                   ctx->dflags);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

template <int M>
uotk_status launch_gather(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                          const NfftPoints& S, const float* grid, float* out) {
  const size_t smem = unit_smem<M>();
  UOTK_CUDA(ctx, cudaFuncSetAttribute(k_gather<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
  k_gather<M><<<S.max_units, 256, smem, s>>>(S.win, S.ckey, S.unit_tile, S.unit_begin,
                                             S.unit_count, S.num_units, P.n, P.tiles1, grid, out,
                                             ctx->dflags);
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
                                const NfftPoints& S, const float* wts, float* grid) {
#define UOTK_SPREAD_CALL(M) launch_spread<M>(ctx, s, P, S, wts, grid)
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
  const long long total = (long long)P.n * P.n * P.n;
  UOTK_CUDA(ctx, cudaMemsetAsync(grid_out, 0, sizeof(float) * total, s));
  if (S.n == 0) return UOTK_OK;
  const float* wts = w.base;
  if (w.pot) {
    UOTK_PROF(ctx, s, "weights");
    k_point_weights<<<grid_for(ctx, S.n + 4, 256, 4), 256, 0, s>>>(w.base, w.pot, w.lam,
                                                                   w.shift_slot, S.n, W.wts);
    UOTK_LAUNCHED(ctx);
    wts = W.wts;
  }
  UOTK_PROF(ctx, s, "spread");
  return spread_units(ctx, s, P, S, wts, grid_out);
}

uotk_status nfft_convolve(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, NfftWork& W,
                          const float* grid_in, float* grid_out) {
  const int n = P.n, N = P.N;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  UOTK_PROF(ctx, s, "fft");
  const size_t slab_smem = sizeof(float2) * (n / 2 + (size_t)n * N + SLAB_ROWS * n);
  if (n <= 128 && (N * N) % FFT_LINES == 0 && slab_smem <= (size_t)ctx->max_smem_optin) {
    // pruned: forward x+y per slab, z lines with the scale, inverse y+x per slab
    UOTK_CUDA(ctx, cudaFuncSetAttribute(k_fft_slab_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)slab_smem));
    UOTK_CUDA(ctx, cudaFuncSetAttribute(k_fft_slab_inv, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                        (int)slab_smem));
    k_fft_slab_fwd<<<n, SLAB_THREADS, slab_smem, s>>>(grid_in, W.cgrid, n, logn, N);
    UOTK_LAUNCHED(ctx);
    const size_t zsmem = sizeof(float2) * (n / 2 + 2 * FFT_LINES * n);
    k_fft_zlines<<<N * N / FFT_LINES, FFT_THREADS, zsmem, s>>>(W.cgrid, n, logn, N, W.scale);
    UOTK_LAUNCHED(ctx);
    k_fft_slab_inv<<<n, SLAB_THREADS, slab_smem, s>>>(W.cgrid, grid_out, n, logn, N);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  }
  const int blocks = n * n / FFT_LINES;
  const size_t smem = sizeof(float2) * (n / 2 + FFT_LINES * n);
  // forward x (real -> complex), forward y, z (forward, scale, inverse), inverse y, inverse x
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(grid_in, nullptr, nullptr, W.cgrid, n, logn, 0, 0,
                                               -1, nullptr, N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 1, 1,
                                               -1, nullptr, N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 2, 3,
                                               -1, W.scale, N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 1, 1,
                                               +1, nullptr, N);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, grid_out, nullptr, n, logn, 0, 2,
                                               +1, nullptr, N);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status nfft_gather(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& S,
                        const float* grid, float* out_sorted) {
  if (S.n == 0) return UOTK_OK;
  UOTK_PROF(ctx, s, "gather");
  return gather_units(ctx, s, P, S, grid, out_sorted);
}

size_t nfft_work_bytes(const NfftParams& P, int64_t max_points) {
  Carver cv(nullptr);
  NfftWork W;
  nfft_work_carve(cv, P, max_points, W);
  return cv.off;
}

void nfft_work_carve(Carver& cv, const NfftParams& P, int64_t max_points, NfftWork& W) {
  const size_t n3 = (size_t)P.n * P.n * P.n;
  W.wts = cv.take<float>((size_t)(max_points > 0 ? max_points : 1) + 4);
  W.grid = cv.take<float>(n3);
  W.cgrid = cv.take<float2>(n3);
  W.scale = cv.take<float>(3 * P.N);
}

}  // namespace uotk
