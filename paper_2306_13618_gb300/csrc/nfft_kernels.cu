// NFFT stage kernels (Sec. 4, Eq. 1724): spread (adjoint NFFT step 1), the
// grid convolution (FFT, multiply by b_k and the double deconvolution,
// inverse FFT) and gather (NFFT final step).
//
// Work units.  Points are sorted by grid cell, cells tile by tile (8^3 cells
// per tile), and inside a cell in caller order (a stable sort), so every sum
// below is taken in the same order on every run.  The sorted points are cut
// into chunks of equal cost (points, plus a fixed cost per occupied cell and
// tile), one per CTA the device holds at once, and a chunk into units where a
// tile ends; a CTA takes its chunk's units in turn, and for each owns the E^3
// block of grid nodes the unit's tile reaches with its windows
// (E = 8 + 2m - 1).  Window rows, cells and
// weights arrive in shared memory by double-buffered 1-D bulk copies (TMA)
// completing on mbarriers, so the copy of the next chunk overlaps the
// arithmetic of the current one.
// Spread.  The threads partition the footprint of one cell; the points of a
// cell run accumulate their rank-1 window products w phi_z phi_y phi_x in
// registers (packed FP32x2 over point pairs, from the pair window table) and
// are added to the shared block once per run, a barrier separating the
// additions of consecutive runs.  In a Sinkhorn half-step the spread forms the
// weights itself.  Each unit writes its block to a workspace; the fold sums the
// blocks of every grid node in a fixed order (no atomics anywhere).
// Gather.  The CTA stages the E^3 grid block around its tile.  For even m <= 6
// each warp stages and evaluates its own run of targets (k_gather_w); lanes
// split the footprint, which stays in registers while consecutive targets share
// a cell.  Odd m and m = 8 use the CTA-staged form (k_gather).  In a Sinkhorn
// half-step the gather also runs the dual update of its targets.
#include <math.h>

#include "nfft.cuh"

namespace uotk {

namespace {

constexpr int CH = NFFT_CHUNK;
constexpr int STAGES = 2;

template <int M, int C = CH>
struct Geo {
  static constexpr int W2 = 2 * M;
  static constexpr int E = NFFT_TILE + 2 * M - 1;
  static constexpr int E2 = E * E;
  static constexpr int E3 = E2 * E;
  static constexpr int E3P = (E3 + 3) & ~3;           // block floats, 16-byte multiple
  static constexpr int WS = nfft_win_stride(M);      // floats per window-table row
  static constexpr int STAGE_F = C * WS + 2 * (C + 4);  // floats per staging buffer (C points)
};

// Issue the bulk copies of chunk `k` of a unit into staging buffer `st`:
// the window rows (16-byte aligned by construction), and the packed cells and
// weights from the 16-byte-aligned element at or below the chunk start, whose
// offset `off` (0..3) the consumer adds back.
template <int M, int C = CH>
__device__ __forceinline__ void stage_chunk(float* st, unsigned long long* bar, const float* win,
                                            const int* ckey, const float* wts, int q0, int cn) {
  using G = Geo<M, C>;
  const int off = q0 & 3;
  const unsigned wbytes = (unsigned)(cn * G::WS * 4);
  const unsigned kbytes = (unsigned)(((cn + off + 3) & ~3) * 4);
  mbar_expect(bar, wbytes + (wts ? 2 * kbytes : kbytes));
  bulk_copy(st, win + (size_t)q0 * G::WS, wbytes, bar);
  bulk_copy(st + C * G::WS, ckey + (q0 - off), kbytes, bar);
  if (wts) bulk_copy(st + C * G::WS + C + 4, wts + (q0 - off), kbytes, bar);
}

// Bounded wait for a staging buffer; on time-out every thread learns it, the
// copies still in flight are waited for (bounded) and the CTA leaves.
// The first wait (k = 0) goes through first_wait (the context's time-out test
// waits on `never` there); the copies are drained with the normal limit.
__device__ __forceinline__ bool stage_ready(unsigned long long* bars, int k, int nchunks,
                                            long long* flags, unsigned long long* never) {
  const bool ok = k == 0 ? first_wait(&bars[0], 0u, never, flags)
                         : mbar_wait(&bars[k % STAGES], (unsigned)(k / STAGES) & 1u);
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

// Grid node index v mod n for v in [-n, 2n): a tile's block reaches at most
// m - 1 nodes below its tile and m - 2 above it, and n >= 16 > m.
__device__ __forceinline__ int wrap_node(int v, int n) {
  return v < 0 ? v + n : (v >= n ? v - n : v);
}

// NFFT half-steps take the weights and the logarithms of the sums in FP32 from
// the FP64 exponent: w = base e^{lam pot - shift} with the difference in FP64 and
// the exponential in FP32.  A weight e^a then carries a relative error of about
// |a| 2^-24, an absolute error below e^-1 2^-24 of the largest weight, far below
// the window sums' own error of about 1e-5 of the total weight; likewise log t
// in FP32 (about 4e-6 absolute at the extreme |log t| = 88) against the sums'
// relative error.  This leaves one FP64 FMA and one conversion per point, on a
// GPU where an FP64 warp instruction holds the FP64 unit for about 64 cycles.
__device__ __forceinline__ float nfft_weight(float base, double lam, double pot, double shift) {
  return base * expf((float)fma(lam, pot, -shift));
}

__device__ __forceinline__ void tile_origin(int tile, int tiles1, int& x, int& y, int& z) {
  x = (tile % tiles1) * NFFT_TILE;
  y = ((tile / tiles1) % tiles1) * NFFT_TILE;
  z = (tile / (tiles1 * tiles1)) * NFFT_TILE;
}

// K consecutive floats from 16-byte-aligned shared memory: 16-byte loads, then
// an 8-byte and a 4-byte load for the remainder.
template <int K>
__device__ __forceinline__ void load_vec(const float* p, float* r) {
  int j = 0;
#pragma unroll
  for (; j + 4 <= K; j += 4) {
    const float4 v = *reinterpret_cast<const float4*>(p + j);
    r[j] = v.x; r[j + 1] = v.y; r[j + 2] = v.z; r[j + 3] = v.w;
  }
  if (K - j >= 2) {
    const float2 v = *reinterpret_cast<const float2*>(p + j);
    r[j] = v.x; r[j + 1] = v.y;
    j += 2;
  }
  if (K - j == 1) r[j] = p[j];
}

// ---------------------------------------------------------------- spread ----
// Thread (zg, y, xh) of the NT = ZG 2m 2 threads owns the ZB = 2m/ZG nodes
// z in [zg ZB, zg ZB + ZB) of footprint row y, x in [xh m, xh m + m).  The
// spread reads the pair window table: every value is the pair (point 2p, point
// 2p + 1), so one packed FP32x2 FMA adds the contributions of two points of a
// cell to a node, the two halves summing the even and the odd points (added
// when the cell's run ends).  Per point pair a thread forms ZB packed products
// w phi_z phi_y and adds each times its m phi_x pairs.  The threads partition
// the footprint, so the per-cell additions into the shared block need no
// atomics; a barrier separates consecutive cells.
template <int M>
struct SpreadMap {
  static constexpr int W2 = 2 * M;
  static constexpr int ZG = (M % 2 == 0) ? 4 : 2;  // z groups
  static constexpr int ZB = W2 / ZG;               // z rows per thread
  static constexpr int NT = ZG * W2 * 2;           // threads owning footprint nodes
  static constexpr int NTH = NT < 32 ? 32 : NT;    // threads launched (warp 0 lists cell runs)
};
template <int M, int CP>
struct SpreadGeo {
  static constexpr int E = NFFT_TILE + 2 * M - 1;
  static constexpr int E2 = E * E, E3 = E2 * E, E3P = (E3 + 3) & ~3;
  static constexpr int WSP = nfft_winp_stride(M);   // floats per pair row
  static constexpr int CPT = 2 * CP;                 // point positions per chunk
  static constexpr int STAGE_F = CP * WSP + 2 * (CPT + 4);  // pair rows, cells, weights
};
constexpr int SPREAD_CP = 32;   // point pairs per staging chunk

// Copies of chunk k of a unit: pair rows [pc0, pc0 + cpn), and the cells and
// weights of points 2 pc0 .. from the 16-byte-aligned element at or below,
// whose offset (0 or 2) the consumer adds back.
template <int M, int CP>
__device__ __forceinline__ void stage_pairs(float* st, unsigned long long* bar, const float* winp,
                                            const int* ckey, const float* wts, int pc0, int cpn) {
  using SG = SpreadGeo<M, CP>;
  const int q0 = 2 * pc0, off = q0 & 3;
  const unsigned wbytes = (unsigned)(cpn * SG::WSP * 4);
  const unsigned kbytes = (unsigned)(((2 * cpn + off + 3) & ~3) * 4);
  mbar_expect(bar, wbytes + (wts ? 2 * kbytes : kbytes));
  bulk_copy(st, winp + (size_t)pc0 * SG::WSP, wbytes, bar);
  bulk_copy(st + CP * SG::WSP, ckey + (q0 - off), kbytes, bar);
  if (wts) bulk_copy(st + CP * SG::WSP + SG::CPT + 4, wts + (q0 - off), kbytes, bar);
}

// POT: the weights are the half-step's w = base e^{lam pot - shift}, formed here
// when a chunk lands (threads WT0.. hold the pot and base of the chunk's points,
// loaded a chunk ahead; wts unused); else they are staged from wts.  Points of
// a pair that lie outside the unit get weight 0.  The warp that lists the cell
// runs also takes the range of local z and y cells of the unit; the block's
// entries that those cells reach (z-planes and y-rows, whole x-rows) go to
// blocks[u], and the range to unit_box[u] for k_fold_units and k_fold, which
// add the blocks into the grid.
template <int M, bool POT, int CP>
__global__ void __launch_bounds__(SpreadMap<M>::NTH)
    k_spread(const float* __restrict__ winp, const int* __restrict__ ckey,
             const float* __restrict__ wts, const int* __restrict__ unit_tile,
             const int* __restrict__ unit_begin, const int* __restrict__ unit_count,
             int* __restrict__ unit_box, const int* __restrict__ chunk_unit_start, int tiles1,
             float* __restrict__ blocks, long long* __restrict__ flags, SpreadWeights pw) {
  using SG = SpreadGeo<M, CP>;
  using SM = SpreadMap<M>;
  constexpr int W2 = 2 * M, E = SG::E, E2 = SG::E2, E3 = SG::E3, WSP = SG::WSP, CPT = SG::CPT;
  constexpr int NT = SM::NTH, ZB = SM::ZB;
  constexpr int HP2 = nfft_winp_half(M), YO2 = nfft_winp_yoff(M), ZO2 = nfft_winp_zoff(M);
  // threads SM::NT.. (present when the footprint needs fewer than a warp) own
  // no nodes; they take part in the listing, the weights and the copies
  const bool owner = (int)threadIdx.x < SM::NT;
  // POT: threads WT0 .. NT-1 form the weights (warp 0 lists the cell runs
  // meanwhile when the CTA has a warp to spare), WK chunk positions each
  constexpr int WT0 = NT >= CPT + 32 ? 32 : 0;
  constexpr int WTN = NT - WT0;
  constexpr int WK = (CPT + WTN - 1) / WTN;
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) unsigned long long bars[STAGES];
  __shared__ __align__(8) unsigned long long never;  // nothing arrives (time-out test)
  __shared__ int gstart[CPT + 1];
  __shared__ int ngroups;
  float* blk = smem;
  float* stage0 = smem + SG::E3P;
  // the CTA's chunk: units ubeg .. uend - 1, taken in turn; kb counts the
  // staging chunks of the earlier units (the barriers' phases run on)
  const int ubeg = chunk_unit_start[blockIdx.x], uend = chunk_unit_start[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    mbar_init(&never, 1);
    mbar_fence_init();
  }
  // POT: FP64 work by whole warps (FP64 is scarce on this GPU and a partial
  // warp costs the pipe a whole one)
  const int wt = (int)threadIdx.x - WT0;
  const int xh = threadIdx.x & 1;
  const int y = (threadIdx.x >> 1) % W2;
  const int z0 = ((threadIdx.x >> 1) / W2) * ZB;
  const int lane = threadIdx.x & 31;
  __shared__ int box_s;
  const unsigned long long keep_hi = f2_pack(0.f, 1.f), keep_lo = f2_pack(1.f, 0.f);
  double shift = 0.0;
  if (POT) shift = ordered_to_dbl(*pw.shift_slot);
  int kb = 0;
  for (int u = ubeg; u < uend; ++u) {
    const int b0 = unit_begin[u], e0 = b0 + unit_count[u];
    const int pb = b0 >> 1, pe = (e0 + 1) >> 1;
    const int nchunks = (pe - pb + CP - 1) / CP;
    if (threadIdx.x == 0) {
      // the staging buffers were last read by the generic proxy (previous unit)
      if (u != ubeg) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int k = 0; k < STAGES && k < nchunks; ++k)
        stage_pairs<M, CP>(stage0 + ((kb + k) % STAGES) * SG::STAGE_F, &bars[(kb + k) % STAGES],
                           winp, ckey, POT ? nullptr : wts, pb + k * CP, min(CP, pe - pb - k * CP));
    }
    double ppot[WK];
    float pbase[WK];
    auto prefetch = [&](int pc0) {
#pragma unroll
      for (int j = 0; j < WK; ++j) {
        const int q = 2 * pc0 + wt + j * WTN;
        ppot[j] = 0.0;
        pbase[j] = 1.f;
        if (wt >= 0 && wt + j * WTN < CPT && q >= b0 && q < e0) {
          ppot[j] = pw.pot[q];
          if (pw.base) pbase[j] = pw.base[q];
        }
      }
    };
    if (POT) prefetch(pb);
    for (int i = threadIdx.x; i < E3; i += NT) blk[i] = 0.f;
    __syncthreads();  // barriers initialised and block zeroed before anyone waits or adds
    int tx0, ty0, tz0;
    tile_origin(unit_tile[u], tiles1, tx0, ty0, tz0);
    // range of the unit's local z and y cells (kept by the listing warp)
    int bz_lo = NFFT_TILE, bz_hi = -1, by_lo = NFFT_TILE, by_hi = -1;
    for (int k = 0; k < nchunks; ++k) {
      if (!stage_ready(bars, kb + k, kb + nchunks, flags, &never)) return;
      const int pc0 = pb + k * CP, cpn = min(CP, pe - pc0), P0 = 2 * pc0;
      const int lo = max(b0, P0) - P0, hi = min(e0, P0 + 2 * cpn) - P0;  // unit positions
      float* sw = stage0 + ((kb + k) % STAGES) * SG::STAGE_F;
      const int koff = P0 & 3;
      const int* skey = reinterpret_cast<const int*>(sw + CP * WSP) + koff;
      const float* swt = sw + CP * WSP + CPT + 4 + koff;
      // Fold each point's weight into its phi_z lane (0 outside the unit), and
      // list where each cell's run of points starts (points are sorted by cell).
      if (POT) {
        if (wt >= 0) {
#pragma unroll
          for (int j = 0; j < WK; ++j) {
            const int t = wt + j * WTN;
            if (t < 2 * cpn) {
              const float w = (t >= lo && t < hi) ? nfft_weight(pbase[j], pw.lam, ppot[j], shift)
                                                  : 0.f;
              float* zr = sw + (t >> 1) * WSP + ZO2 + (t & 1);
#pragma unroll
              for (int i = 0; i < W2; ++i) zr[2 * i] *= w;
            }
          }
          if (k + 1 < nchunks) prefetch(pc0 + CP);
        }
      } else {
        for (int i = threadIdx.x; i < 2 * cpn * W2; i += NT) {
          const int t = i / W2, z = i - t * W2;
          const float w = (t >= lo && t < hi) ? swt[t] : 0.f;
          sw[(t >> 1) * WSP + ZO2 + 2 * z + (t & 1)] *= w;
        }
      }
      if (threadIdx.x < 32) {
        int base = 0;
        for (int h = 0; h < CPT; h += 32) {
          const int t = h + lane;
          const bool f = t >= lo && t < hi && (t == lo || skey[t] != skey[t - 1]);
          const unsigned bal = __ballot_sync(0xffffffffu, f);
          if (f) {
            gstart[base + __popc(bal & ((1u << lane) - 1u))] = t;
            const int key = skey[t];
            const int cz = (key >> 20) - tz0, cy = ((key >> 10) & 1023) - ty0;
            bz_lo = min(bz_lo, cz);
            bz_hi = max(bz_hi, cz);
            by_lo = min(by_lo, cy);
            by_hi = max(by_hi, cy);
          }
          base += __popc(bal);
        }
        if (lane == 0) { ngroups = base; gstart[base] = hi; }
      }
      __syncthreads();
      const int ng = ngroups;
      for (int g = 0; g < ng; ++g) {
        if (owner) {
          const int t0 = gstart[g], t1 = gstart[g + 1];
          const int key = skey[t0];
          unsigned long long acc2[ZB][M];
#pragma unroll
          for (int r = 0; r < ZB; ++r)
#pragma unroll
            for (int j = 0; j < M; ++j) acc2[r][j] = 0ull;
          const int pp0 = t0 >> 1, pp1 = (t1 - 1) >> 1;
          // one point pair: the masked y factor, the m phi_x pairs and the ZB
          // products w phi_z phi_y, all loaded before any FMA of the pair
          // a pair half outside the run (the neighbouring cell's point) is masked:
          // the run's first pair keeps only its odd point when t0 is odd, its last
          // pair only its even point when t1 is odd
          auto load_pair = [&](int pp, unsigned long long (&fx2)[M], unsigned long long (&A2)[ZB],
                               unsigned long long mask) {
            const float* row = sw + pp * WSP;
            unsigned long long fy2 = *reinterpret_cast<const unsigned long long*>(row + YO2 + 2 * y);
            if (mask) fy2 = f2_mul(fy2, mask);
            const float* xr = row + xh * HP2;
#pragma unroll
            for (int j = 0; j + 1 < M; j += 2) {
              const float4 v = *reinterpret_cast<const float4*>(xr + 2 * j);
              fx2[j] = f2_pack(v.x, v.y);
              fx2[j + 1] = f2_pack(v.z, v.w);
            }
            if (M & 1) fx2[M - 1] = *reinterpret_cast<const unsigned long long*>(xr + 2 * (M - 1));
#pragma unroll
            for (int r = 0; r < ZB; ++r)
              A2[r] = f2_mul(*reinterpret_cast<const unsigned long long*>(row + ZO2 + 2 * (z0 + r)),
                             fy2);
          };
          int pp = pp0, pe1 = pp1;
          // the boundary pairs with a masked half, then the inner pairs unmasked
          if ((t0 & 1) || pp0 == pp1) {
            unsigned long long m0 = (t0 & 1) ? keep_hi : f2_pack(1.f, 1.f);
            if (pp0 == pp1 && (t1 & 1)) m0 = f2_mul(m0, keep_lo);
            unsigned long long fa[M], Aa[ZB];
            load_pair(pp0, fa, Aa, m0);
#pragma unroll
            for (int r = 0; r < ZB; ++r)
#pragma unroll
              for (int j = 0; j < M; ++j) acc2[r][j] = f2_fma(Aa[r], fa[j], acc2[r][j]);
            ++pp;
          }
          if (pp <= pp1 && (t1 & 1)) {
            unsigned long long fa[M], Aa[ZB];
            load_pair(pp1, fa, Aa, keep_lo);
#pragma unroll
            for (int r = 0; r < ZB; ++r)
#pragma unroll
              for (int j = 0; j < M; ++j) acc2[r][j] = f2_fma(Aa[r], fa[j], acc2[r][j]);
            --pe1;
          }
          // two pairs per iteration: the second pair's loads overlap the first's FMAs
          for (; pp + 1 <= pe1; pp += 2) {
            unsigned long long fa[M], fb[M], Aa[ZB], Ab[ZB];
            load_pair(pp, fa, Aa, 0ull);
            load_pair(pp + 1, fb, Ab, 0ull);
#pragma unroll
            for (int r = 0; r < ZB; ++r)
#pragma unroll
              for (int j = 0; j < M; ++j) acc2[r][j] = f2_fma(Ab[r], fb[j], f2_fma(Aa[r], fa[j], acc2[r][j]));
          }
          if (pp <= pe1) {
            unsigned long long fa[M], Aa[ZB];
            load_pair(pp, fa, Aa, 0ull);
#pragma unroll
            for (int r = 0; r < ZB; ++r)
#pragma unroll
              for (int j = 0; j < M; ++j) acc2[r][j] = f2_fma(Aa[r], fa[j], acc2[r][j]);
          }
          const int bx = (key & 1023) - tx0, by = ((key >> 10) & 1023) - ty0, bz = (key >> 20) - tz0;
          float* dst = blk + ((bz + z0) * E + by + y) * E + bx + xh * M;
#pragma unroll
          for (int r = 0; r < ZB; ++r)
#pragma unroll
            for (int j = 0; j < M; ++j) {
              float e, o;
              f2_unpack(acc2[r][j], e, o);
              dst[r * E2 + j] += e + o;
            }
        }
        __syncthreads();
      }
      if (threadIdx.x == 0 && k + STAGES < nchunks)
        stage_pairs<M, CP>(stage0 + ((kb + k) % STAGES) * SG::STAGE_F, &bars[(kb + k) % STAGES],
                           winp, ckey, POT ? nullptr : wts, pc0 + STAGES * CP,
                           min(CP, pe - pc0 - STAGES * CP));
    }
    if (threadIdx.x < 32) {
      bz_lo = warp_min_i(bz_lo);
      bz_hi = warp_max_i(bz_hi);
      by_lo = warp_min_i(by_lo);
      by_hi = warp_max_i(by_hi);
      if (lane == 0) {
        const int box = bz_lo | (bz_hi << 4) | (by_lo << 8) | (by_hi << 12);
        box_s = box;
        unit_box[u] = box;
      }
    }
    __syncthreads();
    // the entries the unit's cells reach: local cells z in [zlo, zhi], y in
    // [ylo, yhi] reach block planes zlo .. zhi + 2m - 1 and rows ylo .. yhi + 2m - 1
    const int box = box_s;
    const int pz0 = box & 15, pz1 = ((box >> 4) & 15) + W2;
    const int py0 = (box >> 8) & 15, ny = ((box >> 12) & 15) + W2 - py0;
    float* outb = blocks + (size_t)u * SG::E3P;
    for (int pz = pz0; pz < pz1; ++pz) {
      const int i0 = (pz * E + py0) * E;
      for (int q = threadIdx.x; q < ny * E; q += NT) outb[i0 + q] = blk[i0 + q];
    }
    kb += nchunks;
    __syncthreads();  // the block is written out before the next unit clears it
  }
}

// Fold, step 1: the units of one tile (a tile that meets several chunks has
// several) are summed into the block of the tile's first unit, in
// a fixed order; a unit contributes the entries it wrote (unit_box).  The U
// units of a tile share the work: CTA k of the tile takes the k-th of U slices
// of the block's entries.  When a slice has fewer entries than the CTA has
// threads, G groups of threads each sum the units g, g + G, g + 2G, .. of
// every entry, and the G partial sums are then added in group order: a dense
// tile costs about one block's reads per CTA and short dependency chains.
// Longer slices (tiles of few units) give each thread four entries at once,
// loaded four units per round.
constexpr int FOLD_THREADS = 256;
constexpr int FOLD_BOX_CACHE = 2048;  // unit boxes of a tile held in shared memory
template <int M>
__global__ void __launch_bounds__(FOLD_THREADS)
    k_fold_units(float* __restrict__ blocks, const int* __restrict__ unit_tile,
                 const int* __restrict__ tile_unit_start, const int* __restrict__ unit_box,
                 const int* __restrict__ num_units) {
  constexpr int W2 = 2 * M, E = NFFT_TILE + 2 * M - 1, E2 = E * E, E3 = E2 * E;
  constexpr int E3P = (E3 + 3) & ~3;
  __shared__ float part[FOLD_THREADS];
  __shared__ int boxes[FOLD_BOX_CACHE];
  const int u = blockIdx.x;
  if (u >= *num_units) return;
  const int t = unit_tile[u];
  const int u0 = tile_unit_start[t], U = tile_unit_start[t + 1] - u0;
  if (U < 2) return;
  const int k = u - u0;
  const int chunk = (E3 + U - 1) / U;
  const int e0 = min(E3, k * chunk), e1 = min(E3, e0 + chunk);
  const int ne = e1 - e0;
  if (ne <= 0) return;
  for (int v = threadIdx.x; v < U && v < FOLD_BOX_CACHE; v += FOLD_THREADS)
    boxes[v] = unit_box[u0 + v];
  __syncthreads();
  float* first = blocks + (size_t)u0 * E3P;
  // block entry e of unit v, or 0 where that unit wrote nothing (outside the
  // z-planes and y-rows of its box)
  auto entry = [&](int v, int e) -> float {
    const int box = v < FOLD_BOX_CACHE ? boxes[v] : unit_box[u0 + v];
    const int pz = e / E2, py = (e / E) % E;
    const bool in = pz >= (box & 15) && pz < ((box >> 4) & 15) + W2 &&
                    py >= ((box >> 8) & 15) && py < ((box >> 12) & 15) + W2;
    return in ? first[(size_t)v * E3P + e] : 0.f;
  };
  // G groups of threads per entry; group g sums the units g, g + G, ..: eight
  // running sums (unit index mod 8 within the group) keep eight loads in
  // flight, added in a fixed order
  int G = FOLD_THREADS / ne;
  G = G < 1 ? 1 : (G < U ? G : U);
  if (G == 1) {
    // long slices (tiles of few units): four entries per thread at once, each
    // summed over the units in order, four units per round: 16 loads in flight
    constexpr int EPT = 4, UPR = 4;
    for (int eb0 = e0 + (int)threadIdx.x; eb0 < e1; eb0 += EPT * FOLD_THREADS) {
      float acc[EPT] = {0.f, 0.f, 0.f, 0.f};
      for (int v0 = 0; v0 < U; v0 += UPR) {
        float tv[UPR][EPT];
#pragma unroll
        for (int j = 0; j < UPR; ++j)
#pragma unroll
          for (int i = 0; i < EPT; ++i) {
            const int eb = eb0 + i * FOLD_THREADS;
            tv[j][i] = (v0 + j < U && eb < e1) ? entry(v0 + j, eb) : 0.f;
          }
#pragma unroll
        for (int j = 0; j < UPR; ++j)
#pragma unroll
          for (int i = 0; i < EPT; ++i) acc[i] += tv[j][i];
      }
#pragma unroll
      for (int i = 0; i < EPT; ++i)
        if (eb0 + i * FOLD_THREADS < e1) first[eb0 + i * FOLD_THREADS] = acc[i];
    }
    return;
  }
  const int ei = threadIdx.x % ne, g = threadIdx.x / ne;
  for (int eb = e0 + ei; eb < e1; eb += e1) {
    float s8[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (g < G) {
      int v = g;
      for (; v + 7 * G < U; v += 8 * G) {
        float tv[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) tv[j] = entry(v + j * G, eb);
#pragma unroll
        for (int j = 0; j < 8; ++j) s8[j] += tv[j];
      }
      for (int j = 0; v < U; v += G, ++j) s8[j] += entry(v, eb);
    }
    const float sum = ((s8[0] + s8[1]) + (s8[2] + s8[3])) + ((s8[4] + s8[5]) + (s8[6] + s8[7]));
    part[threadIdx.x] = sum;
    __syncthreads();  // every group has read its units before the first block is overwritten
    if (threadIdx.x < ne) {
      float r = 0.f;
      for (int q = 0; q < G; ++q) r += part[q * ne + threadIdx.x];
      first[e0 + threadIdx.x] = r;
    }
  }
}

// Fold, step 2: grid node g is the sum of the tile blocks (in each tile's
// first unit) of the up to 27 tiles whose blocks cover it, in a fixed order
// (tile offsets dz, dy, dx = -1, 0, 1): no atomics, and every node is summed
// in the same order on every run.  A tile's block covers nodes 8T - m + 1 ..
// 8T + 8 + m - 2 (mod n) per axis, within one tile of T for m <= 8; on a grid
// of two tiles per axis the offsets -1 and +1 name the same tile, whose block
// then covers some nodes twice, as the torus requires.  A tile of one unit
// holds only the entries of that unit's box.  One CTA per output tile, each
// thread four consecutive x nodes (one 16-byte store).
constexpr int FOLD2_THREADS = NFFT_TILE * NFFT_TILE * NFFT_TILE / 4;
template <int M>
__global__ void __launch_bounds__(FOLD2_THREADS)
    k_fold(const float* __restrict__ blocks, const int* __restrict__ tile_unit_start,
           const int* __restrict__ unit_box, int n, int tiles1, float* __restrict__ grid) {
  constexpr int W2 = 2 * M, E = NFFT_TILE + 2 * M - 1;
  constexpr int E3P = (E * E * E + 3) & ~3;
  static_assert(M - 1 < NFFT_TILE, "a block reaches at most one tile beyond its own");
  __shared__ int first[27], offs[27], zlo[27], zhi[27], ylo[27], yhi[27];
  __shared__ int nlist;
  const int t0 = blockIdx.x;
  const int tx = t0 % tiles1, ty = (t0 / tiles1) % tiles1, tz = t0 / (tiles1 * tiles1);
  if (threadIdx.x < 32) {
    // the non-empty neighbour tiles, listed in offset order
    const int c = threadIdx.x;
    int us = -1, lo = 0, hi = E, ylo_ = 0, yhi_ = E;
    if (c < 27) {
      const int dz = c / 9 - 1, dy = (c / 3) % 3 - 1, dx = c % 3 - 1;
      const int T = (((tz + dz + tiles1) % tiles1) * tiles1 + (ty + dy + tiles1) % tiles1) *
                        tiles1 + (tx + dx + tiles1) % tiles1;
      const int a = tile_unit_start[T], b = tile_unit_start[T + 1];
      if (b > a) {
        us = a;
        if (b - a == 1) {
          const int box = unit_box[a];
          lo = box & 15;
          hi = ((box >> 4) & 15) + W2;
          ylo_ = (box >> 8) & 15;
          yhi_ = ((box >> 12) & 15) + W2;
        }
      }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, us >= 0);
    if (us >= 0) {
      const int slot = __popc(bal & ((1u << c) - 1u));
      first[slot] = us;
      offs[slot] = c;
      zlo[slot] = lo;
      zhi[slot] = hi;
      ylo[slot] = ylo_;
      yhi[slot] = yhi_;
    }
    if (c == 0) nlist = __popc(bal);
  }
  __syncthreads();
  const int lx = (threadIdx.x & 1) * 4, ly = (threadIdx.x >> 1) & 7, lz = threadIdx.x >> 4;
  const int nl = nlist;
  float4* dst = reinterpret_cast<float4*>(
      grid + ((long long)(tz * NFFT_TILE + lz) * n + ty * NFFT_TILE + ly) * n + tx * NFFT_TILE + lx);
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  // in batches of four neighbours: the 16 loads of a batch in flight together,
  // then added in list order
  for (int q0 = 0; q0 < nl; q0 += 4) {
    float t[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int q = q0 + j;
#pragma unroll
      for (int i = 0; i < 4; ++i) t[j][i] = 0.f;
      if (q < nl) {
        const int c = offs[q];
        const int dz = c / 9 - 1, dy = (c / 3) % 3 - 1, dx = c % 3 - 1;
        const int Lz = lz - NFFT_TILE * dz + M - 1, Ly = ly - NFFT_TILE * dy + M - 1,
                  Lx = lx - NFFT_TILE * dx + M - 1;
        if (Lz >= zlo[q] && Lz < zhi[q] && Ly >= ylo[q] && Ly < yhi[q]) {
          const float* row = blocks + (size_t)first[q] * E3P + (Lz * E + Ly) * E;
#pragma unroll
          for (int i = 0; i < 4; ++i)
            if (Lx + i >= 0 && Lx + i < E) t[j][i] = row[Lx + i];
        }
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) v[i] += t[j][i];
  }
  *dst = make_float4(v[0], v[1], v[2], v[3]);
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
// ---- warp FFT: n = 32 R points, R complex values per lane -----------------
// Lane L holds v[j] = x[32 j + L].  With m = 32 j + L and k = k1 + R k2,
//   X[k] = sum_L W_32^{L k2} [ W_n^{L k1} sum_j x[32 j + L] W_R^{j k1} ],
// so each lane first takes an R-point DFT over its registers, multiplies by
// W_n^{L k1}, and the warp then takes 32-point DFTs across lanes by radix-2
// decimation in frequency with shuffles (spans 16, 8, 4, 2, 1).  On return
// lane L, register k1 holds X[k1 + R bitrev5(L)].  tw[j] = W_n^j = exp(-2 pi i j/n)
// for j < n; dir = +1 conjugates every twiddle (unnormalised inverse).
template <int R>
__device__ __forceinline__ void warp_fft(float2 (&v)[R], const float2* tw, int dir) {
  constexpr int n = 32 * R;
  const int L = threadIdx.x & 31;
  const float sg = dir > 0 ? -1.f : 1.f;
  float2 y[R];
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) {
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int j = 0; j < R; ++j) {
      float2 w = tw[(32 * j * k1) % n];
      w.y *= sg;
      acc.x += v[j].x * w.x - v[j].y * w.y;
      acc.y += v[j].x * w.y + v[j].y * w.x;
    }
    y[k1] = acc;
  }
#pragma unroll
  for (int k1 = 1; k1 < R; ++k1) {
    float2 w = tw[(L * k1) % n];
    w.y *= sg;
    y[k1] = cmul(y[k1], w);
  }
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    float2 w = tw[((L & (s - 1)) * (16 / s)) * R];
    w.y *= sg;
    const bool upper = (L & s) != 0;
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      float2 o;
      o.x = __shfl_xor_sync(0xffffffffu, y[k1].x, s);
      o.y = __shfl_xor_sync(0xffffffffu, y[k1].y, s);
      if (!upper) y[k1] = make_float2(y[k1].x + o.x, y[k1].y + o.y);
      else y[k1] = cmul(make_float2(o.x - y[k1].x, o.y - y[k1].y), w);
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) v[k1] = y[k1];
}

__device__ __forceinline__ void full_twiddles(float2* tw, int n) {
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    float sn, cs;
    sincospif(-2.0f * (float)j / (float)n, &sn, &cs);
    tw[j] = make_float2(cs, sn);
  }
}

// Position k' in I_N (k' = k + N/2) of FFT index f, or -1 if f is not kept.
__device__ __forceinline__ int kept_pos(int f, int N, int n) {
  if (f < N / 2) return f + N / 2;
  if (f >= n - N / 2) return f - n + N / 2;
  return -1;
}

constexpr int WF_WARPS = 8;
constexpr int WF_LINES = 16;   // adjacent lines per CTA in the strided passes
constexpr int WF_PITCH = WF_LINES + 1;

// Pass 1: forward x, real grid [z][y][x] -> A1[z][y][kx'] (n x n x N), one row per warp.
template <int R>
__global__ void __launch_bounds__(32 * WF_WARPS)
    k_wfft_x_fwd(const float* __restrict__ g, float2* __restrict__ A1, int N) {
  constexpr int n = 32 * R;
  __shared__ float2 tw[n];
  __shared__ float2 rowbuf[WF_WARPS][n];
  full_twiddles(tw, n);
  __syncthreads();
  const int L = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r = (long long)blockIdx.x * WF_WARPS + w;
  float2 v[R];
#pragma unroll
  for (int j = 0; j < R; ++j) v[j] = make_float2(g[r * n + 32 * j + L], 0.f);
  warp_fft<R>(v, tw, -1);
  const int br = (int)(__brev((unsigned)L) >> 27);
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) {
    const int kp = kept_pos(k1 + R * br, N, n);
    if (kp >= 0) rowbuf[w][kp] = v[k1];
  }
  __syncwarp();
  for (int i = L; i < N; i += 32) A1[r * N + i] = rowbuf[w][i];
}

// Pass 5: inverse x, A4[z][y][kx'] -> real grid [z][y][x], one row per warp.
template <int R>
__global__ void __launch_bounds__(32 * WF_WARPS)
    k_wfft_x_inv(const float2* __restrict__ A4, float* __restrict__ g, int N) {
  constexpr int n = 32 * R;
  __shared__ float2 tw[n];
  __shared__ float rowbuf[WF_WARPS][n];
  full_twiddles(tw, n);
  __syncthreads();
  const int L = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long r = (long long)blockIdx.x * WF_WARPS + w;
  float2 v[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const int kp = kept_pos(32 * j + L, N, n);
    v[j] = kp >= 0 ? A4[r * N + kp] : make_float2(0.f, 0.f);
  }
  warp_fft<R>(v, tw, +1);
  const int br = (int)(__brev((unsigned)L) >> 27);
#pragma unroll
  for (int k1 = 0; k1 < R; ++k1) rowbuf[w][k1 + R * br] = v[k1].x;
  __syncwarp();
  for (int i = L; i < n; i += 32) g[r * n + i] = rowbuf[w][i];
}

// Passes 1 + 2 fused, one CTA per z-plane (grids up to 128^3): the plane's n
// rows are transformed along x (N of n outputs kept) into shared memory, then
// its N columns along y (N kept), and the N x N block is written to
// A2[z][ky'][kx'].  Shared rows are padded by one element so that a column's
// lanes fall into different banks.
constexpr int WP_WARPS = 16;   // warps of a plane CTA
template <int R>
__global__ void __launch_bounds__(32 * WP_WARPS)
    k_wfft_xy_fwd(const float* __restrict__ g, float2* __restrict__ A2, int N) {
  constexpr int n = 32 * R;
  extern __shared__ __align__(16) float2 psh[];
  float2* tw = psh;                  // [n]
  float2* plane = tw + n;            // [n][N + 1]: rows after the x transform
  float2* blk = plane + n * (N + 1); // [N][N]: the kept (ky', kx') block
  const int P = N + 1;
  full_twiddles(tw, n);
  __syncthreads();
  const int L = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long z = blockIdx.x;
  const int br = (int)(__brev((unsigned)L) >> 27);
  for (int y = w; y < n; y += WP_WARPS) {
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = make_float2(g[(z * n + y) * n + 32 * j + L], 0.f);
    warp_fft<R>(v, tw, -1);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const int kp = kept_pos(k1 + R * br, N, n);
      if (kp >= 0) plane[y * P + kp] = v[k1];
    }
  }
  __syncthreads();
  for (int kx = w; kx < N; kx += WP_WARPS) {
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) v[j] = plane[(32 * j + L) * P + kx];
    warp_fft<R>(v, tw, -1);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) {
      const int kp = kept_pos(k1 + R * br, N, n);
      if (kp >= 0) blk[kp * N + kx] = v[k1];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) A2[z * N * N + i] = blk[i];
}

// Passes 4 + 5 fused, one CTA per z-plane: the N x N block of A2[z] is
// transformed back along y (zero outside I_N, n outputs), then every row along x,
// and the real parts are written to the grid.
template <int R>
__global__ void __launch_bounds__(32 * WP_WARPS)
    k_wfft_yx_inv(const float2* __restrict__ A2, float* __restrict__ g, int N) {
  constexpr int n = 32 * R;
  extern __shared__ __align__(16) float2 psh[];
  float2* tw = psh;                  // [n]
  float2* blk = tw + n;              // [N][N + 1]
  float2* plane = blk + N * (N + 1); // [n][N + 1]: columns after the y transform
  float* rowbuf = reinterpret_cast<float*>(plane + n * (N + 1));  // [WP_WARPS][n]
  const int P = N + 1;
  full_twiddles(tw, n);
  const long long z = blockIdx.x;
  for (int i = threadIdx.x; i < N * N; i += blockDim.x) blk[(i / N) * P + i % N] = A2[z * N * N + i];
  __syncthreads();
  const int L = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int br = (int)(__brev((unsigned)L) >> 27);
  for (int kx = w; kx < N; kx += WP_WARPS) {
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int kp = kept_pos(32 * j + L, N, n);
      v[j] = kp >= 0 ? blk[kp * P + kx] : make_float2(0.f, 0.f);
    }
    warp_fft<R>(v, tw, +1);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) plane[(k1 + R * br) * P + kx] = v[k1];
  }
  __syncthreads();
  float* rb = rowbuf + w * n;
  for (int y = w; y < n; y += WP_WARPS) {
    float2 v[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const int kp = kept_pos(32 * j + L, N, n);
      v[j] = kp >= 0 ? plane[y * P + kp] : make_float2(0.f, 0.f);
    }
    warp_fft<R>(v, tw, +1);
#pragma unroll
    for (int k1 = 0; k1 < R; ++k1) rb[k1 + R * br] = v[k1].x;
    __syncwarp();
    for (int i = L; i < n; i += 32) g[(z * n + y) * n + i] = rb[i];
    __syncwarp();
  }
}

template <int R>
constexpr size_t wfft_plane_smem(int N) {
  return sizeof(float2) * (32 * R + (size_t)(32 * R) * (N + 1) + (size_t)N * (N + 1)) +
         sizeof(float) * WP_WARPS * 32 * R;
}

// Passes 2 and 4 (y) and 3 (z): lines at a stride, WF_LINES adjacent lines per
// CTA staged through shared memory so global accesses stay coalesced.
//   mode 0 (y forward):  in A1[z][y][kx']  (n rows)  -> out A2[z][ky'][kx'] (N rows)
//   mode 1 (y inverse):  in A2[z][ky'][kx'] (N rows) -> out A4[z][y][kx']   (n rows)
//   mode 2 (z, scaled):  in/out A2 lines along z at fixed (ky', kx')
// Row e of a line group starts at base + e * rstride; the group's lines are
// the WF_LINES consecutive complex values there.
template <int R>
__global__ void __launch_bounds__(32 * WF_WARPS)
    k_wfft_lines(const float2* __restrict__ in, float2* __restrict__ out, int N, int mode,
                 const float* __restrict__ scale, const float* __restrict__ full) {
  constexpr int n = 32 * R;
  extern __shared__ __align__(16) float2 wsh[];
  float2* tw = wsh;
  float2* tin = wsh + n;               // [n][WF_PITCH]
  float2* tout = tin + n * WF_PITCH;   // [n][WF_PITCH]
  full_twiddles(tw, n);
  const int groups = N / WF_LINES;
  const int gi = blockIdx.x % groups;
  const long long outer = blockIdx.x / groups;   // z (modes 0, 1) or ky' (mode 2)
  const int kx0 = gi * WF_LINES;
  const int rows_in = mode == 1 ? N : n, rows_out = mode == 0 ? N : n;
  long long in_base, in_stride, out_base, out_stride;
  if (mode == 2) {
    in_base = out_base = outer * N + kx0;
    in_stride = out_stride = (long long)N * N;
  } else {
    in_base = outer * rows_in * (long long)N + kx0;
    out_base = outer * rows_out * (long long)N + kx0;
    in_stride = out_stride = N;
  }
  for (int i = threadIdx.x; i < rows_in * WF_LINES; i += blockDim.x) {
    const int e = i / WF_LINES, l = i - e * WF_LINES;
    tin[e * WF_PITCH + l] = in[in_base + e * in_stride + l];
  }
  __syncthreads();
  const int L = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int br = (int)(__brev((unsigned)L) >> 27);
  for (int l = w; l < WF_LINES; l += WF_WARPS) {
    float2 v[R];
    if (mode == 1) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        const int kp = kept_pos(32 * j + L, N, n);
        v[j] = kp >= 0 ? tin[kp * WF_PITCH + l] : make_float2(0.f, 0.f);
      }
    } else {
#pragma unroll
      for (int j = 0; j < R; ++j) v[j] = tin[(32 * j + L) * WF_PITCH + l];
    }
    warp_fft<R>(v, tw, mode == 1 ? +1 : -1);
    if (mode == 2) {
      // keep I_N, multiply by scale_k, back to natural frequency order, inverse
      // (scale_k separable, or the full table [kz'][ky'][kx'] of a non-smooth kernel)
      const int kyp = (int)outer, kxp = kx0 + l;
      const float fxy = full ? 0.f : scale[kxp] * scale[N + kyp];
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) {
        const int f = k1 + R * br;
        const int kp = kept_pos(f, N, n);
        const float fz = kp < 0 ? 0.f
                         : full ? full[((size_t)kp * N + kyp) * N + kxp]
                                : fxy * scale[2 * N + kp];
        tout[f * WF_PITCH + l] = make_float2(v[k1].x * fz, v[k1].y * fz);
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < R; ++j) v[j] = tout[(32 * j + L) * WF_PITCH + l];
      __syncwarp();
      warp_fft<R>(v, tw, +1);
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) tout[(k1 + R * br) * WF_PITCH + l] = v[k1];
    } else if (mode == 0) {
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) {
        const int kp = kept_pos(k1 + R * br, N, n);
        if (kp >= 0) tout[kp * WF_PITCH + l] = v[k1];
      }
    } else {
#pragma unroll
      for (int k1 = 0; k1 < R; ++k1) tout[(k1 + R * br) * WF_PITCH + l] = v[k1];
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < rows_out * WF_LINES; i += blockDim.x) {
    const int e = i / WF_LINES, l = i - e * WF_LINES;
    out[out_base + e * out_stride + l] = tout[e * WF_PITCH + l];
  }
}

// ---- separable circulant passes (Gaussian kernel) -------------------------
// For the Gaussian the scale b_k / prod_t (n phihat(k_t))^2 is a product over
// the axes, so the grid convolution is one real circulant operator applied
// along each axis in turn: per line, a forward DFT, the axis's factor at every
// kept frequency, an inverse DFT.  With the kept band taken symmetric,
// |k| <= N/2 - 1 (the frequency -N/2 of I_N carries b_k below the plan's
// truncation bound), the operator is real, so two real lines share one complex
// transform: line a in the real part, line b in the imaginary part.
//
// 128-point transforms by 16 threads each (2 per warp), split as 128 = 8 x 16:
// with m = 16a + b and k = c + 8d,
//   X[c + 8d] = sum_b W16^{bd} W128^{bc} sum_a x[16a + b] W8^{ac}.
// Thread b holds x[16a + b], a < 8, takes the 8-point DFT over a in registers
// and applies W128^{bc}.  A transpose through shared memory hands thread
// t = 2c' + b0 the values of column c' at b = 2 b1 + b0, b1 < 8; their
// 8-point DFT over b1, the twiddle W16^{b0 d1} and a 2-point DFT with the
// partner thread t ^ 1 (a shuffle) give X[c' + 8 d1 + 64 b0] (the 16-point
// DFT over b split as 8 x 2).  The inverse runs the same steps backwards.  A
// CTA of 8 warps takes 32 lines (16 pairs): transform f of warp w holds line
// 4w + f in the real part and line 4w + f + 2 in the imaginary part, so the
// two transforms of a warp read neighbouring columns of the y and z passes'
// [element][line] tile, which keeps global accesses coalesced.  The passes run
// in place: every CTA reads its lines before it writes them, and no other CTA
// of the pass touches them.
constexpr int CIRC_LINES = 32;
constexpr int CIRC_WARPS = 8;
// Shared-memory strides that make every transpose, twiddle-table and tile
// access of a transform (16 threads) one wavefront: rows c of a transform's
// [c][b] block 18 float2 apart, tile rows 34 floats apart.
constexpr int CIRC_RS = 18, CIRC_FS = 8 * CIRC_RS, CIRC_P = 34;

__device__ __forceinline__ float2 c_add(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 c_sub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
// a * w for the complex w = c + i s
__device__ __forceinline__ float2 c_rot(float2 a, float c, float s) {
  return make_float2(a.x * c - a.y * s, a.x * s + a.y * c);
}
// 4-point DFT in place, natural order in and out (forward: exponent -)
template <bool FWD>
__device__ __forceinline__ void dft4(float2& a0, float2& a1, float2& a2, float2& a3) {
  const float2 t0 = c_add(a0, a2), t1 = c_sub(a0, a2), t2 = c_add(a1, a3), t3 = c_sub(a1, a3);
  a0 = c_add(t0, t2);
  a2 = c_sub(t0, t2);
  // forward: X1 = t1 - i t3, X3 = t1 + i t3; inverse the other way round
  const float2 mi = FWD ? make_float2(t3.y, -t3.x) : make_float2(-t3.y, t3.x);
  a1 = c_add(t1, mi);
  a3 = c_sub(t1, mi);
}
// 8-point DFT of v (natural order in and out) as 4 x 2.
template <bool FWD>
__device__ __forceinline__ void dft8(float2 (&v)[8]) {
  constexpr float R2 = 0.70710678118654752f;
  const float sg = FWD ? -1.f : 1.f;
  float2 e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
  float2 o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
  dft4<FWD>(e0, e1, e2, e3);
  dft4<FWD>(o0, o1, o2, o3);
  o1 = c_rot(o1, R2, sg * R2);
  o2 = make_float2(-sg * o2.y, sg * o2.x);
  o3 = c_rot(o3, -R2, sg * R2);
  v[0] = c_add(e0, o0); v[4] = c_sub(e0, o0);
  v[1] = c_add(e1, o1); v[5] = c_sub(e1, o1);
  v[2] = c_add(e2, o2); v[6] = c_sub(e2, o2);
  v[3] = c_add(e3, o3); v[7] = c_sub(e3, o3);
}

template <int AXIS>
__global__ void __launch_bounds__(32 * CIRC_WARPS)
    k_circ(float* __restrict__ g, const float* __restrict__ scale, int N) {
  constexpr int n = 128;
  constexpr int P = CIRC_P;
  constexpr float R2 = 0.70710678118654752f, C1 = 0.92387953251128674f,
                  S1 = 0.38268343236508978f;
  // W16^{d}, d < 8 (cos, -sin)
  constexpr float W16C[8] = {1.f, C1, R2, S1, 0.f, -S1, -R2, -C1};
  constexpr float W16S[8] = {0.f, -S1, -R2, -C1, -1.f, -C1, -R2, -S1};
  __shared__ float2 tw[CIRC_FS];  // W128^{b c} at c * CIRC_RS + b, c < 8, b < 16
  __shared__ float fac[n];
  __shared__ float2 buf[CIRC_WARPS * 2 * CIRC_FS];  // per transform: [c][b] at c * CIRC_RS + b
  __shared__ float tile[AXIS == 0 ? 1 : n * P];
  for (int j = threadIdx.x; j < n; j += blockDim.x) {
    const int cj = j >> 4, bj = j & 15;
    if (cj < 8) {
      float sn, cs;
      sincospif(-2.0f * (float)(bj * cj) / (float)n, &sn, &cs);
      tw[cj * CIRC_RS + bj] = make_float2(cs, sn);
    }
    // this axis's factor at frequency index j (k = j or j - n), zero outside |k| < N/2
    const int k = j < n / 2 ? j : j - n;
    fac[j] = (k > -N / 2 && k < N / 2) ? scale[AXIS * N + k + N / 2] : 0.f;
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int f = lane >> 4, b = lane & 15;      // transform of the warp, thread within it
  const int la = 4 * w + f, lb = la + 2;       // its real and imaginary line
  const int cq = b >> 1, b0 = b & 1;           // column and half of the second stage
  const int c = blockIdx.x;
  auto addr = [&](int e, int l) -> long long {
    if (AXIS == 0) return ((long long)c * CIRC_LINES + l) * n + e;
    const int x0 = (c % (n / CIRC_LINES)) * CIRC_LINES, o = c / (n / CIRC_LINES);
    if (AXIS == 1) return ((long long)o * n + e) * n + x0 + l;
    return ((long long)e * n + o) * n + x0 + l;
  };
  constexpr int PER = n * CIRC_LINES / (32 * CIRC_WARPS);
  float2 v[8];
  if (AXIS == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = make_float2(g[addr(16 * a + b, la)], g[addr(16 * a + b, lb)]);
  } else {
    float t[PER];
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = threadIdx.x + 32 * CIRC_WARPS * r;
      t[r] = g[addr(i / CIRC_LINES, i % CIRC_LINES)];
    }
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = threadIdx.x + 32 * CIRC_WARPS * r;
      tile[(i / CIRC_LINES) * P + i % CIRC_LINES] = t[r];
    }
  }
  __syncthreads();
  if (AXIS != 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) v[a] = make_float2(tile[(16 * a + b) * P + la], tile[(16 * a + b) * P + lb]);
  }
  float2* B = buf + (w * 2 + f) * CIRC_FS;
  // forward: 8-point DFT over a, twiddle W128^{b c}, transpose
  dft8<true>(v);
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const float2 t = tw[cc * CIRC_RS + b];
    B[cc * CIRC_RS + b] = c_rot(v[cc], t.x, t.y);
  }
  __syncwarp();
#pragma unroll
  for (int b1 = 0; b1 < 8; ++b1) v[b1] = B[cq * CIRC_RS + 2 * b1 + b0];
  __syncwarp();
  // 8-point DFT over b1, twiddle W16^{b0 d1}, 2-point DFT over b0 with the partner
  dft8<true>(v);
#pragma unroll
  for (int d1 = 0; d1 < 8; ++d1) {
    const float wc = b0 ? W16C[d1] : 1.f, ws = b0 ? W16S[d1] : 0.f;
    const float2 z = c_rot(v[d1], wc, ws);
    const float2 p = make_float2(__shfl_xor_sync(0xffffffffu, z.x, 1),
                                 __shfl_xor_sync(0xffffffffu, z.y, 1));
    v[d1] = b0 ? c_sub(p, z) : c_add(z, p);
  }
  // v[d1] = X[cq + 8 d1 + 64 b0]: scale, then the inverse 2-point DFT over d0
  // with the partner, twiddle W16^{-b0 d1}, 8-point DFT over d1
#pragma unroll
  for (int d1 = 0; d1 < 8; ++d1) {
    const float s = fac[cq + 8 * d1 + 64 * b0];
    const float2 z = make_float2(v[d1].x * s, v[d1].y * s);
    const float2 p = make_float2(__shfl_xor_sync(0xffffffffu, z.x, 1),
                                 __shfl_xor_sync(0xffffffffu, z.y, 1));
    const float2 u = b0 ? c_sub(p, z) : c_add(z, p);
    const float wc = b0 ? W16C[d1] : 1.f, ws = b0 ? W16S[d1] : 0.f;
    v[d1] = c_rot(u, wc, -ws);
  }
  dft8<false>(v);
  // v[b1] = value at b = 2 b1 + b0 of column cq: twiddle W128^{-b cq}, transpose
#pragma unroll
  for (int b1 = 0; b1 < 8; ++b1) {
    const int bb = 2 * b1 + b0;
    const float2 t = tw[cq * CIRC_RS + bb];
    B[cq * CIRC_RS + bb] = c_rot(v[b1], t.x, -t.y);
  }
  __syncwarp();
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) v[cc] = B[cc * CIRC_RS + b];
  dft8<false>(v);
  // v[a] = line values at element 16a + b (line la in x, line lb in y)
  if (AXIS == 0) {
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      g[addr(16 * a + b, la)] = v[a].x;
      g[addr(16 * a + b, lb)] = v[a].y;
    }
  } else {
    __syncthreads();  // every warp has read its lines of the tile
#pragma unroll
    for (int a = 0; a < 8; ++a) {
      tile[(16 * a + b) * P + la] = v[a].x;
      tile[(16 * a + b) * P + lb] = v[a].y;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int i = threadIdx.x + 32 * CIRC_WARPS * r;
      g[addr(i / CIRC_LINES, i % CIRC_LINES)] = tile[(i / CIRC_LINES) * P + i % CIRC_LINES];
    }
  }
}

uotk_status circ_convolve(uotk_ctx* ctx, cudaStream_t s, int N, const float* scale, float* g) {
  constexpr int n = 128;
  const unsigned blocks = (unsigned)((long long)n * n / CIRC_LINES);
  k_circ<0><<<blocks, 32 * CIRC_WARPS, 0, s>>>(g, scale, N);
  UOTK_LAUNCHED(ctx);
  k_circ<1><<<blocks, 32 * CIRC_WARPS, 0, s>>>(g, scale, N);
  UOTK_LAUNCHED(ctx);
  k_circ<2><<<blocks, 32 * CIRC_WARPS, 0, s>>>(g, scale, N);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

template <int R>
uotk_status wfft_convolve(uotk_ctx* ctx, cudaStream_t s, int N, const float* scale,
                          const float* full, const float* grid_in, float2* A1, float2* A2,
                          float* grid_out) {
  constexpr int n = 32 * R;
  const size_t lsmem = sizeof(float2) * (n + 2 * n * WF_PITCH);
  UOTK_CUDA(ctx, smem_attr(s, k_wfft_lines<R>, lsmem));
  const size_t psmem = wfft_plane_smem<R>(N);
  if (psmem <= (size_t)ctx->max_smem_optin) {
    // three passes: x and y of each z-plane in one CTA, z, then y and x back
    UOTK_CUDA(ctx, smem_attr(s, k_wfft_xy_fwd<R>, psmem));
    UOTK_CUDA(ctx, smem_attr(s, k_wfft_yx_inv<R>, psmem));
    k_wfft_xy_fwd<R><<<n, 32 * WP_WARPS, psmem, s>>>(grid_in, A2, N);
    UOTK_LAUNCHED(ctx);
    k_wfft_lines<R><<<N * (N / WF_LINES), 32 * WF_WARPS, lsmem, s>>>(A2, A2, N, 2, scale, full);
    UOTK_LAUNCHED(ctx);
    k_wfft_yx_inv<R><<<n, 32 * WP_WARPS, psmem, s>>>(A2, grid_out, N);
    UOTK_LAUNCHED(ctx);
    return UOTK_OK;
  }
  k_wfft_x_fwd<R><<<n * n / WF_WARPS, 32 * WF_WARPS, 0, s>>>(grid_in, A1, N);
  UOTK_LAUNCHED(ctx);
  k_wfft_lines<R><<<n * (N / WF_LINES), 32 * WF_WARPS, lsmem, s>>>(A1, A2, N, 0, scale, full);
  UOTK_LAUNCHED(ctx);
  k_wfft_lines<R><<<N * (N / WF_LINES), 32 * WF_WARPS, lsmem, s>>>(A2, A2, N, 2, scale, full);
  UOTK_LAUNCHED(ctx);
  k_wfft_lines<R><<<n * (N / WF_LINES), 32 * WF_WARPS, lsmem, s>>>(A2, A1, N, 1, scale, full);
  UOTK_LAUNCHED(ctx);
  k_wfft_x_inv<R><<<n * n / WF_WARPS, 32 * WF_WARPS, 0, s>>>(A1, grid_out, N);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
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
               int mode, int dir, const float* __restrict__ scale, int N,
               const float* __restrict__ full) {
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
        f = full ? full[((size_t)(kz + N / 2) * N + ky + N / 2) * N + kx + N / 2]
                 : scale[kx + N / 2] * scale[N + ky + N / 2] * scale[2 * N + kz + N / 2];
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
// Warp sum of four per-lane values at once: lane L returns the total of
// v[L >> 3].  Two transposed butterfly levels (each lane keeps half of its
// values and sends the other half) then three plain ones.
__device__ __forceinline__ float warp_sum4(const float (&v)[4], int lane) {
  const bool b4 = lane & 16, b3 = lane & 8;
  const float r0 = (b4 ? v[2] : v[0]) + __shfl_xor_sync(0xffffffffu, b4 ? v[0] : v[2], 16);
  const float r1 = (b4 ? v[3] : v[1]) + __shfl_xor_sync(0xffffffffu, b4 ? v[1] : v[3], 16);
  float r = (b3 ? r1 : r0) + __shfl_xor_sync(0xffffffffu, b3 ? r0 : r1, 8);
  r += __shfl_xor_sync(0xffffffffu, r, 4);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

// DUAL: the dual half-step `du` of each target follows its sum in the same
// kernel (the arithmetic of k_dual_update<false>; t is still written to out).
template <int M, bool DUAL, int C = CH>
__global__ void __launch_bounds__(256)
    k_gather(const float* __restrict__ win, const int* __restrict__ ckey,
             const int* __restrict__ unit_tile, const int* __restrict__ unit_begin,
             const int* __restrict__ unit_count, const int* __restrict__ num_units, int n,
             int tiles1, const float* __restrict__ grid, float* __restrict__ out,
             long long* __restrict__ flags, DualUpdate du) {
  using G = Geo<M, C>;
  constexpr int W2 = G::W2, E = G::E, E2 = G::E2, E3 = G::E3, WS = G::WS;
  constexpr int YO = nfft_win_yoff(M), ZO = nfft_win_zoff(M);
  constexpr int NIT = (W2 * W2 + 31) / 32;
  // Footprint of the current cell kept in registers while a warp's consecutive
  // targets share that cell.
  constexpr bool CACHE = NIT * W2 <= 64;
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) unsigned long long bars[STAGES];
  __shared__ __align__(8) unsigned long long never;  // nothing arrives (time-out test)
  float* blk = smem;
  float* stage0 = smem + G::E3P;
  const int u = blockIdx.x;
  if (DUAL && u == 0 && threadIdx.x == 0) {
    flags[du.reset_slot] = ORDERED_NEG_INF;
    if (du.reset_delta >= 0) flags[du.reset_delta] = ORDERED_NEG_INF;
  }
  if (u >= *num_units) return;
  const int b0 = unit_begin[u], cnt = unit_count[u];
  const int nchunks = (cnt + C - 1) / C;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) mbar_init(&bars[s], 1);
    mbar_init(&never, 1);
    mbar_fence_init();
    for (int k = 0; k < STAGES && k < nchunks; ++k)
      stage_chunk<M, C>(stage0 + k * G::STAGE_F, &bars[k], win, ckey, nullptr, b0 + k * C,
                     min(C, cnt - k * C));
  }
  // Dual half-step state.  A warp parks the sums of its targets one per lane
  // and updates 32 targets at once with every lane active: an FP64
  // instruction costs the FP64 pipe a whole warp's issue whatever its mask,
  // and FP64 throughput is scarce on this GPU.
  const double qs = DUAL ? du.q * ordered_to_dbl(flags[du.shift_in]) : 0.0;
  double dmx = -INFINITY, ddl = 0.0;
  long long dbad = 0;
  float dt = 0.f;  // parked sum of this lane
  int di = -1;     // its target (-1: none)
  int dn = 0;      // group of four targets that parks next (warp-uniform)
  auto dual_flush = [&]() {
    if (di >= 0) {
      const float lt = logf(dt);  // -inf for 0, nan for negatives: flagged below
      const double v = du.ref == 0 ? fma(-du.q, (double)lt, -qs)
                                   : fma(du.q, (double)(logf(du.base[di]) - lt), -qs);
      if (du.delta_out >= 0) ddl = fmax(ddl, fabs(v - du.pot[di]));
      du.pot[di] = v;
      if (isfinite(v)) dmx = fmax(dmx, v);
      else ++dbad;
    }
    di = -1;
    dn = 0;
  };
  int tx0, ty0, tz0;
  tile_origin(unit_tile[u], tiles1, tx0, ty0, tz0);
  for (int i = threadIdx.x; i < E3; i += blockDim.x) {
    const int lz = i / E2, ly = (i / E) % E, lx = i % E;
    const int gz = wrap_node(tz0 - M + 1 + lz, n), gy = wrap_node(ty0 - M + 1 + ly, n),
              gx = wrap_node(tx0 - M + 1 + lx, n);
    blk[i] = grid[((long long)gz * n + gy) * n + gx];
  }
  __syncthreads();  // barriers initialised and block staged before anyone waits or reads
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int off[NIT], kxs[NIT], kys[NIT];
#pragma unroll
  for (int it = 0; it < NIT; ++it) {
    const int c = lane + 32 * it;
    const int kx = c % W2, ky = c / W2;
    kxs[it] = nfft_win_xoff(M, kx);  // offset of phi_x[kx] in the window row
    kys[it] = YO + ky;               // offset of phi_y[ky]
    off[it] = c < W2 * W2 ? ky * E + kx : -1;
  }
  float hc[CACHE ? NIT * W2 : 1];
  int cached = -1;
  for (int k = 0; k < nchunks; ++k) {
    if (!stage_ready(bars, k, nchunks, flags, &never)) return;
    const int q0 = b0 + k * C, cn = min(C, cnt - k * C), koff = q0 & 3;
    const float* sw = stage0 + (k % STAGES) * G::STAGE_F;
    const int* skey = reinterpret_cast<const int*>(sw + C * WS) + koff;
    // each warp takes a contiguous run of the chunk's targets: neighbours in
    // cell order share a footprint more often than every nwarps-th target
    const int per = (cn + nwarps - 1) / nwarps, pend = min(cn, (warp + 1) * per);
    // this lane's part of the sum of target p (the warp adds the 32 parts)
    auto target_part = [&](int p) -> float {
      const int key = skey[p];
      const int bx = (key & 1023) - tx0, by = ((key >> 10) & 1023) - ty0, bz = (key >> 20) - tz0;
      const float* wq = sw + p * WS;
      const float* src = blk + (bz * E + by) * E + bx;
      float fz[W2];
      load_vec<W2>(wq + ZO, fz);
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
          // z-contraction of the column in packed pairs (z even, z odd)
          unsigned long long s2 = 0ull;
#pragma unroll
          for (int kk = 0; kk < W2; kk += 2)
            s2 = f2_fma(f2_pack(fz[kk], fz[kk + 1]),
                        f2_pack(hc[CACHE ? it * W2 + kk : 0], hc[CACHE ? it * W2 + kk + 1 : 0]),
                        s2);
          float se, so;
          f2_unpack(s2, se, so);
          const float pxy = off[it] >= 0 ? wq[kxs[it]] * wq[kys[it]] : 0.f;
          acc = fmaf(pxy, se + so, acc);
        }
      } else {
#pragma unroll
        for (int it = 0; it < NIT; ++it) {
          if (off[it] >= 0) {
            const float pxy = wq[kxs[it]] * wq[kys[it]];
            const float* col = src + off[it];
            float s = 0.f;
#pragma unroll
            for (int kk = 0; kk < W2; ++kk) s = fmaf(fz[kk], col[kk * E2], s);
            acc = fmaf(pxy, s, acc);
          }
        }
      }
      return acc;
    };
    // Targets in groups of four: each lane keeps its four parts and one
    // transposed reduction adds them (6 shuffles for four sums instead of 20);
    // lanes 8j..8j+7 then hold the sum of target p + j.
    for (int p = warp * per; p < pend; p += 4) {
      float part[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) part[j] = p + j < pend ? target_part(p + j) : 0.f;
      const float tsum = warp_sum4(part, lane);
      const int t = p + (lane >> 3);
      if ((lane & 7) == 0 && t < pend) out[q0 + t] = tsum;
      if (DUAL) {
        // group g of eight parks in lanes 8j + g: eight groups fill the warp
        if ((lane & 7) == dn && t < pend) {
          dt = tsum;
          di = q0 + t;
        }
        if (++dn == 8) dual_flush();
      }
    }
    __syncthreads();
    if (threadIdx.x == 0 && k + STAGES < nchunks)
      stage_chunk<M, C>(stage0 + (k % STAGES) * G::STAGE_F, &bars[k % STAGES], win, ckey, nullptr,
                     b0 + (k + STAGES) * C, min(C, cnt - (k + STAGES) * C));
  }
  if (DUAL) {
    dual_flush();
    // block maxima and count: warp shuffles, then one slot per warp
    dmx = warp_max(dmx);
    ddl = warp_max(ddl);
    dbad = warp_sum(dbad);
    __shared__ double dsh[2][8];
    if (lane == 0) {
      dsh[0][warp] = dmx;
      dsh[1][warp] = ddl;
      if (dbad) flag_add(&flags[FLAG_NONFINITE_DUAL], dbad);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < nwarps; ++w) {
        dmx = fmax(dmx, dsh[0][w]);
        ddl = fmax(ddl, dsh[1][w]);
      }
      atomicMax(&flags[du.max_out], dbl_to_ordered(du.lam * dmx));
      if (du.delta_out >= 0) atomicMax(&flags[du.delta_out], dbl_to_ordered(du.lam * ddl));
    }
  }
}

// Gather, even m <= 6 (the per-warp form).  Each warp takes a contiguous run
// of the unit's targets and stages their window rows and cells itself
// (double-buffered bulk copies of GW targets completing on the warp's own
// mbarriers), so after the grid block is staged no warp waits for another.
// Lane (zg, yg, xh) owns the BZ x BZ x m footprint nodes z in [zg BZ, +BZ),
// y in [yg BZ, +BZ), x in [xh m, +m), BZ = m/2 (4 x 4 x 2 lanes cover the
// (2m)^3 nodes), held in registers as x pairs while consecutive targets share
// a cell.  Per target, lane part = sum_x phi_x sum_{z,y} (phi_z phi_y) g[z][y][x]
// (the inner sums packed over x pairs), and the warp adds the 32 parts.
constexpr int GW = 32;      // targets per per-warp staging buffer (two per warp)
constexpr int GWARPS = 16;  // warps of a gather CTA (one CTA per SM: all 64K registers at 128 a thread)
template <int M>
struct GatherGeo {
  static constexpr int E = NFFT_TILE + 2 * M - 1;
  static constexpr int E3P = (E * E * E + 3) & ~3;
  static constexpr int WS = nfft_win_stride(M);
  static constexpr int BUF_F = GW * WS + GW + 4;   // window rows, then cells (align slack)
  static constexpr int WARP_F = 2 * BUF_F;
  static_assert(BUF_F % 4 == 0, "16-byte aligned buffers");
};

template <int M>
__device__ __forceinline__ void stage_warp(float* buf, unsigned long long* bar,
                                           const float* win, const int* ckey, int q0, int cn) {
  constexpr int WS = GatherGeo<M>::WS;
  const int off = q0 & 3;
  const unsigned wbytes = (unsigned)(cn * WS * 4);
  const unsigned kbytes = (unsigned)(((cn + off + 3) & ~3) * 4);
  mbar_expect(bar, wbytes + kbytes);
  bulk_copy(buf, win + (size_t)q0 * WS, wbytes, bar);
  bulk_copy(buf + GW * WS, ckey + (q0 - off), kbytes, bar);
}

template <int M, bool DUAL>
__global__ void __launch_bounds__(32 * GWARPS, 1)
    k_gather_w(const float* __restrict__ win, const int* __restrict__ ckey,
               const int* __restrict__ unit_tile, const int* __restrict__ unit_begin,
               const int* __restrict__ unit_count, const int* __restrict__ chunk_unit_start,
               int n, int tiles1, const float* __restrict__ grid, float* __restrict__ out,
               long long* __restrict__ flags, DualUpdate du) {
  using GG = GatherGeo<M>;
  constexpr int E = GG::E, E2 = E * E, E3 = E2 * E, WS = GG::WS;
  constexpr int BZ = M / 2, MP = M / 2;
  constexpr int HP = nfft_win_half(M), YO = nfft_win_yoff(M), ZO = nfft_win_zoff(M);
  static_assert(M % 2 == 0 && M <= 6, "per-warp gather: even m <= 6");
  extern __shared__ __align__(16) float smem[];
  __shared__ __align__(8) unsigned long long bars[GWARPS][2];
  __shared__ __align__(8) unsigned long long never;  // nothing arrives (time-out test)
  float* blk = smem;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* wbuf = smem + GG::E3P + warp * GG::WARP_F;
  if (DUAL && blockIdx.x == 0 && threadIdx.x == 0) {
    flags[du.reset_slot] = ORDERED_NEG_INF;
    if (du.reset_delta >= 0) flags[du.reset_delta] = ORDERED_NEG_INF;
  }
  // the CTA's chunk: units ubeg .. uend - 1, taken in turn; kw counts the warp's
  // staging chunks of the earlier units (the barriers' phases run on)
  const int ubeg = chunk_unit_start[blockIdx.x], uend = chunk_unit_start[blockIdx.x + 1];
  if (lane == 0) {
    mbar_init(&bars[warp][0], 1);
    mbar_init(&bars[warp][1], 1);
    if (warp == 0) mbar_init(&never, 1);
    mbar_fence_init();
  }
  // Dual half-step state (as in k_gather): sums parked one per lane, 32 targets
  // updated at once with every lane active.
  const double qs = DUAL ? du.q * ordered_to_dbl(flags[du.shift_in]) : 0.0;
  double dmx = -INFINITY, ddl = 0.0;
  long long dbad = 0;
  float dt = 0.f;
  int di = -1, dn = 0;
  auto dual_flush = [&]() {
    if (di >= 0) {
      const float lt = logf(dt);  // -inf for 0, nan for negatives: flagged below
      const double v = du.ref == 0 ? fma(-du.q, (double)lt, -qs)
                                   : fma(du.q, (double)(logf(du.base[di]) - lt), -qs);
      if (du.delta_out >= 0) ddl = fmax(ddl, fabs(v - du.pot[di]));
      du.pot[di] = v;
      if (isfinite(v)) dmx = fmax(dmx, v);
      else ++dbad;
    }
    di = -1;
    dn = 0;
  };
  const int zg = lane >> 3, yg = (lane >> 1) & 3, xh = lane & 1;
  const int z0 = zg * BZ, y0 = yg * BZ;
  unsigned long long hc[BZ][BZ][MP];
  int kw = 0;
  bool dead = false;  // a wait of this warp ran out: it computes nothing more
  for (int u = ubeg; u < uend; ++u) {
    const int b0 = unit_begin[u], cnt = unit_count[u];
    const int per = (cnt + GWARPS - 1) / GWARPS;
    const int wb = min(cnt, warp * per), we = min(cnt, wb + per);
    const int nch = dead ? 0 : (we - wb + GW - 1) / GW;
    // every warp is done with the previous unit's block before it is replaced
    if (u != ubeg) __syncthreads();
    if (lane == 0) {
      // the warp's staging buffers were last read by the generic proxy
      if (u != ubeg) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int k = 0; k < 2 && k < nch; ++k)
        stage_warp<M>(wbuf + ((kw + k) & 1) * GG::BUF_F, &bars[warp][(kw + k) & 1], win, ckey,
                      b0 + wb + k * GW, min(GW, we - wb - k * GW));
    }
    int tx0, ty0, tz0;
    tile_origin(unit_tile[u], tiles1, tx0, ty0, tz0);
    for (int i = threadIdx.x; i < E3; i += blockDim.x) {
      const int lz = i / E2, ly = (i / E) % E, lx = i % E;
      const int gz = wrap_node(tz0 - M + 1 + lz, n), gy = wrap_node(ty0 - M + 1 + ly, n),
                gx = wrap_node(tx0 - M + 1 + lx, n);
      blk[i] = grid[((long long)gz * n + gy) * n + gx];
    }
    __syncthreads();  // barriers initialised and block staged before anyone waits or reads
    int cached = -1;
    // this lane's part of the sum of the target with window row `row`, cell `key`
    // two targets of the same cell (the footprint cached): their sums share the
    // footprint registers and give six independent FMA chains instead of three
    auto target_pair = [&](const float* ra, const float* rb, float& pa, float& pb) {
      unsigned long long Ha[MP], Hb[MP];
#pragma unroll
      for (int j = 0; j < MP; ++j) Ha[j] = Hb[j] = 0ull;
#pragma unroll
      for (int z = 0; z < BZ; ++z) {
        const float za = ra[ZO + z0 + z], zb = rb[ZO + z0 + z];
#pragma unroll
        for (int yy = 0; yy < BZ; ++yy) {
          const float a = za * ra[YO + y0 + yy], b = zb * rb[YO + y0 + yy];
          const unsigned long long A = f2_pack(a, a), B = f2_pack(b, b);
#pragma unroll
          for (int j = 0; j < MP; ++j) {
            Ha[j] = f2_fma(A, hc[z][yy][j], Ha[j]);
            Hb[j] = f2_fma(B, hc[z][yy][j], Hb[j]);
          }
        }
      }
      float fa[M], fb[M];
      load_vec<M>(ra + xh * HP, fa);
      load_vec<M>(rb + xh * HP, fb);
      unsigned long long sa = f2_mul(f2_pack(fa[0], fa[1]), Ha[0]);
      unsigned long long sb = f2_mul(f2_pack(fb[0], fb[1]), Hb[0]);
#pragma unroll
      for (int j = 1; j < MP; ++j) {
        sa = f2_fma(f2_pack(fa[2 * j], fa[2 * j + 1]), Ha[j], sa);
        sb = f2_fma(f2_pack(fb[2 * j], fb[2 * j + 1]), Hb[j], sb);
      }
      float lo, hi;
      f2_unpack(sa, lo, hi);
      pa = lo + hi;
      f2_unpack(sb, lo, hi);
      pb = lo + hi;
    };
    auto target_part = [&](const float* row, int key) -> float {
      if (key != cached) {
        const int bx = (key & 1023) - tx0, by = ((key >> 10) & 1023) - ty0, bz = (key >> 20) - tz0;
        const float* src = blk + ((bz + z0) * E + by + y0) * E + bx + xh * M;
#pragma unroll
        for (int z = 0; z < BZ; ++z)
#pragma unroll
          for (int yy = 0; yy < BZ; ++yy)
#pragma unroll
            for (int j = 0; j < MP; ++j)
              hc[z][yy][j] = f2_pack(src[(z * E + yy) * E + 2 * j], src[(z * E + yy) * E + 2 * j + 1]);
        cached = key;
      }
      float fz[BZ], fy[BZ], fx[M];
#pragma unroll
      for (int k = 0; k < BZ; ++k) {
        fz[k] = row[ZO + z0 + k];
        fy[k] = row[YO + y0 + k];
      }
      load_vec<M>(row + xh * HP, fx);
      unsigned long long H[MP];
#pragma unroll
      for (int j = 0; j < MP; ++j) H[j] = 0ull;
#pragma unroll
      for (int z = 0; z < BZ; ++z)
#pragma unroll
        for (int yy = 0; yy < BZ; ++yy) {
          const float a = fz[z] * fy[yy];
          const unsigned long long A = f2_pack(a, a);
#pragma unroll
          for (int j = 0; j < MP; ++j) H[j] = f2_fma(A, hc[z][yy][j], H[j]);
        }
      unsigned long long r = f2_mul(f2_pack(fx[0], fx[1]), H[0]);
#pragma unroll
      for (int j = 1; j < MP; ++j) r = f2_fma(f2_pack(fx[2 * j], fx[2 * j + 1]), H[j], r);
      float lo, hi;
      f2_unpack(r, lo, hi);
      return lo + hi;
    };
    for (int k = 0; k < nch; ++k) {
      const int q0 = b0 + wb + k * GW, cn = min(GW, we - wb - k * GW);
      const int kg = kw + k;
      float* sb = wbuf + (kg & 1) * GG::BUF_F;
      const bool ok = kg == 0 ? first_wait(&bars[warp][0], 0u, &never, flags)
                              : mbar_wait(&bars[warp][kg & 1], (unsigned)(kg >> 1) & 1u);
      if (__any_sync(0xffffffffu, !ok)) {
        // give up: record it, let this warp's copies in flight land, and stop
        if (lane == 0) {
          flag_add(&flags[FLAG_TIMEOUT], 1LL);
          for (int q = kg; q < kw + nch && q < kg + 2; ++q)
            mbar_wait(&bars[warp][q & 1], (unsigned)(q >> 1) & 1u);
        }
        __syncwarp();
        dead = true;
        break;
      }
      const int* skey = reinterpret_cast<const int*>(sb + GW * WS) + (q0 & 3);
      for (int p = 0; p < cn; p += 4) {
        float part[4];
#pragma unroll
        for (int j = 0; j < 4; j += 2) {
          if (p + j + 1 < cn && skey[p + j] == skey[p + j + 1]) {
            // the first call loads the pair's footprint if needed; then both together
            if (skey[p + j] != cached) (void)target_part(sb + (p + j) * WS, skey[p + j]);
            target_pair(sb + (p + j) * WS, sb + (p + j + 1) * WS, part[j], part[j + 1]);
          } else {
            part[j] = p + j < cn ? target_part(sb + (p + j) * WS, skey[p + j]) : 0.f;
            part[j + 1] = p + j + 1 < cn ? target_part(sb + (p + j + 1) * WS, skey[p + j + 1]) : 0.f;
          }
        }
        const float tsum = warp_sum4(part, lane);
        const int t = p + (lane >> 3);
        if ((lane & 7) == 0 && t < cn) out[q0 + t] = tsum;
        if (DUAL) {
          if ((lane & 7) == dn && t < cn) {
            dt = tsum;
            di = q0 + t;
          }
          if (++dn == 8) dual_flush();
        }
      }
      __syncwarp();
      if (lane == 0 && k + 2 < nch) {
        // the warp's reads of this buffer are done (generic proxy) before the
        // bulk copy (async proxy) overwrites it
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        stage_warp<M>(sb, &bars[warp][kg & 1], win, ckey, q0 + 2 * GW, min(GW, we - wb - (k + 2) * GW));
      }
    }
    kw += nch;
  }
  if (DUAL) {
    dual_flush();
    dmx = warp_max(dmx);
    ddl = warp_max(ddl);
    dbad = warp_sum(dbad);
    __shared__ double dsh[2][GWARPS];
    if (lane == 0) {
      dsh[0][warp] = dmx;
      dsh[1][warp] = ddl;
      if (dbad) flag_add(&flags[FLAG_NONFINITE_DUAL], dbad);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      for (int w = 1; w < GWARPS; ++w) {
        dmx = fmax(dmx, dsh[0][w]);
        ddl = fmax(ddl, dsh[1][w]);
      }
      atomicMax(&flags[du.max_out], dbl_to_ordered(du.lam * dmx));
      if (du.delta_out >= 0) atomicMax(&flags[du.delta_out], dbl_to_ordered(du.lam * ddl));
    }
  }
}

template <int M, int C = CH>
size_t unit_smem() {
  using G = Geo<M, C>;
  return sizeof(float) * (G::E3P + STAGES * G::STAGE_F);
}

// Points per staging chunk of the CTA-staged gather (odd m and m = 8).
// Registers hold it to two CTAs per SM whatever the chunk, and longer chunks
// mean fewer barriers and longer runs of targets per warp.
constexpr int GATHER_CH = 192;

// SMs of the current device (queried once).
int device_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0, v = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && v > 0)
      sms = v;
    else
      return 1;
  }
  return sms;
}

// pw != NULL: the weights w = base e^{lam pot - shift} are formed in the
// kernel; else staged from wts.  The unit blocks go to W.blocks and the fold
// writes the whole grid.
template <int M>
uotk_status launch_spread(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                          const NfftPoints& S, const float* wts, const SpreadWeights* pw,
                          NfftWork& W, float* grid) {
  using SG = SpreadGeo<M, SPREAD_CP>;
  const size_t smem = sizeof(float) * (SG::E3P + STAGES * SG::STAGE_F);
  constexpr int NT = SpreadMap<M>::NTH;
  auto kern = pw ? k_spread<M, true, SPREAD_CP> : k_spread<M, false, SPREAD_CP>;
  {
    UOTK_PROF(ctx, s, "spread");
    UOTK_CUDA(ctx, smem_attr(s, kern, smem));
    kern<<<S.c_spread, NT, smem, s>>>(S.winp, S.ckey, wts, S.unit_tile, S.unit_begin,
                                      S.unit_count, S.unit_box, S.chunk_unit_start, P.tiles1,
                                      W.blocks, ctx->dflags, pw ? *pw : SpreadWeights{});
    UOTK_LAUNCHED(ctx);
  }
  {
    UOTK_PROF(ctx, s, "fold");
    k_fold_units<M><<<S.max_units, FOLD_THREADS, 0, s>>>(W.blocks, S.unit_tile,
                                                         S.tile_unit_start, S.unit_box,
                                                         S.num_units);
    UOTK_LAUNCHED(ctx);
    k_fold<M><<<P.tiles1 * P.tiles1 * P.tiles1, FOLD2_THREADS, 0, s>>>(
        W.blocks, S.tile_unit_start, S.unit_box, P.n, P.tiles1, grid);
    UOTK_LAUNCHED(ctx);
  }
  return UOTK_OK;
}

template <int M>
uotk_status launch_gather(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                          const NfftPoints& S, const float* grid, float* out,
                          const DualUpdate* du) {
  if constexpr (M % 2 == 0 && M <= 6) {
    using GG = GatherGeo<M>;
    const size_t smem = sizeof(float) * (GG::E3P + GWARPS * GG::WARP_F);
    auto kern = du ? k_gather_w<M, true> : k_gather_w<M, false>;
    UOTK_CUDA(ctx, smem_attr(s, kern, smem));
    kern<<<S.c_gather, 32 * GWARPS, smem, s>>>(S.win, S.ckey, S.g_unit_tile, S.g_unit_begin,
                                                S.g_unit_count, S.g_chunk_unit_start, P.n,
                                                P.tiles1, grid, out, ctx->dflags,
                                                du ? *du : DualUpdate{});
  } else {
    const size_t smem = unit_smem<M, GATHER_CH>();
    auto kern = du ? k_gather<M, true, GATHER_CH> : k_gather<M, false, GATHER_CH>;
    UOTK_CUDA(ctx, smem_attr(s, kern, smem));
    kern<<<S.g_max_units, 256, smem, s>>>(S.win, S.ckey, S.g_unit_tile, S.g_unit_begin,
                                          S.g_unit_count, S.g_num_units, P.n, P.tiles1, grid, out,
                                          ctx->dflags, du ? *du : DualUpdate{});
  }
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
                                const NfftPoints& S, const float* wts, const SpreadWeights* pw,
                                NfftWork& W, float* grid) {
#define UOTK_SPREAD_CALL(M) launch_spread<M>(ctx, s, P, S, wts, pw, W, grid)
  UOTK_M_SWITCH(P.m, UOTK_SPREAD_CALL)
#undef UOTK_SPREAD_CALL
}

static uotk_status gather_units(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                                const NfftPoints& S, const float* grid, float* out,
                                const DualUpdate* du) {
#define UOTK_GATHER_CALL(M) launch_gather<M>(ctx, s, P, S, grid, out, du)
  UOTK_M_SWITCH(P.m, UOTK_GATHER_CALL)
#undef UOTK_GATHER_CALL
}

// CTAs of the spread / gather kernel at cut-off m that one SM holds at once.
template <int M>
static int spread_slots_m() {
  using SG = SpreadGeo<M, SPREAD_CP>;
  const size_t smem = sizeof(float) * (SG::E3P + STAGES * SG::STAGE_F);
  auto kern = k_spread<M, true, SPREAD_CP>;
  int per = 0;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
          cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, SpreadMap<M>::NTH, smem) !=
          cudaSuccess)
    per = 1;
  return per > 0 ? per : 1;
}
template <int M>
static int gather_slots_m() {
  int per = 0;
  if constexpr (M % 2 == 0 && M <= 6) {
    using GG = GatherGeo<M>;
    const size_t smem = sizeof(float) * (GG::E3P + GWARPS * GG::WARP_F);
    auto kern = k_gather_w<M, true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 32 * GWARPS, smem) !=
            cudaSuccess)
      per = 1;
  } else {
    per = 2;  // one CTA per unit (k_gather): the number of chunks only sets the unit sizes
  }
  return per > 0 ? per : 1;
}

int nfft_spread_slots(int m) {
  static int per[NFFT_MAX_M + 1] = {};
  if (m < 2 || m > NFFT_MAX_M) return device_sms();
  if (!per[m]) {
    switch (m) {
      case 2: per[m] = spread_slots_m<2>(); break;
      case 3: per[m] = spread_slots_m<3>(); break;
      case 4: per[m] = spread_slots_m<4>(); break;
      case 5: per[m] = spread_slots_m<5>(); break;
      case 6: per[m] = spread_slots_m<6>(); break;
      case 7: per[m] = spread_slots_m<7>(); break;
      default: per[m] = spread_slots_m<8>(); break;
    }
  }
  return per[m] * device_sms();
}

int nfft_gather_slots(int m) {
  static int per[NFFT_MAX_M + 1] = {};
  if (m < 2 || m > NFFT_MAX_M) return device_sms();
  if (!per[m]) {
    switch (m) {
      case 2: per[m] = gather_slots_m<2>(); break;
      case 4: per[m] = gather_slots_m<4>(); break;
      case 6: per[m] = gather_slots_m<6>(); break;
      default: per[m] = gather_slots_m<3>(); break;
    }
  }
  return per[m] * device_sms();
}

uotk_status nfft_spread(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& S,
                        const SpreadWeights& w, NfftWork& W, float* grid_out) {
  if (S.n == 0) {
    const long long total = (long long)P.n * P.n * P.n;
    UOTK_CUDA(ctx, cudaMemsetAsync(grid_out, 0, sizeof(float) * total, s));
    return UOTK_OK;
  }
  UOTK_TRY(nfft_points_windows(ctx, s, P, S, true));
  // Gaussian kernel: the spread forms the weights as its chunks land (the
  // non-smooth kernels' near field reads them from W.wts)
  if (w.pot && P.kernel == UOTK_KERNEL_GAUSS)
    return spread_units(ctx, s, P, S, nullptr, &w, W, grid_out);
  const float* wts = w.base;
  if (w.pot) {
    UOTK_PROF(ctx, s, "weights");
    k_point_weights<<<grid_for(ctx, S.n + 4, 256, 4), 256, 0, s>>>(w.base, w.pot, w.lam,
                                                                   w.shift_slot, S.n, W.wts);
    UOTK_LAUNCHED(ctx);
    wts = W.wts;
  }
  return spread_units(ctx, s, P, S, wts, nullptr, W, grid_out);
}

uotk_status nfft_convolve(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, NfftWork& W,
                          const float* grid_in, float* grid_out) {
  const int n = P.n, N = P.N;
  const float* full = P.kernel != UOTK_KERNEL_GAUSS ? W.full : nullptr;
  int logn = 0;
  while ((1 << logn) < n) ++logn;
  UOTK_PROF(ctx, s, "fft");
  if (!full && n == 128) {
    // Gaussian: three separable circulant passes, in place on the output grid
    if (grid_out != grid_in)
      UOTK_CUDA(ctx, cudaMemcpyAsync(grid_out, grid_in, sizeof(float) * (size_t)n * n * n,
                                     cudaMemcpyDeviceToDevice, s));
    return circ_convolve(ctx, s, N, W.scale, grid_out);
  }
  if (n >= 32 && N % WF_LINES == 0) {
    // pruned warp-FFT passes: A1 = n x n x N, A2 = n x N x N complex inside cgrid
    float2* A1 = W.cgrid;
    float2* A2 = W.cgrid + (size_t)n * n * N;
    switch (n) {
      case 32: return wfft_convolve<1>(ctx, s, N, W.scale, full, grid_in, A1, A2, grid_out);
      case 64: return wfft_convolve<2>(ctx, s, N, W.scale, full, grid_in, A1, A2, grid_out);
      case 128: return wfft_convolve<4>(ctx, s, N, W.scale, full, grid_in, A1, A2, grid_out);
      case 256: return wfft_convolve<8>(ctx, s, N, W.scale, full, grid_in, A1, A2, grid_out);
      default: break;
    }
  }
  const int blocks = n * n / FFT_LINES;
  const size_t smem = sizeof(float2) * (n / 2 + FFT_LINES * n);
  // forward x (real -> complex), forward y, z (forward, scale, inverse), inverse y, inverse x
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(grid_in, nullptr, nullptr, W.cgrid, n, logn, 0, 0,
                                               -1, nullptr, N, nullptr);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 1, 1,
                                               -1, nullptr, N, nullptr);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 2, 3,
                                               -1, W.scale, N, full);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, nullptr, W.cgrid, n, logn, 1, 1,
                                               +1, nullptr, N, nullptr);
  UOTK_LAUNCHED(ctx);
  k_fft_pass<<<blocks, FFT_THREADS, smem, s>>>(nullptr, W.cgrid, grid_out, nullptr, n, logn, 0, 2,
                                               +1, nullptr, N, nullptr);
  UOTK_LAUNCHED(ctx);
  return UOTK_OK;
}

uotk_status nfft_gather(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& S,
                        const float* grid, float* out_sorted, const DualUpdate* du) {
  if (S.n == 0) return UOTK_OK;
  UOTK_TRY(nfft_points_windows(ctx, s, P, S, false));
  UOTK_PROF(ctx, s, "gather");
  return gather_units(ctx, s, P, S, grid, out_sorted, du);
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
  // one E^3 block per spread work unit, folded into the grid in a fixed order
  const int E = NFFT_TILE + 2 * P.m - 1;
  W.blocks = cv.take<float>((size_t)nfft_max_units(P, max_points > 0 ? max_points : 1,
                                                   nfft_spread_slots(P.m)) *
                            (size_t)((E * E * E + 3) & ~3));
  // complex work grid: n^3 for the unpruned passes, n^2 N + n N^2 for the
  // pruned ones (A1 and A2)
  const size_t pr = (size_t)P.n * P.n * P.N + (size_t)P.n * P.N * P.N;
  W.cgrid = cv.take<float2>(pr > n3 ? pr : n3);
  W.scale = cv.take<float>(3 * P.N);
  W.full = P.kernel != UOTK_KERNEL_GAUSS ? cv.take<float>((size_t)P.N * P.N * P.N) : nullptr;
  if (P.kernel != UOTK_KERNEL_GAUSS) {
    // one item per (tile, chunk of NFFT_NEAR_CHUNK targets)
    const size_t tiles = (size_t)P.tiles1 * P.tiles1 * P.tiles1;
    W.near_items = cv.take<int2>(tiles + (size_t)(max_points > 0 ? max_points : 0) /
                                              NFFT_NEAR_CHUNK + 1);
    W.near_ctr = cv.take<int>(2);
  } else {
    W.near_items = nullptr;
    W.near_ctr = nullptr;
  }
}

}  // namespace uotk
