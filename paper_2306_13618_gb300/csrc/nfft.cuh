// NFFT fast summation (Sec. 4, Eq. 1724) for the Gaussian kernel: shared
// declarations of the plan, the binned point sets and the stage kernels.
//
// Torus coordinates (Eq. boundaries, translated by 1/2): u = (p - c)/h + 1/2,
// grid node l at u = l/n.  In grid units t = u*n the point sits in cell
// floor(t) with fraction delta = t - floor(t), and the window touches the 2m
// nodes floor(t) - m + 1 + k, k = 0..2m-1, at distance v = delta + m - 1 - k.
// Grids are n^3 FP32, layout [z][y][x]; d < 3 is embedded in 3-D with the
// missing coordinates at the centre (their 1-D kernel factor is the constant 1).
#pragma once

#include "engine.cuh"

namespace uotk {

constexpr int NFFT_TILE = 8;           // grid cells per tile edge (work-unit granularity)
// Work split.  Clustered clouds fill few tiles (the 2^20-point mixture
// workload: 83 of 4096, one of them with a quarter of the points), so work is
// not cut by tile.  Every point costs 1, every occupied cell and every
// occupied tile a fixed cost (a cell's run of points ends in a flush or a
// footprint load, a tile's block is staged and written once per piece), in
// points; the sorted points, each cell's and tile's cost before its first
// point, are cut into chunks of equal cost Q, one chunk per CTA that the GPU
// holds at once, and a chunk is cut further where a tile ends.  These pieces
// are the work units: a piece lies in one tile (its CTA stages that tile's
// block) and a CTA takes the pieces of its chunk in turn.  Q is at least the
// minimum.
constexpr int NFFT_SPREAD_TILE_COST = 64;
constexpr int NFFT_GATHER_TILE_COST = 128;
constexpr int NFFT_SPREAD_CELL_COST = 8;
constexpr int NFFT_GATHER_CELL_COST = 8;
constexpr int NFFT_SPREAD_MIN_CHUNK = 64;
constexpr int NFFT_GATHER_MIN_CHUNK = 256;
constexpr int NFFT_MAX_M = 8;
constexpr int NFFT_CHUNK = 64;          // default points per bulk-copied staging chunk
constexpr int NFFT_NEAR_CHUNK = 1024;   // targets per near-field work item
// Window table row of one point (floats): phi_x split in two halves of m
// values, then phi_y (2m), then phi_z (2m); every block padded to a 16-byte
// multiple, so that every chunk of the table is a legal bulk-copy source and
// each half of phi_x and all of phi_z are 16-byte vector loads.
__host__ __device__ constexpr int nfft_win_half(int m) { return (m + 3) & ~3; }
__host__ __device__ constexpr int nfft_win_yoff(int m) { return 2 * nfft_win_half(m); }
__host__ __device__ constexpr int nfft_win_zoff(int m) {
  return 2 * nfft_win_half(m) + ((2 * m + 3) & ~3);
}
__host__ __device__ constexpr int nfft_win_stride(int m) {
  return nfft_win_zoff(m) + ((2 * m + 3) & ~3);
}
// Offset in the row of phi_x[kx], kx in [0, 2m).
__host__ __device__ constexpr int nfft_win_xoff(int m, int kx) {
  return kx < m ? kx : nfft_win_half(m) + kx - m;
}
// Pair window table (the spread's): sorted points 2p and 2p + 1 share row p,
// every window value stored as the pair (value of 2p, value of 2p + 1): the two
// halves of phi_x (m pairs each, padded to a 16-byte multiple), phi_y (2m
// pairs), phi_z (2m pairs).  Packed FP32x2 FMAs then run over point pairs.
__host__ __device__ constexpr int nfft_winp_half(int m) { return (2 * m + 3) & ~3; }
__host__ __device__ constexpr int nfft_winp_yoff(int m) { return 2 * nfft_winp_half(m); }
__host__ __device__ constexpr int nfft_winp_zoff(int m) { return nfft_winp_yoff(m) + 4 * m; }
__host__ __device__ constexpr int nfft_winp_stride(int m) { return nfft_winp_zoff(m) + 4 * m; }

struct NfftParams {
  int d = 3;
  int n = 128;         // oversampled grid
  int N = 64;          // bandwidth
  int m = 6;           // window cut-off
  float c[3] = {0, 0, 0};
  float inv_h = 1.f;
  double h = 1.0;
  double eps = 1.0;
  float b = 0.f;       // Kaiser-Bessel shape pi (2 - 1/sigma)
  int tiles1 = 16;     // tiles per dimension = n / NFFT_TILE
  int E = 19;          // smem block edge = NFFT_TILE + 2m - 1
  // Non-smooth kernels (Sec. 4.2): uotk_kernel, regularisation degree p (the
  // pieces match p derivatives) and eps_I = eps_B (torus units); eps above is
  // then the kernel's parameter.  kernel == UOTK_KERNEL_GAUSS: unused.
  int kernel = 0;
  int reg_p = 0;
  double eps_i = 0.0;
  double reg_target = 1e-3;   // bound the plan's self-check enforces (error per unit weight)
};

// Host: choose h, m; fill params (bounding box given).
uotk_status nfft_make_params(uotk_ctx* ctx, int d, const float lo[3], const float hi[3], double eps,
                             const uotk_sum_opts* opts, NfftParams* P);
// Host: 1-D factors g(k) of scale_k = prod_t g_t(k_t), k in {-N/2..N/2-1}
// (FP64 -> FP32 table of 3*N floats, one row per dimension).
void nfft_scale_table(const NfftParams& P, float* host_table /* 3*N */);
// Host: the deconvolution rows 1/(n phihat(k))^2 (FP64, 3*N; an embedded
// dimension keeps k = 0 only).
void nfft_deconv_rows(const NfftParams& P, double* rows /* 3*N */);

// A point set sorted by grid cell, cells ordered tile by tile (tile-major,
// then z, y, x inside the tile): points of one cell are contiguous.
struct NfftPoints {
  int64_t n = 0;
  int4* cell = nullptr;      // sorted: (cx | cy<<10 | cz<<20, frac x, y, z as float bits)
  float* win = nullptr;      // sorted: [n][nfft_win_stride(m)] window rows (layout above)
  int* ckey = nullptr;       // sorted: packed cell (cx | cy<<10 | cz<<20), n + 4 entries
  float* winp = nullptr;     // [ceil(n/2)][nfft_winp_stride(m)] pair window rows (spread)
  // the window tables are built on first use (nfft_points_windows): a cloud that
  // is only spread, or only gathered at, never builds the other one
  mutable bool win_ready = false, winp_ready = false;
  int* perm = nullptr;       // sorted position -> caller index
  int* tile_start = nullptr; // [tiles+1] start of each tile in sorted order
  int* tile_rank = nullptr;  // [tiles+1] occupied tiles before each tile
  int* cell_rank = nullptr;  // [n^3+1] occupied cells before each cell (tile-major order)
  long long* chunk_q = nullptr;  // [2] cost per chunk: spread, gather
  // spread work units (pieces of the c_spread chunks, each in one tile)
  int* unit_tile = nullptr;  // [max_units] tile of each work unit
  int* unit_begin = nullptr; // [max_units] first sorted point of the unit
  int* unit_count = nullptr; // [max_units]
  int* unit_box = nullptr;   // [max_units] box of the unit's local cells, written by the
                             // spread: 4-bit fields zlo, zhi, ylo, yhi, xlo, xhi (bits 0..23)
  int* num_units = nullptr;  // [1] device count
  int* tile_unit_start = nullptr;  // [tiles+1] first unit of each tile
  int* unit_chunk = nullptr;       // [max_units] chunk of each unit
  int* chunk_unit_start = nullptr; // [c_spread+1] first unit of each chunk
  int max_units = 0;
  int c_spread = 0;                // chunks (CTAs of the spread)
  // gather work units (pieces of the c_gather chunks, each in one tile)
  int* g_unit_tile = nullptr;
  int* g_unit_begin = nullptr;
  int* g_unit_count = nullptr;
  int* g_num_units = nullptr;
  int* g_tile_unit_start = nullptr;
  int* g_unit_chunk = nullptr;
  int* g_chunk_unit_start = nullptr;
  int g_max_units = 0;
  int c_gather = 0;
  int* scratch = nullptr;    // [tiles] counters
  int* cell_count = nullptr; // [n^3] histogram, then 0/1 occupied flags
  int* cell_start = nullptr; // [n^3 + 1] exclusive scan
  int* block_sums = nullptr; // scan partials
  // stable radix sort of the cell keys (deterministic order inside a cell)
  int* rs_key[2] = {nullptr, nullptr};  // [n] keys, ping-pong
  int* rs_val[2] = {nullptr, nullptr};  // [n] caller indices, ping-pong
  int* rs_hist = nullptr;     // [256 * blocks + 1] digit counts, then their scan
  int* rs_start = nullptr;    // [256 * blocks + 1]
  int* rs_bsum = nullptr;     // scan partials
  int4* tmp_cell = nullptr;   // [n] caller order: packed cell and fractions
};
size_t nfft_points_bytes(const NfftParams& P, int64_t n);
void nfft_points_carve(Carver& cv, const NfftParams& P, int64_t n, NfftPoints& S);
// Bin, sort and precompute windows for caller-order points (n x d FP32).
uotk_status nfft_points_build(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                              const float* pts, int64_t n, NfftPoints& S);

// Work buffers of one summation.
struct NfftWork {
  float* wts = nullptr;    // [max points + 4] spread weights (sorted order)
  float* grid = nullptr;   // [n^3] real grid
  float* blocks = nullptr; // [max units][E^3 rounded to 4] spread blocks, one per work unit
  float2* cgrid = nullptr; // [n^3] complex work grid
  float* scale = nullptr;  // [3*N] device table
  float* full = nullptr;   // [N^3] non-separable table [kz'][ky'][kx'] (non-smooth kernels)
  int2* near_items = nullptr;  // near-field work items (target tile, first target)
  int* near_ctr = nullptr;     // [2] item count, next item to take
};
size_t nfft_work_bytes(const NfftParams& P, int64_t max_points);
void nfft_work_carve(Carver& cv, const NfftParams& P, int64_t max_points, NfftWork& W);

// Weights of the spread: w_i = base_i * exp(lam*pot_i - shift) (sorted order),
// or plain w_i = base_i when pot == NULL (base then needs n + 4 entries).
struct SpreadWeights {
  const float* base = nullptr;
  const double* pot = nullptr;
  double lam = 0.0;
  const long long* shift_slot = nullptr;
};

uotk_status nfft_spread(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& S,
                        const SpreadWeights& w, NfftWork& W, float* grid_out);
uotk_status nfft_convolve(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, NfftWork& W,
                          const float* grid_in, float* grid_out);
// du != NULL: the dual half-step of each target follows its sum in the same
// kernel (t still written to out_sorted).
uotk_status nfft_gather(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& S,
                        const float* grid, float* out_sorted, const DualUpdate* du = nullptr);

// Non-smooth kernels (nfft_reg.cu): fill W.full with b_k / prod_t (n phihat(k_t))^2,
// b_k the DFT of the regularised kernel K_R sampled on I_N^d (FP64 on the
// device, W.cgrid as scratch); and add the near-field correction
// sum_{|x_i - y_j| < eps_I h} w_j (K - K_R) to out (target order).
uotk_status nfft_reg_table(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, NfftWork& W);
uotk_status nfft_near(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P, const NfftPoints& src,
                      const float* w, const NfftPoints& tgt, NfftWork& W, float* out);

// Bounding box of point clouds on the device -> host (synchronises).
uotk_status nfft_bbox(uotk_ctx* ctx, cudaStream_t s, int d, const float* a, int64_t na,
                      const float* b, int64_t nb, float lo[3], float hi[3]);

// Upper bound of the work units of n points cut into `chunks` chunks.
int nfft_max_units(const NfftParams& P, int64_t n, int chunks);
// Build the gather's window table (pair = false) or the spread's pair table
// (pair = true) of a binned cloud unless it is built already.
uotk_status nfft_points_windows(uotk_ctx* ctx, cudaStream_t s, const NfftParams& P,
                                const NfftPoints& S, bool pair);
// Chunks of the spread and of the gather at cut-off m: the CTAs of the kernel
// that the device holds at once.
int nfft_spread_slots(int m);
int nfft_gather_slots(int m);

}  // namespace uotk
