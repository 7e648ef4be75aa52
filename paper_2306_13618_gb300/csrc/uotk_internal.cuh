// Internal declarations of the uotk CUDA library (sm_103a).  Not installed.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "../../include/uotk.h"

// ---------------------------------------------------------------------------
// Context: device, workspace arena, pinned host staging, error text.
// ---------------------------------------------------------------------------
constexpr int UOTK_PROF_POOL = 1024;   // event pairs in flight before a fold
constexpr int UOTK_PROF_STAGES = 32;
struct uotk_prof {
  bool on = false;
  int nstages = 0;
  char names[UOTK_PROF_STAGES][24] = {};
  long long counts[UOTK_PROF_STAGES] = {};
  double ms[UOTK_PROF_STAGES] = {};
  cudaEvent_t ev[2 * UOTK_PROF_POOL] = {};
  int stage_of[UOTK_PROF_POOL] = {};
  int pending = 0;
  bool created = false;
};

// One autotuned summation form (see op_autotune_sum), keyed by the problem.
constexpr int UOTK_AUTO_CACHE = 8;
struct AutoEntry {
  bool valid = false;
  int d = 0;
  int64_t n = 0, m = 0;
  double eps = 0.0, target = 0.0;
  int grid_in = 0, cutoff_in = 0;
  bool per_sum = false;  // timed per sum on a built plan (see op_autotune_sum)
  float box[6] = {0, 0, 0, 0, 0, 0};
  uotk_sum_opts chosen = {};
  double report[8] = {0, 0, 0, 0, 0, 0, 0, 0};
};

struct uotk_ctx {
  int device = 0;
  int num_sms = 0;
  int max_smem_optin = 0;
  char err[512] = {0};
  // Device workspace: one allocation, carved per call.
  char* ws = nullptr;
  size_t ws_cap = 0;
  size_t ws_limit = 0;        // largest workspace allowed (0: none)
  long long wait_test = 0;    // > 0: first wait per CTA runs out after this many cycles
  // Pinned host staging for scalars read back at the end of a call.
  double* host = nullptr;   // 128 doubles
  // Device flags/counters (int64 slots), zeroed per call where used.
  long long* dflags = nullptr;  // NUM_FLAGS slots
  int64_t launches = 0;
  uotk_prof prof;
  // The context's own stream for captured loops (a caller's legacy default
  // stream cannot be captured), fenced to the caller's stream with events.
  cudaStream_t gs = nullptr;
  cudaEvent_t fence_in = nullptr, fence_out = nullptr;
  // autotuned forms, most recent first out
  AutoEntry autos[UOTK_AUTO_CACHE];
  int auto_next = 0;
  std::vector<int> batch_forms;  // form of every pair of the last batched solve (uotk_method)
};

namespace uotk {

// Flag slots in ctx->dflags.
enum FlagSlot {
  FLAG_NEG_WEIGHT = 0,     // count of negative weights
  FLAG_NONFINITE = 1,      // count of non-finite weights/coordinates
  FLAG_TIMEOUT = 2,        // a bounded device wait gave up
  FLAG_INTERNAL = 3,       // an internal bound check failed
  FLAG_MAX_G0 = 4,         // ordered-int64 maxima of lambda*gamma (two parities)
  FLAG_MAX_G1 = 5,
  FLAG_MAX_B0 = 6,         // ordered-int64 maxima of lambda*beta (two parities)
  FLAG_MAX_B1 = 7,
  FLAG_DELTA0 = 8,         // max |lambda * change| over a sweep (two parities)
  FLAG_DELTA1 = 9,
  FLAG_NONFINITE_DUAL = 10,  // count of non-finite dual values produced
  FLAG_WAIT_TEST = 11,     // > 0: the first wait per CTA runs out (uotk_set_wait_timeout_test)
  FLAG_BBOX = 16,          // 6 slots: max x,y,z and max of -x,-y,-z (ordered encodings)
  NUM_FLAGS = 32
};

uotk_status set_error(uotk_ctx* ctx, uotk_status st, const char* fmt, ...);

// The fastest summation form within in->target_err for the sum src -> tgt
// (autotune.cu; uotk_autotune_sum).
uotk_status op_autotune_sum(uotk_ctx* ctx, cudaStream_t s, int d, const float* src, int64_t n,
                            const float* w, const float* tgt, int64_t m, double eps,
                            const uotk_sum_opts* in, uotk_sum_opts* out, double* report,
                            bool per_sum = false);

// One dual half-step of Alg. 1 / Alg. 2 on the targets of a kernel sum t:
//   pot_i <- -q (log t_i + shift)                 (ref 0)
//   pot_i <- q (log base_i - log t_i - shift)     (ref 1),
// shift read from flags[shift_in]; max lam*pot -> flags[max_out] (ordered
// int64); when delta_out >= 0 also max lam*|change| -> flags[delta_out]; the
// slots reset_slot / reset_delta (>= 0) are set to -inf for the next half-step;
// non-finite results counted in FLAG_NONFINITE_DUAL.  Internal point order.
struct DualUpdate {
  const float* base;  // ref 1: weights of the targets; unused for ref 0
  double* pot;        // the targets' dual potential, read (delta) and written
  double q, lam;
  int ref, shift_in, max_out, reset_slot, delta_out, reset_delta;
};

// Order work: everything enqueued on `from` so far runs before what is
// enqueued on `to` next (an event recorded on `from`, waited for on `to`).
uotk_status stream_fence(uotk_ctx* ctx, cudaStream_t from, cudaStream_t to, cudaEvent_t ev);

// Grow the workspace to `bytes` (synchronises the device when it reallocates).
uotk_status ws_reserve(uotk_ctx* ctx, size_t bytes);

// Sub-allocation from the workspace.  Usage: first pass computes the size with
// a null base; second pass hands out pointers.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(char* b) : base(b) {}
  template <class T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

#define UOTK_CUDA(ctx, call)                                                    \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return uotk::set_error((ctx), UOTK_ERR_CUDA, "%s failed: %s (%s:%d)",     \
                             #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

#define UOTK_LAUNCHED(ctx)                                                      \
  do {                                                                          \
    cudaError_t e_ = cudaGetLastError();                                        \
    if (e_ != cudaSuccess)                                                      \
      return uotk::set_error((ctx), UOTK_ERR_CUDA, "kernel launch failed: %s (%s:%d)", \
                             cudaGetErrorString(e_), __FILE__, __LINE__);       \
    (ctx)->launches++;                                                          \
  } while (0)

// Per-stage CUDA-event timing of the launch that follows in the same scope.
int prof_begin(uotk_ctx* ctx, cudaStream_t s, const char* name);
void prof_end(uotk_ctx* ctx, cudaStream_t s, int slot);
struct ProfScope {
  uotk_ctx* ctx;
  cudaStream_t s;
  int slot;
  ProfScope(uotk_ctx* c, cudaStream_t st, const char* name)
      : ctx(c), s(st), slot(c->prof.on ? prof_begin(c, st, name) : -1) {}
  ~ProfScope() {
    if (slot >= 0) prof_end(ctx, s, slot);
  }
};
#define UOTK_PROF(ctx, s, name) uotk::ProfScope uotk_prof_scope_((ctx), (s), (name))

// Opt a kernel in to `bytes` of dynamic shared memory.  Skipped while the
// stream is being captured into a graph: the attribute was set by the eager
// launch that precedes every capture.
template <class K>
inline cudaError_t smem_attr(cudaStream_t s, K kernel, size_t bytes) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone)
    return cudaSuccess;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

#define UOTK_TRY(expr)                 \
  do {                                 \
    uotk_status s_ = (expr);           \
    if (s_ != UOTK_OK) return s_;      \
  } while (0)

// ---------------------------------------------------------------------------
// Device helpers.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// exp(a) for an FP64 argument, returned in FP32: a = k ln2 + r with integer k
// and |r| <= ln2/2 taken in FP64, expf(r) in FP32, scaled by 2^k.  The result
// has FP32 relative accuracy whatever |a| (converting a itself to FP32 would
// cost |a| ulps).  Underflows to 0 below 2^-149.
// k is taken in FP32 (an off-by-one k next to a half-integer only widens the
// range of r a little) and r = a - k ln2 in one FP64 FMA: ln2's FP64 rounding
// costs |k| 2^-53 < 1e-14 for |k| <= 160, far below FP32 resolution.
__device__ __forceinline__ float exp_shifted(double a) {
  const float k = rintf((float)a * 1.44269504f);
  if (k < -160.f) return 0.f;
  const float r = (float)fma(-(double)k, 0.6931471805599453, a);
  return ldexpf(expf(r), (int)k);
}

// log(t) of a positive FP32 value in FP64: t = f 2^e with f in [0.5, 1),
// log f in FP32 (absolute error < 1e-7), e ln2 in FP64.
__device__ __forceinline__ double log_f32(float t) {
  int e;
  const float f = frexpf(t, &e);
  return (double)logf(f) + (double)e * 0.6931471805599453;
}

// Packed two-wide FP32 arithmetic (one instruction for two lanes of values).
__device__ __forceinline__ unsigned long long f2_pack(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ unsigned long long f2_sub(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_mul(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long f2_add(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

// ---- shared-memory mbarriers and 1-D bulk copies (TMA, cp.async.bulk) ----
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
// global -> shared copy of `bytes` (multiple of 16, both addresses 16-byte
// aligned) completing on `bar`.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
// Bounded wait for phase `parity` of `bar`: gives up after `limit` clocks
// (default ~2^31, about a second).
constexpr long long UOTK_WAIT_CYCLES = 1LL << 31;
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity,
                                          long long limit = UOTK_WAIT_CYCLES) {
  const unsigned a = smem_addr(bar);
  const long long t0 = clock64();
  while (true) {
    unsigned done;
    asm volatile(
        "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}
// The first bounded wait of a CTA, on phase `parity` of `bar`.  With the
// context's time-out test on (flags[FLAG_WAIT_TEST] = cycles > 0) it waits
// instead on `never`, a barrier nothing arrives at, and runs out after that
// many cycles.
__device__ __forceinline__ bool first_wait(unsigned long long* bar, unsigned parity,
                                           unsigned long long* never, const long long* flags) {
  const long long test = flags[FLAG_WAIT_TEST];
  if (test > 0) return mbar_wait(never, 0u, test);
  return mbar_wait(bar, parity);
}

// Order-preserving map of doubles onto signed 64-bit integers, so that the
// maximum of doubles can be taken with integer atomicMax (deterministic).
__device__ __host__ __forceinline__ long long dbl_to_ordered(double v) {
  long long b;
  memcpy(&b, &v, 8);
  return b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
}
__device__ __host__ __forceinline__ double ordered_to_dbl(long long b) {
  long long r = b >= 0 ? b : (b ^ 0x7fffffffffffffffLL);
  double v;
  memcpy(&v, &r, 8);
  return v;
}
static const long long ORDERED_NEG_INF = (long long)0x800fffffffffffffULL;  // encodes -inf

__device__ __forceinline__ void flag_add(long long* p, long long v) {
  atomicAdd(reinterpret_cast<unsigned long long*>(p), static_cast<unsigned long long>(v));
}

template <class T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int warp_min_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
__device__ __forceinline__ int warp_max_i(int v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// ---------------------------------------------------------------------------
// Direct kernel summation (ksum_direct.cu).
// ---------------------------------------------------------------------------
struct DirectLayout {
  int d = 0;
  int64_t n = 0, m = 0;
  int reg_targets = 1;   // targets per thread
  int blocks_x = 0;      // target blocks
  int splits = 1;        // source splits (partial sums reduced in FP64)
  int64_t tiles = 0;     // source tiles of TILE points
  int tiles_per_split = 0;
  int dp = 4;            // floats per packed point (general-d path)
  size_t src_bytes = 0, tgt_bytes = 0, part_bytes = 0;
};
constexpr int DIRECT_TILE = 256;
constexpr int DIRECT_THREADS = 256;

// force_r > 0 fixes the targets per thread (d <= 3 kernels).
DirectLayout direct_layout(const uotk_ctx* ctx, int d, int64_t n, int64_t m, int force_r = 0);

// K <= 4 Gaussian sums over the same pairs (d <= 3): out[k][j] = sum_i w_k[i]
// exp(-|s_i - t_j|^2 / eps), w_k[i] = w[k][i] (pot == NULL) or
// w[k][i] exp(lam pot_i - shift) (shift from *shift_slot), from packed source
// positions and targets (the layouts of direct_pack_sources /
// direct_pack_targets); scratch of direct_multi_bytes(ctx, d, n, m) bytes.
size_t direct_multi_bytes(const uotk_ctx* ctx, int d, int64_t n, int64_t m);
uotk_status direct_run_multi(uotk_ctx* ctx, cudaStream_t s, int d, int64_t n, int64_t m,
                             const void* src_packed, const void* tgt_packed, int K,
                             const float* const* w, const double* pot, double lam,
                             const long long* shift_slot, void* scratch, double eps,
                             float* const* out);

// Buffers of one direct summation.
struct DirectBufs {
  void* src = nullptr;    // packed sources (float4 for d<=3, float[dp] otherwise)
  void* tgt = nullptr;    // packed targets
  float* part = nullptr;  // [splits][m] partial sums (splits > 1)
};
void direct_carve(Carver& cv, const DirectLayout& L, DirectBufs& b);

// Pack raw row-major FP32 points (sources with weights / targets without).
// Weight validation counters go to ctx->dflags.
uotk_status direct_pack_sources(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                                const float* pts, const float* w, void* packed);
uotk_status direct_pack_targets(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                                const float* pts, void* packed);
// Rewrite only the weights of packed sources: w_i = base_i * exp(lam*pot_i - shift),
// shift read from the ordered-int64 slot *shift_slot (base may be NULL for 1);
// with pot == NULL, w_i = base_i.
// log2_weights: store log2(w_i) instead (the log-domain form; padding -inf).
uotk_status direct_set_weights(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                               void* packed, const float* base, const double* pot,
                               double lam, const long long* shift_slot,
                               bool log2_weights = false);
// out[j] = sum_i w_i exp(-||s_i - t_j||^2 / eps) from packed buffers.
// kernel: uotk_kernel (Table tab:0); eps is then the kernel's parameter p.
uotk_status direct_run(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                       const DirectBufs& b, double eps, float* out, int kernel = 0);
// Log domain (sources packed with log2 weights): out[j] = {M_j, S_j} with
// log2 sum_i w_i exp(-||s_i - t_j||^2 / eps) = M_j + log2 S_j.  b.part must
// hold splits * m float2 when L.splits > 1.
uotk_status direct_run_lse(uotk_ctx* ctx, cudaStream_t s, const DirectLayout& L,
                           const DirectBufs& b, double eps, float2* out);

int grid_for(const uotk_ctx* ctx, int64_t work, int threads, int per_sm = 8);

// cstar.cu: <mu (x) nu|d^r> (r = 1, 2; r = 1 through the energy kernel in the
// form `method`) with mu(X), nu(X) into out[0..3); c* of Eq. (561), the
// Eq. (W4) objective at c* mu (x) nu and the mean-cost numerator into
// out[0..3); v[0..count) = value.
uotk_status op_mean_cost(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                         const float* a, const float* y, int64_t m, const float* b, int r,
                         int method, double* out);
uotk_status op_cstar(uotk_ctx* ctx, cudaStream_t s, int d, const float* x, int64_t n,
                     const float* a, const float* y, int64_t m, const float* b, double eps,
                     double rho1, double rho2, int r, int method, double* out);
uotk_status fill_f64(uotk_ctx* ctx, cudaStream_t s, double* v, int64_t count, double value);

}  // namespace uotk
