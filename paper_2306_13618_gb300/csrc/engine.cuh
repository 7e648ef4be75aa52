// Summation engines: one kernel summation per Sinkhorn half-step, behind one
// interface so the sweep loop of Alg. 1 (direct) and Alg. 2 (NFFT) is shared.
#pragma once

#include "uotk_internal.cuh"

namespace uotk {

// Two point clouds X (n points) and Y (m points) prepared once per solve.
// Internal order: the engine may permute points (NFFT sorts by grid tile); the
// solver works on internal-order arrays and the engine maps them back.
struct Engine {
  virtual ~Engine() {}
  // t_X[i] = sum_j exp(-||x_i - y_j||^2/eps) * wY_j,  wY_j = baseY_j * exp(lam*potY_j - shift)
  // (side = 0), or the same with X and Y exchanged (side = 1).  base may be
  // NULL (weight 1).  shift is read on the device from an ordered-int64 slot.
  // All arrays are in internal order.
  virtual uotk_status half(cudaStream_t s, int side, const float* base, const double* pot,
                           double lam, const long long* shift_slot, float* out) = 0;
  // half() followed by the dual half-step `du` of its targets, fused into the
  // summation's last kernel; only called when fuses_dual() is true (otherwise
  // the solver runs half() and its own dual-update kernel).
  virtual bool fuses_dual() const { return false; }
  virtual uotk_status half_dual(cudaStream_t s, int side, const float* base, const double* pot,
                                double lam, const long long* shift_slot, float* out,
                                const DualUpdate& du) {
    (void)s; (void)side; (void)base; (void)pot; (void)lam; (void)shift_slot; (void)out; (void)du;
    return UOTK_ERR_UNSUPPORTED;
  }
  // Log-domain half step (the direct FP32 form only): out[i] = {M_i, S_i} with
  //   log t_i = ln2 (M_i + log2 S_i) + shift,
  // t_i the sum of half() (same base, pot, lam and shift slot), evaluated as a
  // per-row log-sum-exp so that no weight or kernel value has to be
  // representable in FP32.
  virtual uotk_status half_log(cudaStream_t s, int side, const float* base, const double* pot,
                               double lam, const long long* shift_slot, float2* out) {
    (void)s; (void)side; (void)base; (void)pot; (void)lam; (void)shift_slot; (void)out;
    return UOTK_ERR_UNSUPPORTED;
  }
  // Plain kernel sum with given internal-order weights w of the source side
  // (w = weights(src) for the caller's weights; any sign, n + 4 entries with
  // the last 4 zero): t = K(src -> tgt) w.
  // src/tgt: 0 = X, 1 = Y.
  virtual uotk_status plain(cudaStream_t s, int src, int tgt, const float* w, float* out) = 0;
  // nrhs sums over the same pairs src -> tgt (0 = X, 1 = Y): out[k] = the sum
  // of plain() with weights base[k] (pot == NULL), or of half() with weights
  // base[k]_j exp(lam pot_j - shift) (pot != NULL; then src != tgt).  The
  // default issues them one by one; an engine may share the kernel values.
  virtual uotk_status sums_multi(cudaStream_t s, int src, int tgt, int nrhs,
                                 const float* const* base, const double* pot, double lam,
                                 const long long* shift_slot, float* const* out) {
    for (int k = 0; k < nrhs; ++k) {
      if (pot) {
        if (src == tgt) return UOTK_ERR_INTERNAL;
        UOTK_TRY(half(s, tgt == 0 ? 0 : 1, base[k], pot, lam, shift_slot, out[k]));
      } else {
        UOTK_TRY(plain(s, src, tgt, base[k], out[k]));
      }
    }
    return UOTK_OK;
  }
  // Internal position -> caller index of `side` (NULL: identity).
  virtual const int* perm(int side) const = 0;
  // Internal-order copies of the caller's weights (may alias the inputs).
  virtual const float* weights(int side) const = 0;
  // Scatter an internal-order FP64 array of `side` back to caller order.
  virtual uotk_status to_caller(cudaStream_t s, int side, const double* in, double* out) = 0;
  // Scatter an internal-order FP32 array of `side` back to caller order.
  virtual uotk_status to_caller_f32(cudaStream_t s, int side, const float* in, float* out) = 0;
  // Gather a caller-order FP64 array into internal order.
  virtual uotk_status from_caller(cudaStream_t s, int side, const double* in, double* out) = 0;
  // True if internal order == caller order (no copies needed).
  virtual bool identity_order() const = 0;
};

// Workspace sizing and construction.  `ws_bytes` is called with base == null
// first (Carver size pass), then for real.
struct EngineSpec {
  int method;        // uotk_method
  int d;
  const float* x; int64_t n; const float* a;
  const float* y; int64_t m; const float* b;
  double eps;
  const uotk_sum_opts* opts;
};

size_t engine_bytes(uotk_ctx* ctx, const EngineSpec& sp);
// Build (pack/sort/plan) in workspace carved from cv.  Returns the engine
// through *out (heap object owned by the caller).
uotk_status engine_create(uotk_ctx* ctx, cudaStream_t s, const EngineSpec& sp, Carver& cv,
                          Engine** out);

// Tensor-core direct engine (ksum_tc.cu): methods UOTK_DIRECT_BF16, UOTK_DIRECT_BF16X3.
size_t tc_engine_bytes(uotk_ctx* ctx, const EngineSpec& sp);
uotk_status tc_engine_create(uotk_ctx* ctx, cudaStream_t s, const EngineSpec& sp, Carver& cv,
                             Engine** out);

// NFFT engine (nfft.cu).
size_t nfft_engine_bytes(uotk_ctx* ctx, const EngineSpec& sp);
uotk_status nfft_engine_create(uotk_ctx* ctx, cudaStream_t s, const EngineSpec& sp, Carver& cv,
                               Engine** out);

// Reset the device flag slots (counters to 0, maxima to -inf).
uotk_status flags_reset(uotk_ctx* ctx, cudaStream_t s);
// Read counters; returns INVALID/NONFINITE/TIMEOUT as recorded (synchronises).
uotk_status flags_check(uotk_ctx* ctx, cudaStream_t s, const char* what);

}  // namespace uotk
