// The Sinkhorn loop of Alg. 1 / Alg. 2 and its FP64 reductions, shared by the
// value operations (sinkhorn.cu) and their gradients (grad.cu).
#pragma once

#include "engine.cuh"

namespace uotk {

// Block partial sums of up to 5 FP64 terms; term k over [0, len_k):
//   kind 0: sum base_i * exp(-pot_i / eta)
//   kind 1: sum base_i
//   kind 2: sum base_i * t_i                     (t FP32)
//   kind 3: sum (base_i or 1) * exp(lam*pot_i + shift) * t_i
//   kind 4: sum (base_i or 1) * exp(lam*pot_i + shift + ln2 (M_i + log2 S_i)),
//           {M, S} = ms_i of the log-domain form
struct SumTerm {
  int kind;
  long long len;
  const float* base;
  const double* pot;
  const float* t;
  double eta, lam;
  int shift_slot;
  const float2* ms = nullptr;
};
struct SumTerms {
  SumTerm k[5];
  int count;
};

struct Reducer {
  double* part = nullptr;  // [5][blocks]
  double* out = nullptr;   // [5]
  int blocks = 0;
};

// Deterministic FP64 sums of T into host_out[0..T.count) (pinned; valid after
// the stream synchronises).
uotk_status run_sums(uotk_ctx* ctx, cudaStream_t s, const Reducer& R, const SumTerms& T,
                     double* host_out);
void carve_reducer(uotk_ctx* ctx, Carver& cv, Reducer& R);

// Internal-order work arrays of one solve.
struct SolveBufs {
  double* beta = nullptr;   // internal order (aliases caller's when identity order)
  double* gamma = nullptr;
  float* tx = nullptr;
  float* ty = nullptr;
  float2* lx = nullptr;     // log-domain half-step outputs {M, S}
  float2* ly = nullptr;
};
void carve_solve(Carver& cv, int64_t n, int64_t m, bool need_copies, SolveBufs& B,
                 bool log_domain = false);

struct SolveResult {
  int sweeps = 0;
  double value = 0.0;
  bool converged = false;
};

// Alg. 1 / Alg. 2 for up to max_sweeps sweeps on an engine, then the dual value
// D(beta, gamma) of Eq. (dual_euot).  On return (stream synchronised):
//   ctx->host[8 + 2], ctx->host[8 + 3] hold sum(a) and sum(b);
//   B.ty holds sum_i k_ij a_i e^{lambda beta_i - M_beta} at the final beta
//   (ref 0; without a_i for ref 1), M_beta = max lambda*beta in flag slot
//   FLAG_MAX_B0 + ((sweeps - 1) & 1), and M_gamma = max lambda*gamma at the
//   final gamma in FLAG_MAX_G0 + (sweeps & 1).
// log_domain: every half-step through Engine::half_log (per-row log-sum-exp;
// the direct FP32 form), the dual value's coupling term from its {M, S}.
uotk_status solve(uotk_ctx* ctx, cudaStream_t s, Engine* E, int64_t n, int64_t m, double eps,
                  double eta1, double eta2, int max_sweeps, double tol, int ref, bool warm,
                  const SolveBufs& B, const Reducer& R, SolveResult* res,
                  bool log_domain = false);

}  // namespace uotk
