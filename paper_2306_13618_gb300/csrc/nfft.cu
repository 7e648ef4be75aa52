// NFFT fast summation (Sec. 4): placeholder until the kernels land.
#include "engine.cuh"

namespace uotk {

size_t nfft_engine_bytes(uotk_ctx*, const EngineSpec&) { return 0; }
uotk_status nfft_engine_create(uotk_ctx* ctx, cudaStream_t, const EngineSpec&, Carver&, Engine**) {
  return set_error(ctx, UOTK_ERR_UNSUPPORTED, "NFFT path not built yet");
}
uotk_status op_nfft_plan(uotk_ctx* ctx, cudaStream_t, int, const float*, int64_t, const float*,
                         int64_t, double, const uotk_sum_opts*, uotk_nfft_plan_info*) {
  return set_error(ctx, UOTK_ERR_UNSUPPORTED, "NFFT path not built yet");
}
uotk_status op_nfft_cells(uotk_ctx* ctx, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                          int64_t, int32_t*) {
  return set_error(ctx, UOTK_ERR_UNSUPPORTED, "NFFT path not built yet");
}
uotk_status op_nfft_spread(uotk_ctx* ctx, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                           int64_t, const float*, float*) {
  return set_error(ctx, UOTK_ERR_UNSUPPORTED, "NFFT path not built yet");
}
uotk_status op_nfft_convolve(uotk_ctx* ctx, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                             float*) {
  return set_error(ctx, UOTK_ERR_UNSUPPORTED, "NFFT path not built yet");
}
uotk_status op_nfft_gather(uotk_ctx* ctx, cudaStream_t, const uotk_nfft_plan_info*, const float*,
                           const float*, int64_t, float*) {
  return set_error(ctx, UOTK_ERR_UNSUPPORTED, "NFFT path not built yet");
}

}  // namespace uotk
