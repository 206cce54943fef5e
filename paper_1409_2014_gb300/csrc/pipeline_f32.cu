// FP32 (DSNU_MIXED) instantiation of the pipeline.
#include "pipeline.cuh"

namespace dsnu {
dsnu_status run_pipeline_f32(const PlanGeom& g, const PlanTables& t, const WsLayout& L,
                             const Members& mem, cudaStream_t st, int cj, cudaEvent_t* ev, const Overlap* ov) {
  return run_pipeline<float>(g, t, L, mem, st, cj, ev, ov);
}
cudaError_t prepare_kernels_f32(PlanGeom& g) { return prepare_kernels<float>(g); }
cudaError_t time_spread_f32(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws, int reps,
                            float* ms) {
  return time_spread<float>(g, t, L, ws, reps, ms);
}
}  // namespace dsnu
