// FP64 (DSNU_FP64) instantiation of the pipeline.
#include "pipeline.cuh"

namespace dsnu {
dsnu_status run_pipeline_f64(const PlanGeom& g, const PlanTables& t, const WsLayout& L,
                             const Members& mem, cudaStream_t st, int cj, cudaEvent_t* ev, const Overlap* ov) {
  return run_pipeline<double>(g, t, L, mem, st, cj, ev, ov);
}
cudaError_t prepare_kernels_f64(PlanGeom& g) { return prepare_kernels<double>(g); }
cudaError_t time_spread_f64(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws, int reps,
                            float* ms) {
  return time_spread<double>(g, t, L, ws, reps, ms);
}
}  // namespace dsnu
