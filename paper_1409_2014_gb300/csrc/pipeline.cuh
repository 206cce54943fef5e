// pipeline.cuh -- launch sequence of one solve (included once per precision).
#pragma once

#include "internal.h"
#include "kernels.cuh"

namespace dsnu {

#define DSNU_LOG2_CASES(CALL) \
  case 4: CALL(4); break;     \
  case 5: CALL(5); break;     \
  case 6: CALL(6); break;     \
  case 7: CALL(7); break;     \
  case 8: CALL(8); break;     \
  case 9: CALL(9); break;     \
  case 10: CALL(10); break;   \
  case 11: CALL(11); break;   \
  case 12: CALL(12); break;

template <typename R, int L2>
cudaError_t set_fft_attrs() {
  const int sm = int(fft_smem_bytes<R>());
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_row_fwd<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
  if ((e = cudaFuncSetAttribute(k_col_main<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
  if ((e = cudaFuncSetAttribute(k_band_fwd<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
  if ((e = cudaFuncSetAttribute(k_band_inv<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
  if ((e = cudaFuncSetAttribute(k_row_inv<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))) return e;
  return cudaSuccess;
}

template <typename R>
cudaError_t prepare_kernels(int log2nx, int log2ny) {
  cudaError_t e = cudaSuccess;
  for (int l2 : {log2nx, log2ny}) {
#define DSNU_PREP(L2) e = set_fft_attrs<R, L2>()
    switch (l2) {
      DSNU_LOG2_CASES(DSNU_PREP)
      default: return cudaErrorInvalidValue;
    }
#undef DSNU_PREP
    if (e != cudaSuccess) return e;
  }
  return e;
}

template <typename R>
dsnu_status run_pipeline(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws,
                         const double* rho, double* phi, cudaStream_t st, int cj) {
  char* base = static_cast<char*>(ws);
  cpx<R>* A = reinterpret_cast<cpx<R>*>(base + L.off_A);
  cpx<R>* B = reinterpret_cast<cpx<R>*>(base + L.off_B);
  cpx<R>* Bband = reinterpret_cast<cpx<R>*>(base + L.off_Bband);
  cpx<R>* Sband = reinterpret_cast<cpx<R>*>(base + L.off_Sband);
  cpx<R>* cn = reinterpret_cast<cpx<R>*>(base + L.off_c);
  const AxisTabs<R> ax{static_cast<const cpx<R>*>(t.twN_x), static_cast<const cpx<R>*>(t.twM_x),
                       static_cast<const R*>(t.decon_x)};
  const AxisTabs<R> ay{static_cast<const cpx<R>*>(t.twN_y), static_cast<const cpx<R>*>(t.twM_y),
                       static_cast<const R*>(t.decon_y)};
  const MultTabs<R> mt{static_cast<const R*>(t.m_wx2), static_cast<const R*>(t.m_gx),
                       static_cast<const R*>(t.m_wy2), static_cast<const R*>(t.m_gy), g.sharp,
                       R(g.cut_radius * g.cut_radius)};
  const R* dcy = static_cast<const R*>(t.decon_y);
  const R* wts = static_cast<const R*>(t.node_w);
  const size_t smem = fft_smem_bytes<R>();
  const int rpc = 4096 >> g.log2nx;
  const int cpc = 4096 >> g.log2ny;
  const int grid_rows = (g.ny + rpc - 1) / rpc;
  const int grid_cols = (g.nx + 1 + cpc - 1) / cpc;
  const int grid_band = (g.Q + 1 + cpc - 1) / cpc;

#define DSNU_ROWF(L2) \
  k_row_fwd<R, L2><<<grid_rows, kThreads, smem, st>>>(rho, A, L.lda, B, L.ldb, g.Q, g.ny, ax, dcy, cj)
#define DSNU_COLM(L2) k_col_main<R, L2><<<grid_cols, kThreads, smem, st>>>(A, L.lda, g.nx + 1, ay, mt, cj)
#define DSNU_BANDF(L2) \
  k_band_fwd<R, L2><<<grid_band, kThreads, smem, st>>>(B, L.ldb, g.Q + 1, Bband, L.ldq, g.Q, ay, cj)
#define DSNU_BANDI(L2) \
  k_band_inv<R, L2><<<grid_band, kThreads, smem, st>>>(Sband, L.ldq, g.Q, g.Q + 1, B, L.ldb, ay, cj)
#define DSNU_ROWI(L2)                                                                          \
  k_row_inv<R, L2><<<grid_rows, kThreads, smem, st>>>(A, L.lda, B, L.ldb, g.Q, phi, g.ny, ax, dcy, \
                                                      R(g.scale), cj)
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_ROWF)
    default: return DSNU_EUNSUPPORTED;
  }
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_COLM)
    default: return DSNU_EUNSUPPORTED;
  }
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_BANDF)
    default: return DSNU_EUNSUPPORTED;
  }
  k_interp<R><<<(g.n_nodes + 7) / 8, 256, 0, st>>>(Bband, L.ldq, g.Q, t.node_q0, wts, t.node_D,
                                                   g.n_nodes, g.w, cn, cj);
  k_spread<R><<<g.n_tiles, 256, 0, st>>>(cn, t.node_q0, wts, g.w, t.tile_ptr, t.tile_nodes,
                                          g.tiles_x, g.Q, Sband, L.ldq, cj);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_BANDI)
    default: return DSNU_EUNSUPPORTED;
  }
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_ROWI)
    default: return DSNU_EUNSUPPORTED;
  }
#undef DSNU_ROWF
#undef DSNU_COLM
#undef DSNU_BANDF
#undef DSNU_BANDI
#undef DSNU_ROWI
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("kernel launch failed: ") + cudaGetErrorString(e));
    return DSNU_ECUDA;
  }
  return DSNU_OK;
}

}  // namespace dsnu
