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
  using GG = Geo<R, L2>;
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_row_fwd<R, L2>, A, int(GG::smem_row_fwd)))) return e;
  if ((e = cudaFuncSetAttribute(k_col_main<R, L2>, A, int(GG::smem_col)))) return e;
  if ((e = cudaFuncSetAttribute(k_band_fwd<R, L2>, A, int(GG::smem_band_fwd)))) return e;
  if ((e = cudaFuncSetAttribute(k_band_inv<R, L2>, A, int(GG::smem_col)))) return e;
  if ((e = cudaFuncSetAttribute(k_row_inv<R, L2>, A, int(GG::smem_row_inv)))) return e;
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

// One solve.  row_fwd runs on `st`; the band chain (band_fwd, interp, spread,
// band_inv) runs on the plan's side stream concurrently with col_main, and
// row_inv waits for both.  With `ev` (profiling) the kStages + 2 events are:
// 0 before row_fwd, 1 after row_fwd (fork), 2 after col_main, 3..6 after the
// four band kernels (side stream), 7 after the join on `st`, 8 after row_inv.
template <typename R>
dsnu_status run_pipeline(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws,
                         const double* rho, double* phi, cudaStream_t st, int cj,
                         const StreamSet& ss, cudaEvent_t* ev) {
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
  const int ldqA = L.ldqA, ldqB = L.ldqB;
  cudaStream_t sd = ss.side;

#define DSNU_ROWF(L2)                                                                               \
  k_row_fwd<R, L2><<<(g.ny + Geo<R, L2>::RB_F - 1) / Geo<R, L2>::RB_F, Geo<R, L2>::T_RF,            \
                     Geo<R, L2>::smem_row_fwd, st>>>(rho, A, ldqA, B, ldqB, g.Q, g.ny, ax, dcy, cj)
#define DSNU_COLM(L2)                                                                                 \
  k_col_main<R, L2><<<(g.nx + 1 + Geo<R, L2>::CC - 1) / Geo<R, L2>::CC, Geo<R, L2>::T_C,            \
                      Geo<R, L2>::smem_col, st>>>(A, ldqA, g.nx + 1, ay, mt, cj)
#define DSNU_BANDF(L2)                                                                                \
  k_band_fwd<R, L2><<<(g.Q + 1 + Geo<R, L2>::CC - 1) / Geo<R, L2>::CC, Geo<R, L2>::T_C,             \
                      Geo<R, L2>::smem_band_fwd, sd>>>(B, ldqB, g.Q + 1, Bband, L.ldq, g.Q, ay, cj)
#define DSNU_BANDI(L2)                                                                                \
  k_band_inv<R, L2><<<(g.Q + 1 + Geo<R, L2>::CC - 1) / Geo<R, L2>::CC, Geo<R, L2>::T_C,             \
                      Geo<R, L2>::smem_col, sd>>>(Sband, L.ldq, g.Q, g.Q + 1, B, ldqB, ay, cj)
#define DSNU_ROWI(L2)                                                                                 \
  k_row_inv<R, L2><<<(g.ny + Geo<R, L2>::RB_I - 1) / Geo<R, L2>::RB_I, Geo<R, L2>::T_RI,            \
                     Geo<R, L2>::smem_row_inv, st>>>(A, ldqA, B, ldqB, g.Q, phi, g.ny, ax, dcy,     \
                                                     R(g.scale), cj)
#define DSNU_MARK(I, S) \
  if (ev) cudaEventRecord(ev[I], S)
  DSNU_MARK(0, st);
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_ROWF)
    default: return DSNU_EUNSUPPORTED;
  }
  cudaEventRecord(ev ? ev[1] : ss.fork, st);
  cudaStreamWaitEvent(sd, ev ? ev[1] : ss.fork, 0);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_COLM)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(2, st);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_BANDF)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(3, sd);
  k_interp<R><<<(g.n_nodes + 7) / 8, 256, 0, sd>>>(Bband, L.ldq, g.Q, t.node_q0, wts, t.node_D,
                                                   g.n_nodes, g.w, cn, cj);
  DSNU_MARK(4, sd);
  k_spread<R><<<g.n_tiles, kTile * kTile, 0, sd>>>(cn, t.tile_ptr, t.ent_node, t.ent_q0,
                                                   static_cast<const R*>(t.ent_w), g.w, g.tiles_x,
                                                   g.Q, Sband, L.ldq, cj);
  DSNU_MARK(5, sd);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_BANDI)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(6, sd);
  cudaEventRecord(ss.join, sd);
  cudaStreamWaitEvent(st, ss.join, 0);
  DSNU_MARK(7, st);
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_ROWI)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(8, st);
#undef DSNU_ROWF
#undef DSNU_COLM
#undef DSNU_BANDF
#undef DSNU_BANDI
#undef DSNU_ROWI
#undef DSNU_MARK
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("kernel launch failed: ") + cudaGetErrorString(e));
    return DSNU_ECUDA;
  }
  return DSNU_OK;
}

}  // namespace dsnu
