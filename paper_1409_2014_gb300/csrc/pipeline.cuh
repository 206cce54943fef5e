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

template <typename K>
static cudaError_t persistent_grid(K kernel, int threads, size_t smem, int items, int* grid) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  const int cap = sms * per_sm;
  *grid = items < cap ? (items > 0 ? items : 1) : cap;
  return cudaSuccess;
}

template <typename R, int L2>
cudaError_t prepare_rows(PlanGeom& g) {
  using GG = Geo<R, L2>;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_row_fwd<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(GG::smem_row_fwd)))) return e;
  if ((e = cudaFuncSetAttribute(k_row_inv<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(GG::smem_row_inv)))) return e;
  if ((e = persistent_grid(k_row_fwd<R, L2>, GG::T_RF, GG::smem_row_fwd,
                           (g.ny + GG::RB_F - 1) / GG::RB_F, &g.grid_rowf))) return e;
  return persistent_grid(k_row_inv<R, L2>, GG::T_RI, GG::smem_row_inv, (g.ny + GG::RB_I - 1) / GG::RB_I,
                         &g.grid_rowi);
}

template <typename R, int L2>
cudaError_t prepare_cols(PlanGeom& g) {
  using GG = Geo<R, L2>;
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_col_main<R, L2>, A, int(GG::smem_col)))) return e;
  if ((e = cudaFuncSetAttribute(k_band_fwd<R, L2>, A, int(GG::smem_band_fwd)))) return e;
  if ((e = cudaFuncSetAttribute(k_band_inv<R, L2>, A, int(GG::smem_col)))) return e;
  if ((e = persistent_grid(k_col_main<R, L2>, GG::T_C, GG::smem_col, (g.nx + 1 + GG::CC - 1) / GG::CC,
                           &g.grid_col))) return e;
  if ((e = persistent_grid(k_band_fwd<R, L2>, GG::T_C, GG::smem_band_fwd, (g.Q + 1 + GG::CC - 1) / GG::CC,
                           &g.grid_bandf))) return e;
  return persistent_grid(k_band_inv<R, L2>, GG::T_C, GG::smem_col, (g.Q + 1 + GG::CC - 1) / GG::CC,
                         &g.grid_bandi);
}

template <typename R>
cudaError_t prepare_kernels(PlanGeom& g) {
  cudaError_t e = cudaSuccess;
#define DSNU_PREP_R(L2) e = prepare_rows<R, L2>(g)
#define DSNU_PREP_C(L2) e = prepare_cols<R, L2>(g)
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_PREP_R)
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_PREP_C)
    default: return cudaErrorInvalidValue;
  }
#undef DSNU_PREP_R
#undef DSNU_PREP_C
  return e;
}

// One solve, all kernels in order on `st`: row_fwd, the band chain
// (band_fwd, interp, spread, spread_reduce, band_inv), col_main, row_inv.  With `ev`
// (profiling) kProfEvents events are recorded before the first kernel and
// after each kernel, in launch order.
template <typename R>
dsnu_status run_pipeline(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws,
                         const double* rho, double* phi, cudaStream_t st, int cj, cudaEvent_t* ev) {
  char* base = static_cast<char*>(ws);
  cpx<R>* A = reinterpret_cast<cpx<R>*>(base + L.off_A);
  cpx<R>* B = reinterpret_cast<cpx<R>*>(base + L.off_B);
  cpx<R>* Bband = reinterpret_cast<cpx<R>*>(base + L.off_Bband);
  cpx<R>* Sband = reinterpret_cast<cpx<R>*>(base + L.off_Sband);
  cpx<R>* cn = reinterpret_cast<cpx<R>*>(base + L.off_c);
  const AxisTabs<R> ax{static_cast<const cpx<R>*>(t.stw_x), static_cast<const cpx<R>*>(t.twm_lo_x),
                       static_cast<const cpx<R>*>(t.twm_hi_x), g.log2lo_x, static_cast<const R*>(t.decon_x)};
  const AxisTabs<R> ay{static_cast<const cpx<R>*>(t.stw_y), static_cast<const cpx<R>*>(t.twm_lo_y),
                       static_cast<const cpx<R>*>(t.twm_hi_y), g.log2lo_y, static_cast<const R*>(t.decon_y)};
  const MultTabs<R> mt{static_cast<const R*>(t.m_wx2), static_cast<const R*>(t.m_gx),
                       g.n_gy, R(1.0 / (g.sigma * g.sigma)),
                       R(-g.dky2 / (g.sigma * g.sigma) * 1.4426950408889634), R(g.dky2), g.ny, g.sharp,
                       R(g.cut_radius * g.cut_radius)};
  const R* dcy = static_cast<const R*>(t.decon_y);
  const R* wts = static_cast<const R*>(t.node_w);
  const int ldqA = L.ldqA, ldqB = L.ldqB;

#define DSNU_ROWF(L2)                                                                               \
  k_row_fwd<R, L2><<<g.grid_rowf, Geo<R, L2>::T_RF,                                               \
                     Geo<R, L2>::smem_row_fwd, st>>>(rho, A, ldqA, B, ldqB, g.Q, g.ny, ax, dcy, cj)
#define DSNU_COLM(L2)                                                                                 \
  k_col_main<R, L2><<<g.grid_col, Geo<R, L2>::T_C,                                                 \
                      Geo<R, L2>::smem_col, st>>>(A, ldqA, g.nx + 1, ay, mt, cj)
#define DSNU_BANDF(L2)                                                                                \
  k_band_fwd<R, L2><<<g.grid_bandf, Geo<R, L2>::T_C,                                               \
                      Geo<R, L2>::smem_band_fwd, st>>>(B, ldqB, g.Q + 1, Bband, L.ldq, g.Q, ay, cj)
#define DSNU_BANDI(L2)                                                                                \
  k_band_inv<R, L2><<<g.grid_bandi, Geo<R, L2>::T_C,                                               \
                      Geo<R, L2>::smem_col, st>>>(Sband, L.ldq, g.Q, g.Q + 1, B, ldqB, ay, cj)
#define DSNU_ROWI(L2)                                                                                 \
  k_row_inv<R, L2><<<g.grid_rowi, Geo<R, L2>::T_RI,                                                \
                     Geo<R, L2>::smem_row_inv, st>>>(A, ldqA, B, ldqB, g.Q, phi, g.ny, ax, dcy,     \
                                                     R(g.scale), cj)
#define DSNU_MARK(I) \
  if (ev) cudaEventRecord(ev[I], st)
  DSNU_MARK(0);
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_ROWF)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(1);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_BANDF)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(2);
  k_interp<R><<<(g.n_nodes + 7) / 8, 256, 0, st>>>(Bband, L.ldq, g.Q, t.node_q0, wts, t.node_D,
                                                   g.n_nodes, g.w, cn, cj);
  DSNU_MARK(3);
  cpx<R>* partial = reinterpret_cast<cpx<R>*>(base + L.off_partial);
  if (g.n_items > 0)
    k_spread<R><<<g.n_items, kSpreadThreads, 0, st>>>(cn, t.item_range, t.ent_node, t.ent_q0,
                                                      static_cast<const R*>(t.ent_w), t.item_tile, g.w,
                                                      g.tiles_x, g.Q, partial);
  DSNU_MARK(4);
  k_spread_reduce<R><<<g.n_tiles, kTile * kTile, 0, st>>>(partial, t.tile_items, g.tiles_x, g.n_tiles,
                                                         g.Q, Sband, L.ldq, cj);
  DSNU_MARK(5);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_BANDI)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(6);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_COLM)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(7);
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_ROWI)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(8);
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
