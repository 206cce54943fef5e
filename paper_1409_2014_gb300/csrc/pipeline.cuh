// pipeline.cuh -- launch sequence of one solve (included once per precision).
#pragma once

#include <cmath>

#include "internal.h"
#include "kernels.cuh"
#include "standard.cuh"

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

// Number of CTAs of `kernel` that can be resident at once (SMs x occupancy).
template <typename K>
static cudaError_t resident_ctas(K kernel, int threads, size_t smem, int* cap) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  *cap = sms * per_sm;
  return cudaSuccess;
}

// Persistent grid: one CTA per work item up to the resident capacity.
static inline int persistent_grid(long items, int cap) {
  return items < cap ? (items > 0 ? int(items) : 1) : cap;
}

template <typename R, int L2>
cudaError_t prepare_rows(PlanGeom& g) {
  using GG = Geo<R, L2>;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_row_fwd<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(GG::smem_row_fwd)))) return e;
  if ((e = cudaFuncSetAttribute(k_row_inv<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                int(GG::smem_row_inv_limit)))) return e;
  // the band values of the inverse row pass are prefetched when they fit
  // without lowering the CTAs per SM
  g.rowi_bpf = 0;
  g.smem_rowi = GG::smem_row_inv;
  if constexpr (GG::ROWI_PF && DSNU_ROWI_BPF) {
    const size_t with_s = GG::smem_row_inv + size_t(16) * size_t(g.Q + 1);
    if (with_s <= GG::smem_row_inv_limit && size_t(GG::MINB_I0) * (with_s + 1024) <= size_t(233472)) {
      g.rowi_bpf = 1;
      g.smem_rowi = with_s;
    }
  }
  g.row_pf = (GG::ROW_PF ? 1 : 0) | (GG::ROWI_PF ? 2 : 0) | (g.rowi_bpf ? 4 : 0);
  if ((e = resident_ctas(k_row_fwd<R, L2>, GG::T_RF, GG::smem_row_fwd, &g.cap_rowf))) return e;
  return resident_ctas(k_row_inv<R, L2>, GG::T_RI, g.smem_rowi, &g.cap_rowi);
}

template <typename R, int L2>
cudaError_t prepare_cols(PlanGeom& g) {
  using GG = Geo<R, L2>;
  cudaError_t e;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if ((e = cudaFuncSetAttribute(k_col_main<R, L2, false>, A, int(GG::smem_col_main)))) return e;
  if ((e = cudaFuncSetAttribute(k_col_main<R, L2, true>, A, int(GG::smem_col_main)))) return e;
  if ((e = cudaFuncSetAttribute(k_band_fwd<R, L2>, A, int(GG::smem_col)))) return e;
  if ((e = cudaFuncSetAttribute(k_band_inv<R, L2>, A, int(GG::smem_col)))) return e;
  if ((e = g.m_generic ? resident_ctas(k_col_main<R, L2, true>, GG::T_C, GG::smem_col_main, &g.cap_col)
                       : resident_ctas(k_col_main<R, L2, false>, GG::T_C, GG::smem_col_main, &g.cap_col)))
    return e;
  if ((e = resident_ctas(k_band_fwd<R, L2>, GG::T_C, GG::smem_col, &g.cap_bandf))) return e;
  return resident_ctas(k_band_inv<R, L2>, GG::T_C, GG::smem_col, &g.cap_bandi);
}

template <typename R, int L2>
cudaError_t prepare_std_rows(PlanGeom& g) {
  using GS = GeoStd<R, L2>;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_std_row_fwd<R, L2>, A, int(GS::smem_rowf)))) return e;
  if ((e = cudaFuncSetAttribute(k_std_row_inv<R, L2>, A, int(GS::smem_rowi)))) return e;
  if ((e = resident_ctas(k_std_row_fwd<R, L2>, GS::T, GS::smem_rowf, &g.cap_rowf))) return e;
  return resident_ctas(k_std_row_inv<R, L2>, GS::T, GS::smem_rowi, &g.cap_rowi);
}

template <typename R, int L2>
cudaError_t prepare_std_cols(PlanGeom& g) {
  using GS = GeoStd<R, L2>;
  cudaError_t e = cudaFuncSetAttribute(k_std_col<R, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(GS::smem));
  if (e) return e;
  return resident_ctas(k_std_col<R, L2>, GS::T, GS::smem, &g.cap_col);
}

template <typename R>
cudaError_t prepare_kernels(PlanGeom& g) {
  cudaError_t e = cudaSuccess;
  if (g.standard) {
#define DSNU_PREP_SR(L2) e = prepare_std_rows<R, L2>(g)
#define DSNU_PREP_SC(L2) e = prepare_std_cols<R, L2>(g)
    switch (g.log2nx) {
      DSNU_LOG2_CASES(DSNU_PREP_SR)
      default: return cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
    switch (g.log2ny) {
      DSNU_LOG2_CASES(DSNU_PREP_SC)
      default: return cudaErrorInvalidValue;
    }
#undef DSNU_PREP_SR
#undef DSNU_PREP_SC
    return e;
  }
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
// The standard periodic FFT solver (standard.cuh): row_fwd, col, row_inv.
// With `ev` the same kProfEvents events are recorded as for the split solver,
// the band-chain stages being empty, so that the stage names keep their
// meaning (row_fwd, col_main, row_inv).
template <typename R>
dsnu_status run_standard(const PlanGeom& g, const PlanTables& t, const WsLayout& L, const Members& mem,
                         cudaStream_t st, int cj, cudaEvent_t* ev) {
  // FP32 row passes read the compact stage table (GeoStd::PF)
  const cpx<R>* sx = static_cast<const cpx<R>*>(sizeof(R) == 4 ? t.stwc_x : t.stw_x);
  const cpx<R>* sy = static_cast<const cpx<R>*>(t.stw_y);
  MultTabs<R> mt{};
  mt.wx2 = static_cast<const R*>(t.m_wx2);
  mt.dky2 = R(g.dky2);
  mt.dky = R(std::sqrt(g.dky2));
  mt.generic = g.m_generic;
  mt.alpha = g.m_alpha;
  mt.a0 = R(g.m_a0);
  mt.ac = R(g.m_ac);
  mt.as2 = R(2.0 * g.m_as);
  mt.kx = static_cast<const R*>(t.m_kx);
  const long nm = mem.count;
  const int ldq = L.ldqA;
#define DSNU_SROWF(L2)                                                                             \
  launch_k(g.pdl != 0, k_std_row_fwd<R, L2>,                                                       \
           dim3(persistent_grid(nm * ((g.ny / 2 + GeoStd<R, L2>::PER - 1) / GeoStd<R, L2>::PER),    \
                                g.cap_rowf)),                                                      \
           dim3(GeoStd<R, L2>::T), GeoStd<R, L2>::smem_rowf, st, mem, L.off_A, ldq, g.ny, sx, cj, t.status)
#define DSNU_SCOL(L2)                                                                              \
  launch_k(g.pdl != 0, k_std_col<R, L2>,                                                           \
           dim3(persistent_grid(nm * ((ldq + GeoStd<R, L2>::PER - 1) / GeoStd<R, L2>::PER), g.cap_col)), \
           dim3(GeoStd<R, L2>::T), GeoStd<R, L2>::smem, st, mem, L.off_A, ldq, ldq, sy, mt, R(g.scale), cj)
#define DSNU_SROWI(L2)                                                                             \
  launch_k(g.pdl != 0, k_std_row_inv<R, L2>,                                                       \
           dim3(persistent_grid(nm * ((g.ny / 2 + GeoStd<R, L2>::PER - 1) / GeoStd<R, L2>::PER),    \
                                g.cap_rowi)),                                                      \
           dim3(GeoStd<R, L2>::T), GeoStd<R, L2>::smem_rowi, st, mem, L.off_A, ldq, g.ny, sx, cj)
  if (ev) cudaEventRecord(ev[0], st);
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_SROWF)
    default: return DSNU_EUNSUPPORTED;
  }
  if (ev)
    for (int i = 1; i <= 6; ++i) cudaEventRecord(ev[i], st);
  switch (g.log2ny) {
    DSNU_LOG2_CASES(DSNU_SCOL)
    default: return DSNU_EUNSUPPORTED;
  }
  if (ev) cudaEventRecord(ev[7], st);
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_SROWI)
    default: return DSNU_EUNSUPPORTED;
  }
  if (ev) cudaEventRecord(ev[8], st);
#undef DSNU_SROWF
#undef DSNU_SCOL
#undef DSNU_SROWI
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_last_error(std::string("kernel launch failed: ") + cudaGetErrorString(e));
    return DSNU_ECUDA;
  }
  return DSNU_OK;
}

template <typename R>
dsnu_status run_pipeline(const PlanGeom& g, const PlanTables& t, const WsLayout& L, const Members& mem,
                         cudaStream_t st, int cj, cudaEvent_t* ev, const Overlap* ov) {
  if (g.standard) return run_standard<R>(g, t, L, mem, st, cj, ev);
  const WsOff off{L.off_A, L.off_B, L.off_Bband, L.off_Sband, L.off_c, L.off_partial, L.off_sched};
  const AxisTabs<R> ax{static_cast<const cpx<R>*>(t.stw_x), static_cast<const cpx<R>*>(t.twm_lo_x),
                       static_cast<const cpx<R>*>(t.twm_hi_x), g.log2lo_x, static_cast<const R*>(t.decon_x),
                       static_cast<const cpx<R>*>(t.stwc_x)};
  const AxisTabs<R> ay{static_cast<const cpx<R>*>(t.stw_y), static_cast<const cpx<R>*>(t.twm_lo_y),
                       static_cast<const cpx<R>*>(t.twm_hi_y), g.log2lo_y, static_cast<const R*>(t.decon_y),
                       nullptr};
  const MultTabs<R> mt{static_cast<const R*>(t.m_wx2), static_cast<const R*>(t.m_gx),
                       g.n_gy, R(1.0 / (g.sigma * g.sigma)),
                       R(-g.dky2 / (g.sigma * g.sigma) * 1.4426950408889634), R(g.dky2), g.ny, g.sharp,
                       R(g.cut_radius * g.cut_radius), g.m_generic, g.m_alpha, R(g.m_a0), R(g.m_ac),
                       R(2.0 * g.m_as), R(std::sqrt(g.dky2)), static_cast<const R*>(t.m_kx),
                       static_cast<const R*>(t.m1tab), g.ny + 4};
  const R* dcy = static_cast<const R*>(t.decon_y);
  const R* wts = static_cast<const R*>(t.node_w);
  const int ldqA = L.ldqA, ldqB = L.ldqB;
  const long nm = mem.count;

#define DSNU_ROWF(L2)                                                                               \
  launch_k(g.pdl != 0, k_row_fwd<R, L2>,                                                            \
           dim3(persistent_grid(nm * ((g.ny + Geo<R, L2>::RB_F - 1) / Geo<R, L2>::RB_F), g.cap_rowf)), \
           dim3(Geo<R, L2>::T_RF), Geo<R, L2>::smem_row_fwd, st, mem, off, ldqA, ldqB, g.Q, g.ny, ax, dcy, cj, \
           t.status)
#define DSNU_COLM(L2)                                                                               \
  if (g.m_generic)                                                                                  \
    launch_k(g.pdl != 0, k_col_main<R, L2, true>,                                                   \
             dim3(persistent_grid(nm * ((g.nx + 1 + Geo<R, L2>::CC - 1) / Geo<R, L2>::CC), capc)), \
             dim3(Geo<R, L2>::T_C), Geo<R, L2>::smem_col_main, st, mem, off, ldqA, g.nx + 1, ay, mt, cj); \
  else                                                                                              \
    launch_k(g.pdl != 0, k_col_main<R, L2, false>,                                                  \
             dim3(persistent_grid(nm * ((g.nx + 1 + Geo<R, L2>::CC - 1) / Geo<R, L2>::CC), capc)), \
             dim3(Geo<R, L2>::T_C), Geo<R, L2>::smem_col_main, st, mem, off, ldqA, g.nx + 1, ay, mt, cj)
#define DSNU_BANDF(L2)                                                                              \
  launch_k(g.pdl != 0, k_band_fwd<R, L2>,                                                           \
           dim3(persistent_grid(nm * ((g.Q + 1 + Geo<R, L2>::CC - 1) / Geo<R, L2>::CC), g.cap_bandf)), \
           dim3(Geo<R, L2>::T_C), Geo<R, L2>::smem_col, bst, mem, off, ldqB, g.Q + 1, L.ldq, g.Q, ay, cj)
#define DSNU_BANDI(L2)                                                                              \
  launch_k(g.pdl != 0, k_band_inv<R, L2>,                                                           \
           dim3(persistent_grid(nm * ((g.Q + 1 + Geo<R, L2>::CC - 1) / Geo<R, L2>::CC), g.cap_bandi)), \
           dim3(Geo<R, L2>::T_C), Geo<R, L2>::smem_col, bst, mem, off, L.ldq, g.Q, g.Q + 1, ldqB, ay, cj)
#define DSNU_ROWI(L2)                                                                               \
  launch_k(g.pdl != 0, k_row_inv<R, L2>,                                                            \
           dim3(persistent_grid(nm * ((g.ny + Geo<R, L2>::RB_I - 1) / Geo<R, L2>::RB_I), g.cap_rowi)), \
           dim3(Geo<R, L2>::T_RI), g.smem_rowi, st, mem, off, ldqA, ldqB, g.Q, g.ny, ax, dcy, R(g.scale), cj, \
           g.rowi_bpf, g.acc64)
#define DSNU_MARK(I) \
  if (ev) cudaEventRecord(ev[I], st)
  // the band chain (type-2 columns, interpolation, weighting, spreading,
  // inverse band columns) on stream bst
  cudaStream_t bst = st;
  int capc = g.cap_col;
  auto band_chain = [&](bool marks) -> dsnu_status {
    switch (g.log2ny) {
      DSNU_LOG2_CASES(DSNU_BANDF)
      default: return DSNU_EUNSUPPORTED;
    }
    if (marks) DSNU_MARK(2);
    launch_k(g.pdl != 0, k_interp_tile<R>, dim3(g.n_itiles, mem.count), dim3(256),
             interp_tile_smem(g.w, sizeof(cpx<R>)), bst, mem, off, L.ldq, g.Q, t.node_q0, wts, t.node_D, t.itile_ptr,
             t.itile_org, t.itile_nodes, g.w, cj);
    if (marks) DSNU_MARK(3);
    launch_spread<R>(g.spread_cfg, mem, off, t, g, L.ldq, cj, bst, 0, g.pdl != 0);
    if (marks) DSNU_MARK(4);
    launch_spread<R>(g.spread_cfg, mem, off, t, g, L.ldq, cj, bst, 1, g.pdl != 0);
    if (marks) DSNU_MARK(5);
    switch (g.log2ny) {
      DSNU_LOG2_CASES(DSNU_BANDI)
      default: return DSNU_EUNSUPPORTED;
    }
    return DSNU_OK;
  };
  const bool overlap = ov && ov->reserve > 0 && !ev && g.cap_col > ov->reserve;
  DSNU_MARK(0);
  switch (g.log2nx) {
    DSNU_LOG2_CASES(DSNU_ROWF)
    default: return DSNU_EUNSUPPORTED;
  }
  DSNU_MARK(1);
  if (overlap) {
    // the column pass keeps all but `reserve` SMs; the band chain runs next
    // to it on the plan's low-priority side stream; row_inv joins both
    cudaEventRecord(ov->fork, st);
    cudaStreamWaitEvent(ov->side, ov->fork, 0);
    capc = g.cap_col - ov->reserve;
    switch (g.log2ny) {
      DSNU_LOG2_CASES(DSNU_COLM)
      default: return DSNU_EUNSUPPORTED;
    }
    bst = ov->side;
    const dsnu_status sb = band_chain(false);
    if (sb != DSNU_OK) return sb;
    cudaEventRecord(ov->join, ov->side);
    cudaStreamWaitEvent(st, ov->join, 0);
  } else {
    const dsnu_status sb = band_chain(true);
    if (sb != DSNU_OK) return sb;
    DSNU_MARK(6);
    switch (g.log2ny) {
      DSNU_LOG2_CASES(DSNU_COLM)
      default: return DSNU_EUNSUPPORTED;
    }
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

template <typename R>
cudaError_t time_spread(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws, int reps, float* ms) {
  const WsOff off{L.off_A, L.off_B, L.off_Bband, L.off_Sband, L.off_c, L.off_partial, L.off_sched};
  const Members mem = single_member(nullptr, nullptr, ws);
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) return e;
  launch_spread<R>(g.spread_cfg, mem, off, t, g, L.ldq, 0, 0, 2, false);  // warm-up
  cudaEventRecord(e0, 0);
  for (int i = 0; i < reps; ++i) launch_spread<R>(g.spread_cfg, mem, off, t, g, L.ldq, 0, 0, 2, false);
  cudaEventRecord(e1, 0);
  e = cudaEventSynchronize(e1);
  float total = 0.f;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&total, e0, e1);
  if (e == cudaSuccess) e = cudaGetLastError();
  *ms = total / float(reps);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

}  // namespace dsnu
