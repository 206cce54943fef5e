// batch_ragged.cu -- a batch of densities on grids of different sizes, solved
// by one launch per pipeline stage.
//
// The split solver of Sec. 2.1 runs eight kernels per density (row pass, the
// band chain of both NUFFTs, column pass, inverse row pass).  For a batch of
// mixed-precision members whose grids are 256^2 .. 2048^2 (one plan per
// distinct grid, up to kRagMaxGroups plans), each of the eight stages is one
// launch for every member of every size:
//
//   * the FFT stages (row_fwd, band_fwd, col_main, band_inv, row_inv) are
//     persistent: the grid (SMs x resident CTAs) is cut into one contiguous
//     range of CTAs per plan, sized by the plan's share of the stage's work
//     (work items x log2 of the transform length); a CTA runs the kernel body
//     of its plan's grid size on its range only, as the single-plan launch
//     would on the whole grid (the same arithmetic; compiled into another
//     kernel, where the compiler may contract multiply-adds differently, so a
//     member's result equals its own dsnu_solve to FP32 rounding);
//   * interp, spread and spread_reduce take one CTA per (member, interpolation
//     item / spreading item / tile), numbered plan by plan; the column stage's
//     CTAs of a plan take its columns from that plan's work counter, as in a
//     single solve.
//
// Every FFT body here uses 256 threads (FP32, transform lengths 256 .. 2048),
// so one block size serves all plans.  The spreading pair needs one tile
// configuration for the whole batch; when the plans' autotuners chose
// different ones, that pair is launched once per plan instead.  As in a
// single solve of a large grid, the band chain runs on a low-priority side
// stream next to the column stage, whose CTAs leave it a share of the SMs in
// proportion to the band columns' work.  The stage launches use programmatic
// dependent launch like the single solves.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace dsnu {

namespace {

constexpr int kLog2Min = 8, kLog2Max = 11;  // grid sizes of the one-launch-per-stage schedule
constexpr int kRagThreads = 256;

enum RagStage { RS_ROWF = 0, RS_BANDF, RS_INTERP, RS_SPREAD, RS_REDUCE, RS_BANDI, RS_COL, RS_ROWI, RS_N };

struct RagGroup {
  Members mem;
  WsOff off;
  AxisTabs<float> ax, ay;
  MultTabs<float> mt;
  const float* decon_y;
  float scale;
  int* status;
  int log2nx, log2ny, nx, ny, ldqA, ldqB, ldq, Q, bpf, acc64;
  const int2* node_q0;
  const float* node_w;
  const double* node_D;
  const int* itile_ptr;    // the plan's interpolation items (k_interp_tile)
  const int2* itile_org;
  const int* itile_nodes;
  int n_nodes, w;
  const int2* item_range;
  const int* ent_node;
  const int2* ent_q0;
  const float* ent_w;
  const int* item_tile;
  const int* tile_items;
  int tiles_x, n_tiles, n_items;
};

// lo[s][g] .. lo[s][g + 1] - 1: the CTAs of stage s that work for plan g;
// per[s][g]: CTAs per member in the numbered stages (interp, spread, reduce).
// Passed by value to every stage kernel (a launch copies it; a captured graph
// keeps its copy).
struct RagTable {
  int ngroups;
  int lo[RS_N][kRagMaxGroups + 1];
  int per[RS_N][kRagMaxGroups];
  RagGroup g[kRagMaxGroups];
};
static_assert(sizeof(RagTable) <= 32000, "the stage table must fit the kernel parameter space");

__device__ __forceinline__ int rag_group(const RagTable& T, int s, int b) {
  int g = 0;
  while (g + 1 < T.ngroups && b >= T.lo[s][g + 1]) ++g;
  return g;
}

#define DSNU_RAG_SIZES(CALL) \
  case 8: CALL(8); break;    \
  case 9: CALL(9); break;    \
  case 10: CALL(10); break;  \
  case 11: CALL(11); break;

// The persistent stages: CTA blockIdx.x works for plan g as CTA vb of vg.
// The table is a kernel parameter (constant bank), like a single plan's
// arguments, so that the bodies read it without holding it in registers.
#define DSNU_RAG_PERSISTENT(NAME, STAGE, MINB, AXIS, BODY_CALL)                                    \
  __global__ void __launch_bounds__(kRagThreads, MINB) NAME(const __grid_constant__ RagTable T) { \
    const int g = rag_group(T, STAGE, blockIdx.x);                                                \
    const RagGroup& a = T.g[g];                                                                   \
    const int vb = int(blockIdx.x) - T.lo[STAGE][g];                                              \
    const int vg = T.lo[STAGE][g + 1] - T.lo[STAGE][g];                                           \
    switch (a.AXIS) { DSNU_RAG_SIZES(BODY_CALL) default: break; }                                 \
  }

#define DSNU_RAG_ROWF(L) \
  row_fwd_body<float, L>(vb, vg, a.mem, a.off, a.ldqA, a.ldqB, a.Q, a.ny, a.ax, a.decon_y, 0, a.status)
#define DSNU_RAG_BANDF(L) band_fwd_body<float, L>(vb, vg, a.mem, a.off, a.ldqB, a.Q + 1, a.ldq, a.Q, a.ay, 0)
#define DSNU_RAG_COL(L)                                                                  \
  col_main_body<float, L, false>(vb, vg, a.mem, a.off, a.ldqA, a.nx + 1, a.ay, a.mt, 0, \
                                 ws_ptr<int>(member_at(a.mem, 0), a.off.sched))
#define DSNU_RAG_BANDI(L) band_inv_body<float, L>(vb, vg, a.mem, a.off, a.ldq, a.Q, a.Q + 1, a.ldqB, a.ay, 0)
#define DSNU_RAG_ROWI(L)                                                                                       \
  row_inv_body<float, L>(vb, vg, a.mem, a.off, a.ldqA, a.ldqB, a.Q, a.ny, a.ax, a.decon_y, a.scale, 0, a.bpf, \
                         a.acc64)

// (minimum resident CTAs as in the single-plan launches, but one for the band
// columns: their plan arguments, read with a run-time plan index, take
// registers that the single-plan launch reads from the constant bank)
DSNU_RAG_PERSISTENT(k_rag_row_fwd, RS_ROWF, 2, log2nx, DSNU_RAG_ROWF)
DSNU_RAG_PERSISTENT(k_rag_band_fwd, RS_BANDF, 1, log2ny, DSNU_RAG_BANDF)
DSNU_RAG_PERSISTENT(k_rag_col_main, RS_COL, DSNU_COLMAIN_MINB, log2ny, DSNU_RAG_COL)
DSNU_RAG_PERSISTENT(k_rag_band_inv, RS_BANDI, 1, log2ny, DSNU_RAG_BANDI)
DSNU_RAG_PERSISTENT(k_rag_row_inv, RS_ROWI, 2, log2nx, DSNU_RAG_ROWI)

// The numbered stages: CTA blockIdx.x is CTA r of plan g, i.e. block r % per
// of member r / per.
__device__ __forceinline__ void rag_numbered(const RagTable& T, int s, int* g, int* bx, int* mi) {
  *g = rag_group(T, s, blockIdx.x);
  const int r = int(blockIdx.x) - T.lo[s][*g];
  const int per = T.per[s][*g];
  *mi = r / per;
  *bx = r - *mi * per;
}

__global__ void __launch_bounds__(256) k_rag_interp(const __grid_constant__ RagTable T) {
  int g, bx, mi;
  rag_numbered(T, RS_INTERP, &g, &bx, &mi);
  const RagGroup& a = T.g[g];
  interp_tile_body<float>(bx, mi, a.mem, a.off, a.ldq, a.Q, a.node_q0, a.node_w, a.node_D, a.itile_ptr, a.itile_org,
                          a.itile_nodes, a.w, 0);
}

template <int TILE, int SPLIT, int CHUNK>
__global__ void __launch_bounds__(TILE * TILE * SPLIT) k_rag_spread(const __grid_constant__ RagTable T) {
  int g, bx, mi;
  rag_numbered(T, RS_SPREAD, &g, &bx, &mi);
  const RagGroup& a = T.g[g];
  spread_body<float, TILE, SPLIT, CHUNK>(bx, mi, a.mem, a.off, a.item_range, a.ent_node, a.ent_q0, a.ent_w,
                                         a.item_tile, a.w, a.tiles_x, a.Q);
}

template <int TILE>
__global__ void __launch_bounds__(TILE * TILE) k_rag_spread_reduce(const __grid_constant__ RagTable T) {
  int g, bx, mi;
  rag_numbered(T, RS_REDUCE, &g, &bx, &mi);
  const RagGroup& a = T.g[g];
  spread_reduce_body<float, TILE>(bx, mi, a.mem, a.off, a.tile_items, a.tiles_x, a.n_tiles, a.Q, a.ldq, 0);
}

// Per-size launch constants of the bodies (host side).
struct SizeInfo {
  int rows_f, rows_i, cols;                        // rows per item of the row passes, columns per item
  size_t smem_rowf, smem_col, smem_col_main;
};

template <int L>
SizeInfo size_info_of() {
  using GG = Geo<float, L>;
  static_assert(GG::T_RF == kRagThreads && GG::T_RI == kRagThreads && GG::T_C == kRagThreads,
                "one block size for every grid size of the schedule");
  return SizeInfo{GG::RB_F, GG::RB_I, GG::CC, GG::smem_row_fwd, GG::smem_col, GG::smem_col_main};
}

SizeInfo size_info(int log2n) {
  switch (log2n) {
    case 8: return size_info_of<8>();
    case 9: return size_info_of<9>();
    case 10: return size_info_of<10>();
    default: return size_info_of<11>();
  }
}

// The largest dynamic shared memory any plan of the schedule can ask of each
// persistent stage (set once per process as the kernels' limit).
size_t max_smem(int stage) {
  size_t m = 0;
  for (int l = kLog2Min; l <= kLog2Max; ++l) {
    const SizeInfo s = size_info(l);
    m = std::max(m, stage == RS_ROWF   ? s.smem_rowf
                    : stage == RS_COL  ? s.smem_col_main
                    : stage == RS_ROWI ? size_t(232448)
                                       : s.smem_col);
  }
  return m;
}

// Cut `grid` persistent CTAs into one range per plan, proportional to
// weight[g] and at most items[g] each (at least one each); writes lo[0..n].
int partition(const std::vector<long>& items, const std::vector<double>& weight, int cap, int* lo) {
  const int n = int(items.size());
  long total = 0;
  double wsum = 0.0;
  for (int g = 0; g < n; ++g) {
    total += items[g];
    wsum += weight[g];
  }
  const int grid = int(std::min<long>(cap, std::max<long>(total, n)));
  std::vector<int> cnt(n, 1);
  int used = n;
  // largest remainder: hand out the rest by weight, never beyond a plan's items
  while (used < grid) {
    int best = -1;
    double best_def = 0.0;
    for (int g = 0; g < n; ++g) {
      if (cnt[g] >= items[g]) continue;
      const double def = grid * weight[g] / wsum - cnt[g];
      if (best < 0 || def > best_def) {
        best = g;
        best_def = def;
      }
    }
    if (best < 0) break;
    ++cnt[best];
    ++used;
  }
  lo[0] = 0;
  for (int g = 0; g < n; ++g) lo[g + 1] = lo[g] + cnt[g];
  return lo[n];
}

dsnu_status rfail(dsnu_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

}  // namespace

struct Ragged {
  RagTable host;
  int grid[RS_N] = {};
  size_t smem[RS_N] = {};
  int spread_cfg = -1;   // common tile configuration, or -1: the spreading pair per plan
  int pdl = 1;
  std::vector<RaggedGroupIn> groups;
  // the band chain runs on `side` next to the column stage, which leaves it
  // `reserve` SMs' worth of CTAs
  cudaStream_t side = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  int reserve = 0;
};

bool ragged_eligible(const dsnu_plan* plans, int n, std::string* why) {
  if (n < 1 || n > kRagMaxGroups) {
    if (why) *why = "1 to " + std::to_string(kRagMaxGroups) + " distinct plans";
    return false;
  }
  for (int i = 0; i < n; ++i) {
    const PlanGeom& g = plans[i]->geom;
    if (g.precision != DSNU_MIXED || g.standard || g.m_generic) {
      if (why) *why = "mixed-precision split plans with the DS multiplier only";
      return false;
    }
    if (g.log2nx < kLog2Min || g.log2nx > kLog2Max || g.log2ny < kLog2Min || g.log2ny > kLog2Max) {
      if (why) *why = "grid sizes 256 .. 2048 per axis only";
      return false;
    }
  }
  return true;
}

dsnu_status ragged_create(const RaggedGroupIn* groups, int n, Ragged** out) {
  std::string why;
  std::vector<dsnu_plan> plans;
  for (int i = 0; i < n; ++i) plans.push_back(groups[i].plan);
  if (!ragged_eligible(plans.data(), n, &why)) return rfail(DSNU_EUNSUPPORTED, "one launch per stage: " + why);
  Ragged* R = new (std::nothrow) Ragged();
  if (!R) return rfail(DSNU_ENOMEM, "host allocation failed");
  R->groups.assign(groups, groups + n);
  RagTable& T = R->host;
  T.ngroups = n;
  R->spread_cfg = groups[0].plan->geom.spread_cfg;
  std::vector<long> items[RS_N];
  std::vector<double> weight[RS_N];
  for (int i = 0; i < n; ++i) {
    const dsnu_plan p = groups[i].plan;
    const PlanGeom& g = p->geom;
    const PlanTables& t = p->tab;
    const WsLayout& L = p->ws_layout;
    R->pdl = R->pdl && g.pdl;
    if (g.spread_cfg != R->spread_cfg) R->spread_cfg = -1;
    RagGroup& a = T.g[i];
    a.mem.dev = groups[i].dev_members;
    a.mem.one = groups[i].first;
    a.mem.count = groups[i].count;
    a.off = WsOff{L.off_A, L.off_B, L.off_Bband, L.off_Sband, L.off_c, L.off_partial, L.off_sched};
    a.ax = AxisTabs<float>{static_cast<const cpx<float>*>(t.stw_x), static_cast<const cpx<float>*>(t.twm_lo_x),
                           static_cast<const cpx<float>*>(t.twm_hi_x), g.log2lo_x,
                           static_cast<const float*>(t.decon_x), static_cast<const cpx<float>*>(t.stwc_x)};
    a.ay = AxisTabs<float>{static_cast<const cpx<float>*>(t.stw_y), static_cast<const cpx<float>*>(t.twm_lo_y),
                           static_cast<const cpx<float>*>(t.twm_hi_y), g.log2lo_y,
                           static_cast<const float*>(t.decon_y), nullptr};
    a.mt = MultTabs<float>{static_cast<const float*>(t.m_wx2), static_cast<const float*>(t.m_gx), g.n_gy,
                           float(1.0 / (g.sigma * g.sigma)),
                           float(-g.dky2 / (g.sigma * g.sigma) * 1.4426950408889634), float(g.dky2), g.ny, g.sharp,
                           float(g.cut_radius * g.cut_radius), 0, 0, 0.f, 0.f, 0.f, float(std::sqrt(g.dky2)),
                           static_cast<const float*>(t.m_kx), static_cast<const float*>(t.m1tab), g.ny + 4};
    a.decon_y = static_cast<const float*>(t.decon_y);
    a.scale = float(g.scale);
    a.status = t.status;
    a.log2nx = g.log2nx;
    a.log2ny = g.log2ny;
    a.nx = g.nx;
    a.ny = g.ny;
    a.ldqA = L.ldqA;
    a.ldqB = L.ldqB;
    a.ldq = L.ldq;
    a.Q = g.Q;
    a.bpf = g.rowi_bpf;
    a.acc64 = g.acc64;
    a.node_q0 = t.node_q0;
    a.node_w = static_cast<const float*>(t.node_w);
    a.node_D = t.node_D;
    a.itile_ptr = t.itile_ptr;
    a.itile_org = t.itile_org;
    a.itile_nodes = t.itile_nodes;
    a.n_nodes = g.n_nodes;
    a.w = g.w;
    a.item_range = t.item_range;
    a.ent_node = t.ent_node;
    a.ent_q0 = t.ent_q0;
    a.ent_w = static_cast<const float*>(t.ent_w);
    a.item_tile = t.item_tile;
    a.tile_items = t.tile_items;
    a.tiles_x = g.tiles_x;
    a.n_tiles = g.n_tiles;
    a.n_items = g.n_items;
    const long m = groups[i].count;
    const SizeInfo sx = size_info(g.log2nx), sy = size_info(g.log2ny);
    const double lx = g.log2nx, ly = g.log2ny;
    items[RS_ROWF].push_back(m * ((g.ny + sx.rows_f - 1) / sx.rows_f));
    weight[RS_ROWF].push_back(items[RS_ROWF].back() * lx);
    items[RS_ROWI].push_back(m * ((g.ny + sx.rows_i - 1) / sx.rows_i));
    weight[RS_ROWI].push_back(items[RS_ROWI].back() * lx);
    items[RS_COL].push_back(m * ((g.nx + 1 + sy.cols - 1) / sy.cols));
    weight[RS_COL].push_back(items[RS_COL].back() * ly);
    items[RS_BANDF].push_back(m * ((g.Q + 1 + sy.cols - 1) / sy.cols));
    weight[RS_BANDF].push_back(items[RS_BANDF].back() * ly);
    items[RS_BANDI].push_back(items[RS_BANDF].back());
    weight[RS_BANDI].push_back(weight[RS_BANDF].back());
    T.per[RS_INTERP][i] = std::max(g.n_itiles, 1);
    R->smem[RS_INTERP] = std::max(R->smem[RS_INTERP], interp_tile_smem(g.w, sizeof(cpx<float>)));
    T.per[RS_SPREAD][i] = std::max(g.n_items, 1);
    T.per[RS_REDUCE][i] = std::max(g.n_tiles, 1);
    R->smem[RS_ROWF] = std::max(R->smem[RS_ROWF], sx.smem_rowf);
    R->smem[RS_ROWI] = std::max(R->smem[RS_ROWI], g.smem_rowi);
    R->smem[RS_COL] = std::max(R->smem[RS_COL], sy.smem_col_main);
    R->smem[RS_BANDF] = std::max(R->smem[RS_BANDF], sy.smem_col);
    R->smem[RS_BANDI] = R->smem[RS_BANDF];
  }
  // the numbered stages: plan by plan, member by member
  for (int s : {int(RS_INTERP), int(RS_SPREAD), int(RS_REDUCE)}) {
    T.lo[s][0] = 0;
    for (int i = 0; i < n; ++i) T.lo[s][i + 1] = T.lo[s][i] + T.per[s][i] * groups[i].count;
    R->grid[s] = T.lo[s][n];
  }
  // the band chain's share of the column stage's SMs: its band-column work
  // against the column work (at least 12 of 152, at most half)
  int sms = 0;
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    double wb = 0.0, wc = 0.0;
    for (int i = 0; i < n; ++i) {
      wb += weight[RS_BANDF][i] + weight[RS_BANDI][i];
      wc += weight[RS_COL][i];
    }
    R->reserve = std::min(sms / 2, std::max((sms * 12 + 76) / 152, int(std::lround(sms * wb / (wb + wc)))));
  }
  // the persistent stages: one range of CTAs per plan
  cudaError_t e = cudaSuccess;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
  struct {
    int s;
    const void* k;
  } pers[] = {{RS_ROWF, (const void*)k_rag_row_fwd}, {RS_BANDF, (const void*)k_rag_band_fwd},
              {RS_COL, (const void*)k_rag_col_main}, {RS_BANDI, (const void*)k_rag_band_inv},
              {RS_ROWI, (const void*)k_rag_row_inv}};
  for (auto& q : pers) {
    if (e == cudaSuccess) e = cudaFuncSetAttribute(q.k, A, int(max_smem(q.s)));
    int cap = 0;
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cap, q.k, kRagThreads, R->smem[q.s]);
    if (e == cudaSuccess) {
      if (cap < 1) e = cudaErrorInvalidConfiguration;
      else R->grid[q.s] = partition(items[q.s], weight[q.s], cap * (q.s == RS_COL ? sms - R->reserve : sms),
                                    T.lo[q.s]);
    }
  }
  int lo_prio = 0, hi_prio = 0;
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
  if (e == cudaSuccess) e = cudaStreamCreateWithPriority(&R->side, cudaStreamNonBlocking, lo_prio);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&R->join, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    ragged_destroy(R);
    return rfail(DSNU_ECUDA, std::string("one launch per stage: set-up: ") + cudaGetErrorString(e));
  }
  *out = R;
  return DSNU_OK;
}

dsnu_status ragged_enqueue(const Ragged* R, cudaStream_t st) {
  const bool pdl = R->pdl != 0;
  const RagTable& T = R->host;
  const dim3 b(kRagThreads);
  launch_k(pdl, k_rag_row_fwd, dim3(R->grid[RS_ROWF]), b, R->smem[RS_ROWF], st, T);
  // the column stage on `st`, the band chain on the side stream next to it
  cudaEventRecord(R->fork, st);
  cudaStreamWaitEvent(R->side, R->fork, 0);
  launch_k(pdl, k_rag_col_main, dim3(R->grid[RS_COL]), b, R->smem[RS_COL], st, T);
  cudaStream_t bs = R->side;
  launch_k(pdl, k_rag_band_fwd, dim3(R->grid[RS_BANDF]), b, R->smem[RS_BANDF], bs, T);
  launch_k(pdl, k_rag_interp, dim3(R->grid[RS_INTERP]), b, R->smem[RS_INTERP], bs, T);
  if (R->spread_cfg >= 0) {
#define DSNU_RAG_SPREAD(TL, SP, CH)                                                                         \
  launch_k(pdl, k_rag_spread<TL, SP, CH>, dim3(R->grid[RS_SPREAD]), dim3(TL * TL * SP), 0, bs, T);          \
  launch_k(pdl, k_rag_spread_reduce<TL>, dim3(R->grid[RS_REDUCE]), dim3(TL * TL), 0, bs, T)
    switch (R->spread_cfg) {
      case 1: DSNU_RAG_SPREAD(8, 2, 128); break;
      case 2: DSNU_RAG_SPREAD(16, 1, 128); break;
      case 3: DSNU_RAG_SPREAD(16, 2, 64); break;
      default: DSNU_RAG_SPREAD(8, 4, 128); break;
    }
#undef DSNU_RAG_SPREAD
  } else {
    // the plans' autotuners chose different tiles: the spreading pair per plan
    for (const RaggedGroupIn& gi : R->groups) {
      const dsnu_plan p = gi.plan;
      const WsLayout& L = p->ws_layout;
      Members m;
      m.dev = gi.dev_members;
      m.one = gi.first;
      m.count = gi.count;
      const WsOff off{L.off_A, L.off_B, L.off_Bband, L.off_Sband, L.off_c, L.off_partial, L.off_sched};
      launch_spread<float>(p->geom.spread_cfg, m, off, p->tab, p->geom, L.ldq, 0, bs, 2, pdl);
    }
  }
  launch_k(pdl, k_rag_band_inv, dim3(R->grid[RS_BANDI]), b, R->smem[RS_BANDI], bs, T);
  cudaEventRecord(R->join, bs);
  cudaStreamWaitEvent(st, R->join, 0);
  launch_k(pdl, k_rag_row_inv, dim3(R->grid[RS_ROWI]), b, R->smem[RS_ROWI], st, T);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return rfail(DSNU_ECUDA, std::string("one launch per stage: ") + cudaGetErrorString(e));
  return DSNU_OK;
}

int ragged_launches(const Ragged* R) { return R->spread_cfg >= 0 ? 8 : 6 + 2 * int(R->groups.size()); }

void ragged_destroy(Ragged* R) {
  if (!R) return;
  if (R->side) {
    cudaStreamSynchronize(R->side);
    cudaStreamDestroy(R->side);
  }
  if (R->fork) cudaEventDestroy(R->fork);
  if (R->join) cudaEventDestroy(R->join);
  delete R;
}

}  // namespace dsnu
