// internal.h -- plan layout shared by the host plan builder and the launchers.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>

#include "dsnufft.h"

namespace dsnu {

// Device tables of a plan.  Real-valued tables are in the plan's working
// precision (float for DSNU_MIXED, double for DSNU_FP64); node_D is FP64.
// The standard solver uses stw_x, stwc_x, stw_y, m_wx2 ((q_x dk_x)^2,
// q_x <= nx/2), m_kx and status only.
struct PlanTables {
  void* stw_x;    // cpx, FFT stage twiddles of length nx (fft_stage_tw_elems)
  void* stwc_x;   // cpx, the same in compact form (fft_stage_tw_elems_ct)
  void* twm_lo_x; // cpx, e^{-2 pi i n/Mx}, n < Lx = min(64, nx)
  void* twm_hi_x; // cpx, e^{-2 pi i Lx j/Mx}, j < nx/Lx
  void* decon_x;  // real, nx  phi_hat(0)/phi_hat(2 pi (n - nx/2)/Mx)
  void* stw_y;
  void* twm_lo_y;
  void* twm_hi_y;
  void* decon_y;
  void* m_wx2;    // real, nx + 1  (q_x dk_x)^2
  void* m_gx;     // real, nx + 1  1 - exp(-(q_x dk_x)^2/sigma^2)
  void* m_gy;     // real, n_gy    1 - exp(-(a dk_y)^2/sigma^2), a < n_gy
  void* m_kx;     // real, k_x per column for the sin 2theta term (0 at the Nyquist column); generic only
  int2* node_q0;  // n_nodes
  int* itile_ptr;   // n_itiles + 1: interpolation item -> range of itile_nodes
  int2* itile_org;  // n_itiles: the item's tile's first (q_x, q_y) (its nodes' stencil origins from there)
  int* itile_nodes; // n_nodes: node indices grouped by the tile of their stencil origin
  void* node_w;   // real, n_nodes * 2w (x weights then y weights)
  double* node_D; // n_nodes
  int* tile_items;  // n_tiles + 1: spreading tile -> range of work items
  int2* item_range; // per work item: [first, end) entry
  int* item_tile;   // per work item: its tile
  int* ent_node;  // per entry: node index
  int2* ent_q0;   // per entry: stencil origin of the node
  void* ent_w;    // real, per entry: the node's 2w ES weights
  int* status;    // one int
  void* m1tab;    // split plans with the DS multiplier: m1(q_x, |qbar_y|) in the plan's precision,
                  // (nx + 1) rows of ny + 4 entries, each row's even |qbar_y| first (MultTabs::m1); else NULL
};



// One density of a (possibly batched) launch: input, output and the base of
// its workspace (laid out by WsLayout).
struct Member {
  const double* rho;
  double* phi;
  char* ws;
};

// The members of a launch: `one` when count == 1, else a device array.
struct Members {
  const Member* dev;
  Member one;
  int count;
};

// Workspace layout (offsets in bytes from the workspace base).
struct WsLayout {
  // off_sched: the column pass's work counter (one int, reset by the forward row pass)
  size_t off_A, off_B, off_Bband, off_Sband, off_c, off_partial, off_sched, total;
  int ldqA, ldqB, ldq;  // q columns of the row-tiled A and B; band column length
};

struct PlanGeom {
  int nx, ny, mx, my, log2nx, log2ny;
  int log2lo_x, log2lo_y;  // two-level e^{-2 pi i n/M} tables
  int n_gy;                // entries of the short partition table
  double dky2;             // dk_y^2
  int cap_rowf, cap_col, cap_bandf, cap_bandi, cap_rowi;  // resident CTAs (SMs x occupancy)
  int rowi_bpf;            // inverse row pass prefetches the band values too (FP32)
  int row_pf;              // bit 0 forward row prefetch, bit 1 inverse, bit 2 rowi_bpf
  size_t smem_rowi;        // its dynamic shared memory per CTA
  int w, Q, n_nodes, n_tiles, tiles_x, tiles_y, max_tile_nodes, n_items;
  int n_itiles;            // interpolation items (at most kItileNodes nodes of one kItile x kItile tile)
  int spread_cfg;          // index into kSpreadCfgs (chosen by the autotuner)
  int spread_tile;         // its tile edge (cells)
  int precision, sharp;
  int acc64;     // mixed plans: Phi = I1 + I2 added in FP64 (dsnu_accumulation)
  int standard;  // 1: the standard periodic FFT solver (kappa = 1, p = 0; standard.cuh)
  int pdl;       // 1: pipeline kernels launched with programmatic dependent launch
  // multiplier |k|^alpha (a0 + ac cos 2theta + as sin 2theta) when m_generic (else -k_x^2/|k|^2)
  int m_generic, m_alpha;
  double m_a0, m_ac, m_as;
  double beta, sigma, cut_radius;
  double scale;  // 1/(Mx My) (split solver) or 1/(nx ny) (standard solver)
};

constexpr int kStages = 8;       // kernels per solve
constexpr int kProfEvents = kStages + 1;  // events per profiled solve (see run_pipeline)

// Concurrency of the band chain with the column pass: the band kernels run
// on `side` (a low-priority stream owned by the plan) while the column pass's
// persistent grid leaves `reserve` SMs free for them.
struct Overlap {
  cudaStream_t side;
  cudaEvent_t fork, join;
  int reserve;
};

// Launchers (one translation unit per precision).  `ev`, when not NULL,
// holds kProfEvents events recorded around the kernels (the kernels then run
// one after the other on `st`); `ov`, when not NULL, runs the band chain
// concurrently with the column pass.
dsnu_status run_pipeline_f32(const PlanGeom& g, const PlanTables& t, const WsLayout& L,
                             const Members& mem, cudaStream_t st, int cj, cudaEvent_t* ev,
                             const Overlap* ov = nullptr);
// Time one spreading configuration (spread + reduce, `reps` launches) on
// scratch buffers laid out by L; returns the average milliseconds in *ms.
cudaError_t time_spread_f32(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws, int reps,
                            float* ms);
cudaError_t time_spread_f64(const PlanGeom& g, const PlanTables& t, const WsLayout& L, void* ws, int reps,
                            float* ms);
dsnu_status run_pipeline_f64(const PlanGeom& g, const PlanTables& t, const WsLayout& L,
                             const Members& mem, cudaStream_t st, int cj, cudaEvent_t* ev,
                             const Overlap* ov = nullptr);

// A single density as a one-member launch.
inline Members single_member(const double* rho, double* phi, void* ws) {
  Members m;
  m.dev = nullptr;
  m.one.rho = rho;
  m.one.phi = phi;
  m.one.ws = static_cast<char*>(ws);
  m.count = 1;
  return m;
}
// Set the kernels' shared-memory limits and compute persistent grid sizes.
cudaError_t prepare_kernels_f32(PlanGeom& g);
cudaError_t prepare_kernels_f64(PlanGeom& g);

// A batch's plans solved by one launch per pipeline stage (batch_ragged.cu):
// one entry per distinct plan with its members' device table.
constexpr int kRagMaxGroups = 8;
struct RaggedGroupIn {
  dsnu_plan plan;
  const Member* dev_members;  // count members (device)
  Member first;               // the first of them (for one-member groups)
  int count;
};
struct Ragged;
// Whether these plans can share stage launches (why not, in *why).
bool ragged_eligible(const dsnu_plan* plans, int n, std::string* why);
// Build the stage table (host memory; the stage launches pass it by value).
dsnu_status ragged_create(const RaggedGroupIn* groups, int n, Ragged** out);
dsnu_status ragged_enqueue(const Ragged* r, cudaStream_t st);
int ragged_launches(const Ragged* r);  // kernel launches per batch solve
void ragged_destroy(Ragged* r);

void set_last_error(const std::string& msg);

}  // namespace dsnu

struct dsnu_plan_s {
  dsnu_params prm;          // resolved parameters
  dsnu::PlanGeom geom;
  dsnu::PlanTables tab;
  dsnu::WsLayout ws_layout;
  void* table_block;        // one device allocation holding every table but the spreading ones
  void* spread_block;       // spreading tables of the chosen tile configuration
  void* m1_block;           // PlanTables::m1tab
  size_t table_bytes;
  void* ws;                 // caller-owned workspace
  size_t ws_bytes;
  cudaEvent_t* prof_events; // profiling: max_solves * kProfEvents events, or NULL
  int prof_max, prof_used;
  // streaming host solves (dsnu_solve_host_stream): two copy streams and the
  // per-slot events, created on first use
  bool has_copy_streams;
  cudaStream_t copy_in, copy_out;
  cudaEvent_t ev_start, ev_in[2], ev_solved[2], ev_out[2];
  dsnu::Overlap overlap;    // band chain next to the column pass (reserve 0: off)
};
