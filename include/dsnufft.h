/*
 * dsnufft.h -- C ABI of the GB300 (sm_103a) split nonlocal potential solver.
 *
 * Operation (Mauser, Stimming, Zhang, "A novel nonlocal potential solver based
 * on nonuniform FFT for efficient simulation of the Davey-Stewartson
 * equations", Sec. 2.1):
 *
 *     Phi = F^-1[ -k_x^2 / |k|^2  rho_hat ]           (eqs. Def_Fourier, FourTransDef)
 *         = I1 + I2                                   (eqs. PotSplitWhoSpace, SubInt1, SubInt2)
 *
 *   I1: zero-padded (kappa = 2) uniform FFT of rho, multiplied by
 *       (1 - p(k)) (-k_x^2/|k|^2), inverse FFT, restricted to the grid.
 *   I2: polar Gauss quadrature over the disk |k| <= P (eq. I2PolarDisc):
 *       rho_hat at radial Gauss-Legendre x uniform angular nodes by a type-2
 *       NUFFT (eq. 2.2), weights -cos^2(theta) r w_r w_theta p(r) (2 pi)^-2,
 *       and a type-1 NUFFT back onto the grid (eq. 2.1).
 *   p(k) = exp(-|k|^2 / sigma^2) (Sec. 2.1).  Frequencies are angular
 *   (rad/length); the grid is x_n = -L + n h, n = 0..N-1, h = 2L/N, periodic.
 *
 * Conventions shared by every entry point:
 *   - Arrays are row-major [ny][nx] (x fastest), i.e. a (ny, nx) tensor.
 *   - Pointers named *_dev are DEVICE pointers; the caller owns them.
 *   - Calls that take a stream enqueue work on it and return at once
 *     (stream == NULL means the legacy default stream).  Only the calls that
 *     build or free state wait for the GPU (dsnu_plan_create and
 *     dsnu_ds_plan_create for their table uploads, dsnu_batch_bind for its
 *     member tables, the destroy calls for the plan's own streams), besides
 *     dsnu_profile_end and dsnu_status_poll, which read results back.
 *   - Errors: every call returns a dsnu_status.  Invalid arguments give
 *     DSNU_EINVAL before any launch.  dsnu_last_error() returns a
 *     thread-local message for the last failing call on this thread.
 *     Nothing exits the process and nothing throws across the ABI.
 */
#ifndef DSNUFFT_H
#define DSNUFFT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DSNU_OK = 0,
  DSNU_EINVAL = 1,        /* invalid argument (nothing was launched) */
  DSNU_ENOMEM = 2,        /* a plan table allocation failed */
  DSNU_ECUDA = 3,         /* a CUDA runtime call failed; see dsnu_last_error() */
  DSNU_ETIMEOUT = 4,      /* a bounded device-side wait gave up */
  DSNU_EUNSUPPORTED = 5   /* valid request outside what the library supports */
} dsnu_status;

typedef enum {
  DSNU_FP64 = 0,   /* every step in FP64 */
  DSNU_MIXED = 1   /* FFT butterflies, ES spreading/interpolation in FP32;
                      nodes, weights, twiddle/phase tables generated in FP64;
                      the per-node low-frequency weighting in FP64; the final
                      accumulation Phi = I1 + I2 in FP64 (dsnu_accumulation);
                      rho in and Phi out are FP64 */
} dsnu_precision;

/* How a mixed plan forms Phi = I1 + I2 (eq. PotSplitWhoSpace) from the two
 * FP32 terms of its last pass.  FP64 plans always work in FP64. */
typedef enum {
  DSNU_ACCUM_FP64 = 0,    /* each term widened to FP64 (exactly) and added in FP64 */
  DSNU_ACCUM_WORKING = 1  /* added in FP32, the sum widened at the store */
} dsnu_accumulation;

typedef enum {
  DSNU_PARTITION_GAUSS = 0,  /* p(k) = exp(-|k|^2/sigma^2) (Sec. 2.1) */
  DSNU_PARTITION_SHARP = 1,  /* p(k) = 1 on |k| <= P, 0 outside */
  DSNU_PARTITION_NONE = 2    /* p = 0 with pad_factor = 1: the standard periodic
                                FFT solver the paper compares against (Sec. 2.1,
                                Table 1): Phi = IDFT[-k_x^2/|k|^2 DFT(rho)] on
                                the unpadded grid, value 0 at k = 0, dk = pi/l.
                                cut_radius, sigma, n_r, n_theta, kernel_width
                                are ignored. */
} dsnu_partition;

typedef enum {
  DSNU_RADIAL_LEGENDRE = 0,  /* Gauss-Legendre on [0, P], the Jacobian r in the weights */
  DSNU_RADIAL_JACOBI = 1     /* Gauss-Jacobi for the weight (1 + t) on [-1, 1], i.e.
                                the Jacobian r itself (Sec. 2.1) */
} dsnu_radial_rule;

/* Solver parameters (Sec. 2.1).  Zero-valued optional fields take defaults. */
typedef struct {
  int32_t nx, ny;          /* grid points per axis: powers of two, 16..4096 */
  double  lx, ly;          /* half-widths: domain [-lx,lx) x [-ly,ly), h = 2l/n */
  double  cut_radius;      /* P: disk radius of the polar part, rad/length.
                              Needs P*h + w*pi/(2n) < pi on both axes so that
                              the disk plus the ES stencil lies inside the
                              padded frequency grid. */
  double  sigma;           /* partition width; 0 => P/6 (p(P) = e^-36) */
  int32_t n_r, n_theta;    /* radial Gauss-Legendre x uniform angular nodes;
                              n_theta even (node set symmetric under k -> -k) */
  int32_t kernel_width;    /* ES kernel width w in fine-grid cells, 2..16;
                              0 => 15 (FP64) or 8 (MIXED) */
  int32_t pad_factor;      /* kappa; 0 or 2 for the split solver, 1 (and only 1)
                              with DSNU_PARTITION_NONE */
  int32_t precision;       /* dsnu_precision */
  int32_t partition;       /* dsnu_partition */
  int32_t radial_rule;     /* dsnu_radial_rule of the polar quadrature */
  int32_t accumulation;    /* dsnu_accumulation of mixed plans; 0 = FP64 */
} dsnu_params;

typedef struct dsnu_plan_s* dsnu_plan;

/* A Fourier multiplier of the family (the Remark of Sec. 2.2: the split
 * applies to any multiplier given analytically)
 *     m(k) = |k|^alpha (a0 + a_cos cos 2theta + a_sin sin 2theta),  theta = arg k,
 * alpha in {-1, 0, 1}, m(0) = 0 in the I1 part.  The DS multiplier -k_x^2/|k|^2
 * is (0, -1/2, -1/2, 0); 2 pi/|k| (alpha = -1, a0 = 2 pi) is the 2D
 * transform of the 3D Coulomb kernel 1/|x|; |k| (alpha = 1) the half
 * Laplacian.  The split needs m (1 - p) continuous at 0 (alpha > -2) and
 * m p r smooth in polar coordinates (alpha >= -1). */
typedef struct {
  int32_t alpha;
  int32_t reserved;  /* set to 0 */
  double a0, a_cos, a_sin;
} dsnu_multiplier;

/* Build a plan: validates params, computes (FP64, on the host) the polar
 * Gauss nodes and weights, the ES kernel weights of every node, the
 * deconvolution and multiplier tables and the twiddle tables, bins the nodes
 * into spreading tiles, and uploads the tables with cudaMemcpyAsync on
 * `stream` (cudaStream_t, may be NULL), then synchronises that stream.
 * The spreading tile configuration is chosen by timing the candidates on the
 * device (temporary scratch, cached per device and parameters for the
 * process); DSNU_AUTOTUNE=0 in the environment keeps the default one.
 * Plans with the DS multiplier also tabulate the column multiplier
 * m1(q_x, |qbar_y|) of I1 on the device in FP64, stored in the plan's
 * precision ((nx + 1) (ny + 4) entries: 67 MB mixed, 134 MB FP64 at
 * 4096 x 4096).
 * Ownership: the plan owns its tables (device memory, freed by
 * dsnu_plan_destroy); it does not own the workspace.
 * Errors: DSNU_EINVAL (bad params, *out untouched), DSNU_ENOMEM, DSNU_ECUDA. */
dsnu_status dsnu_plan_create(const dsnu_params* params, void* stream, dsnu_plan* out);

/* dsnu_plan_create for another multiplier of the family above: the column
 * pass of I1 (and of the standard solver) applies m (1 - p), the polar
 * weights carry r^alpha (a0 + a_cos cos 2theta + a_sin sin 2theta) in place of
 * -cos^2 theta.  mult == NULL is dsnu_plan_create.  The operator stays real and
 * symmetric, so dsnu_solve_adjoint and the batch and no-alloc entry points
 * apply unchanged.  Errors: those of dsnu_plan_create, and DSNU_EINVAL for
 * alpha outside {-1, 0, 1} or non-finite coefficients. */
dsnu_status dsnu_plan_create_multiplier(const dsnu_params* params, const dsnu_multiplier* mult, void* stream,
                                        dsnu_plan* out);

/* Bytes of device scratch one solve needs (intermediate spectra).  0 on a
 * NULL plan. */
size_t dsnu_workspace_bytes(dsnu_plan plan);

/* Attach caller-owned device scratch of at least dsnu_workspace_bytes(plan)
 * bytes, 256-byte aligned.  The plan keeps the pointer until it is replaced
 * or the plan is destroyed; the caller must keep the memory alive and must
 * not run two solves of the same plan concurrently (they share it).
 * Errors: DSNU_EINVAL (NULL plan/pointer, too small, misaligned). */
dsnu_status dsnu_set_workspace(dsnu_plan plan, void* workspace_dev, size_t bytes);

/* Phi = I1 + I2 (Sec. 2.1, eq. PotSplitWhoSpace) for one density.
 * For mixed plans on grids of at least 2048 x 2048 the band chain (the NUFFT
 * part) runs on a low-priority stream owned by the plan, concurrently with the
 * column pass of I1, which then leaves 12 of every 152 SMs free
 * (DSNU_BAND_SMS=<n> in the environment at plan creation sets the number of
 * SMs, 0 runs everything on `stream`); the plan orders that stream after
 * `stream`'s earlier work and `stream` after it, so the call behaves as if
 * everything ran on `stream`.
 * rho_dev: [ny][nx] FP64 density (device, read only).
 * phi_dev: [ny][nx] FP64 potential (device, written); must not alias rho_dev.
 * Both 16-byte aligned (every cudaMalloc'd or torch-allocated buffer is).
 * Enqueued on `stream` (cudaStream_t or NULL).
 * Errors: DSNU_EINVAL (NULL/aliased/misaligned pointers, no workspace),
 * DSNU_ECUDA (a launch failed). */
dsnu_status dsnu_solve(dsnu_plan plan, const double* rho_dev, double* phi_dev, void* stream);

/* Transpose of the discrete operator of dsnu_solve: the same pipeline with
 * every transform conjugated, i.e. the transposed type-1/type-2 pair (type-1
 * of the transpose = type-2 with e^{+i k.x}, and the reverse) around the same
 * real weights, and the transposed padded FFT part.  The operator is
 * symmetric (real even multiplier, node set symmetric under k -> -k), so the
 * result equals dsnu_solve(g) up to rounding.  Same layout, ownership and
 * errors as dsnu_solve. */
dsnu_status dsnu_solve_adjoint(dsnu_plan plan, const double* g_dev, double* out_dev, void* stream);

/* Read and clear the plan's device status word (written by bounded device
 * waits); synchronises `stream`.  Returns DSNU_OK or the recorded status. */
dsnu_status dsnu_status_poll(dsnu_plan plan, void* stream);

/* Free the plan's tables.  The caller must make sure no work that uses the
 * plan is still in flight.  NULL is accepted (DSNU_OK). */
dsnu_status dsnu_plan_destroy(dsnu_plan plan);

/* Thread-local message of the last failing call on this thread ("" if none). */
const char* dsnu_last_error(void);

/* Host-buffer variant of dsnu_solve (end-to-end use): enqueues on `stream`
 * the copy rho_host -> rho_dev, the solve into phi_dev, and the copy
 * phi_dev -> phi_host, and returns at once; phi_host is valid after the
 * stream is synchronised.  rho_host/phi_host: [ny][nx] FP64 host memory
 * (page-locked for the copies to be asynchronous); rho_dev/phi_dev:
 * caller-owned [ny][nx] FP64 device staging buffers (16-byte aligned).
 * Same errors as dsnu_solve, returned before anything is enqueued. */
dsnu_status dsnu_solve_host(dsnu_plan plan, const double* rho_host, double* phi_host,
                            double* rho_dev, double* phi_dev, void* stream);

/* Many host densities through one plan with the copies overlapped (the
 * streaming form of dsnu_solve_host): for i = 0 .. count-1, rho_host[i] is
 * copied into one of two device staging slots, solved on `stream`, and the
 * result copied back to phi_host[i].  The upload of density i+1 and the
 * download of result i-1 run on two copy streams owned by the plan while
 * density i is solved.  rho_host[i], phi_host[i]: host arrays of ny*nx
 * doubles ([ny][nx]); pinned memory (cudaHostAlloc / cudaHostRegister) keeps
 * the copies asynchronous; a buffer may appear several times (a phi_host
 * buffer receives the results in order).  staging_dev: caller-owned device
 * memory of at least dsnu_stream_staging_bytes(plan) bytes, 256-byte aligned
 * (two density and two potential slots).  The solves use the plan's
 * workspace.  Asynchronous: on return everything is enqueued and `stream` is
 * ordered after the last download, so synchronising `stream` completes the
 * batch; the caller must not touch the host or staging buffers before that.
 * Errors: DSNU_EINVAL (NULL arguments, count < 1, staging too small or
 * misaligned, no workspace), DSNU_ECUDA. */
size_t dsnu_stream_staging_bytes(dsnu_plan plan);
dsnu_status dsnu_solve_host_stream(dsnu_plan plan, int32_t count, const double* const* rho_host,
                                   double* const* phi_host, void* staging_dev, size_t staging_bytes,
                                   void* stream);

/* Per-kernel timing.  After dsnu_profile_begin(plan, max_solves), each of the
 * next max_solves solves of this plan records CUDA events on its stream
 * before its first kernel and after each of its dsnu_stage_count() kernels.
 * dsnu_profile_end synchronises those events, adds the elapsed time of
 * every stage over the recorded solves into stage_ms[0 .. n_stages) (ms),
 * writes the number of recorded solves to *n_solves, and frees the events.
 * Errors: DSNU_EINVAL (bad arguments, profiling already active / not active),
 * DSNU_ECUDA. */
dsnu_status dsnu_profile_begin(dsnu_plan plan, int max_solves);
dsnu_status dsnu_profile_end(dsnu_plan plan, double* stage_ms, int n_stages, int* n_solves);

/* The radial rule of the polar quadrature (eq. I2PolarDisc), host only, no
 * device needed: n_r nodes r[i] in (0, cut_radius), ascending, and weights
 * w[i] with sum_i w[i] f(r[i]) ~ int_0^P f(r) r dr (the polar Jacobian
 * included), exact for f a polynomial of degree 2 n_r - 2 (Legendre) or
 * 2 n_r - 1 (Jacobi).  r and w: caller-owned host arrays of n_r doubles.
 * Errors: DSNU_EINVAL (n_r outside [1, 4096], cut_radius <= 0, NULL arrays,
 * unknown rule). */
dsnu_status dsnu_radial_nodes(int32_t n_r, int32_t rule, double cut_radius, double* r, double* w);

/* Parameters for a target accuracy eps of the split solver (host only): the
 * partition width sigma = 12 / min(lx, ly) (sigma = O(1/L), Sec. 2.1: the
 * padded uniform grid resolves the transition of 1 - p), the disk radius
 * P = sigma sqrt(ln(1/eps)) (p(P) = eps), and polar node counts that grow
 * with the largest phase P R of e^{i k.x} on the disk, R = sqrt(lx^2 + ly^2):
 * n_theta = the multiple of 4 >= P R + 16, n_r = the multiple of 8 >= P R/2 + 4
 * (measured on the closed-form Gaussian of Sec. 3 for eps = 1e-6..1e-14),
 * with the Gauss-Jacobi radial rule and the default ES width.  eps is clamped
 * to [1e-15, 1e-2] (FP64) or [1e-7, 1e-2] (MIXED).
 * Errors: DSNU_EINVAL (bad sizes or eps; or the grid is too coarse for the
 * disk plus the ES stencil), *out untouched. */
dsnu_status dsnu_params_auto(int32_t nx, int32_t ny, double lx, double ly, double eps, int32_t precision,
                             dsnu_params* out);

/* Number of kernels one solve launches, and their names (static strings). */
int32_t dsnu_stage_count(void);
const char* dsnu_stage_name(int32_t stage);

/* Solve without any device allocation by the caller or the library.
 * The paper has no counterpart: this entry point exists for callers that
 * cannot call cudaMalloc (or any allocating routine) when they solve, e.g.
 * code running under an allocator that forbids new device allocations, or a
 * host loop that must not allocate after start-up.  It computes exactly what
 * dsnu_solve computes, but its scratch is a fixed array compiled into the
 * library (dsnu_noalloc_scratch_bytes() = 32 MiB on every GPU that loads the
 * library, held until the process exits) instead of the plan's workspace; no
 * workspace needs to be attached.  Enough for grids up to 1024 x 1024 in
 * either precision; a plan needing more scratch gets DSNU_EINVAL with a
 * message naming both sizes.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call on a device shares the one array,
 * which keeps the previous call's contents (nothing in it needs clearing):
 * calls whose work overlaps on the GPU (other streams, other threads, other
 * plans) race on it and must be serialised by the caller.
 * rho_dev, phi_dev, stream: as in dsnu_solve.  Errors: as dsnu_solve, plus
 * DSNU_EINVAL when the plan needs more than the static scratch. */
dsnu_status dsnu_solve_noalloc(dsnu_plan plan, const double* rho_dev, double* phi_dev, void* stream);

/* Size in bytes of the static scratch used by dsnu_solve_noalloc. */
size_t dsnu_noalloc_scratch_bytes(void);

/* ---------------------------------------------------------------------------
 * Split-step pieces of the DS time loop (Sec. 2.3, time-splitting spectral
 * method).  A DS plan holds the unpadded N x N periodic transform of the wave
 * function u on [-lx,lx) x [-ly,ly); u is interleaved complex [ny][nx]
 * (complex64 when precision = DSNU_MIXED, complex128 when DSNU_FP64).
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t nx, ny;    /* powers of two, 16..4096 */
  double  lx, ly;    /* half-widths */
  int32_t precision; /* dsnu_precision: DSNU_MIXED (complex64) or DSNU_FP64 (complex128) */
  int32_t reserved;
} dsnu_ds_params;

typedef struct dsnu_ds_plan_s* dsnu_ds_plan;

/* Build the transform tables (FP64 on the host, uploaded on `stream`, which is
 * then synchronised).  Errors: DSNU_EINVAL, DSNU_ENOMEM, DSNU_ECUDA. */
dsnu_status dsnu_ds_plan_create(const dsnu_ds_params* params, void* stream, dsnu_ds_plan* out);

/* Load the phases of the linear flow over a step tau (eqs. 1st_tssp,
 * 1st_tssp_more): e^{-i tau (k_x^2 - alpha k_y^2)}, k angular wave numbers of
 * the periodic grid.  A small kernel on `stream` evaluates them in FP64 (no
 * host round trip, no synchronisation) unless the same (tau, alpha) is
 * already loaded; later dsnu_ds_linear calls must use the same stream (or be
 * ordered after it).  Errors: DSNU_EINVAL (NULL plan, non-finite values),
 * DSNU_ECUDA (launch failed). */
dsnu_status dsnu_ds_set_linear_step(dsnu_ds_plan plan, double tau, double alpha, void* stream);

/* u <- F^-1[ e^{-i tau (k_x^2 - alpha k_y^2)} F[u] ] in place (the exact
 * linear flow); adjoint != 0 applies the conjugate phases, i.e. the inverse
 * (= adjoint, the flow is unitary) propagator.  Errors: DSNU_EINVAL (no step
 * loaded), DSNU_ECUDA. */
dsnu_status dsnu_ds_linear(dsnu_ds_plan plan, void* u_dev, int32_t adjoint, void* stream);

/* rho <- |u|^2 (FP64 [ny][nx], device), the density of eq. DSII_exact_pot. */
dsnu_status dsnu_ds_abs2(dsnu_ds_plan plan, const void* u_dev, double* rho_dev, void* stream);

/* Vector-Jacobian product of rho = |u|^2 (the last link of the adjoint of
 * Phi(|u|^2) with respect to u): grad_u = 2 g_rho u for a real loss, in the
 * d/dRe + i d/dIm convention.  u_dev and grad_dev: the plan's complex type
 * [ny][nx] (may alias); g_rho_dev: FP64 [ny][nx] (e.g. dsnu_solve_adjoint of
 * the gradient at Phi).  Errors: DSNU_EINVAL (NULL argument), DSNU_ECUDA. */
dsnu_status dsnu_ds_abs2_vjp(dsnu_ds_plan plan, const void* u_dev, const double* g_rho_dev, void* grad_dev,
                             void* stream);

/* Nonlinear flow with the density and Phi frozen over a step (eqs. 2nd_tssp,
 * 2nd_tssp_more): u <- u e^{i tau (2 beta |u|^2 + 4 beta Phi)} in place;
 * phi_dev: FP64 [ny][nx] potential of the current density. */
dsnu_status dsnu_ds_nonlinear(dsnu_ds_plan plan, void* u_dev, const double* phi_dev, double tau,
                              double beta, void* stream);

/* Vector-Jacobian product of the nonlinear flow u' = u e^{i theta}, theta =
 * tau (2 beta |u|^2 + 4 beta Phi(|u|^2)), for a real loss with gradients in
 * the d/dRe + i d/dIm convention.  Given u (the step's input), Phi and g' (the
 * gradient at u'), writes part = g' e^{-i theta} (complex, like u) and s =
 * Im(g' conj u') (FP64); the caller forms A^T s with dsnu_solve_adjoint and
 * calls dsnu_ds_nonlinear_vjp_finish, which turns part into
 *   grad_u = part + 2 tau (2 beta s + 4 beta A^T s) u. */
dsnu_status dsnu_ds_nonlinear_vjp(dsnu_ds_plan plan, const void* u_dev, const double* phi_dev,
                                  const void* g_dev, double tau, double beta, double* s_dev,
                                  void* part_dev, void* stream);
dsnu_status dsnu_ds_nonlinear_vjp_finish(dsnu_ds_plan plan, const void* u_dev, const double* s_dev,
                                         const double* ats_dev, double tau, double beta,
                                         void* grad_dev, void* stream);

dsnu_status dsnu_ds_plan_destroy(dsnu_ds_plan plan);

/* ---------------------------------------------------------------------------
 * Batches: many densities, possibly on different grids, per launch sequence.
 * Members that share a plan are solved together (each kernel runs once for the
 * group, its CTAs iterating over members and work items).  Distinct plans are
 * scheduled in one of two ways (dsnu_batch_set_schedule):
 *   - one launch per pipeline stage for all plans, eight launches per batch
 *     solve, each plan's members on their own range of the stage's persistent
 *     CTAs, the band chain on a plan-owned side stream next to the column
 *     stage (mixed-precision split plans with the DS multiplier, grids of 256
 *     to 2048 points per axis, at most 8 distinct plans; when the plans'
 *     spreading autotuners chose different tiles, the two spreading kernels
 *     run once per plan instead);
 *   - one launch sequence per distinct plan on forked streams (any plans).
 * With forked streams every member's result is bitwise identical to its own
 * dsnu_solve (the same kernels).  The stage launches run the same kernel
 * bodies compiled into other kernels, where the compiler may contract
 * multiply-adds differently: results equal the member's dsnu_solve to FP32
 * rounding, and repeated batch solves are bitwise reproducible.
 * ------------------------------------------------------------------------- */
typedef struct dsnu_batch_s* dsnu_batch;

typedef enum {
  DSNU_BATCH_AUTO = 0,            /* the faster for this GPU: forked streams (measured on GB300: the 64-member
                                     batch of 256^2 .. 2048^2 grids in 3.26 ms, against 3.43 ms with one
                                     launch per stage, whose stages end for all grid sizes at once) */
  DSNU_BATCH_STAGE_LAUNCHES = 1,  /* one launch per stage (DSNU_EUNSUPPORTED when the plans do not allow it) */
  DSNU_BATCH_FORKED_STREAMS = 2   /* one launch sequence per distinct plan on forked streams */
} dsnu_batch_schedule_kind;

/* count members; plans[i] is member i's plan (plans may repeat).  The batch
 * keeps the plan handles: they must outlive it.  Creates one stream and one
 * event per distinct plan and a small device table per plan.
 * Errors: DSNU_EINVAL, DSNU_ECUDA. */
dsnu_status dsnu_batch_create(int32_t count, const dsnu_plan* plans, dsnu_batch* out);

/* Device scratch for all members (sum of the members' workspaces, 256-byte
 * aligned each). */
size_t dsnu_batch_workspace_bytes(dsnu_batch b);

/* Bind the members' device buffers: rho_dev[i] (FP64 [ny_i][nx_i], read) and
 * phi_dev[i] (written), both 16-byte aligned, and the caller-owned batch workspace (>=
 * dsnu_batch_workspace_bytes, 256-byte aligned).  Uploads the member tables
 * on `stream` and synchronises it (and builds the host table of the
 * one-launch-per-stage schedule when it is used); drops a previously captured
 * graph.
 * Errors: DSNU_EINVAL, DSNU_EUNSUPPORTED (DSNU_BATCH_STAGE_LAUNCHES was asked
 * for plans that do not allow it), DSNU_ECUDA. */
dsnu_status dsnu_batch_bind(dsnu_batch b, const double* const* rho_dev, double* const* phi_dev,
                            void* workspace_dev, size_t bytes, void* stream);

/* Choose how the batch's distinct plans are scheduled (dsnu_batch_schedule_kind;
 * a new batch uses DSNU_BATCH_AUTO).  Host only: once the batch is bound, the
 * one-launch-per-stage schedule's table (CTA ranges per plan and stage, the
 * plans' table pointers) is built in host memory and passed by value to the
 * stage launches.  Drops a previously captured graph.
 * Errors: DSNU_EINVAL (NULL batch, unknown schedule), DSNU_EUNSUPPORTED
 * (DSNU_BATCH_STAGE_LAUNCHES for plans that do not allow it; the previous
 * schedule stays), DSNU_ECUDA. */
dsnu_status dsnu_batch_set_schedule(dsnu_batch b, int32_t schedule);

/* The schedule in use (DSNU_BATCH_STAGE_LAUNCHES or DSNU_BATCH_FORKED_STREAMS),
 * and the number of kernel launches of one batch solve; -1 before
 * dsnu_batch_bind or for a NULL batch. */
int32_t dsnu_batch_schedule(dsnu_batch b);
int32_t dsnu_batch_launches(dsnu_batch b);

/* Capture the batch's launch sequence (the stage launches, or all groups'
 * sequences with the forked streams joined back to `stream`) into a CUDA
 * graph, instantiated once; dsnu_batch_solve then replays it.  `stream` must
 * not be capturing already. */
dsnu_status dsnu_batch_capture_graph(dsnu_batch b, void* stream);

/* Solve every member: graph replay when captured, else the launches.  Only
 * launches (no allocation, no synchronisation). */
dsnu_status dsnu_batch_solve(dsnu_batch b, void* stream);

/* Free the batch (no solve of it may be in flight).  NULL is accepted. */
dsnu_status dsnu_batch_destroy(dsnu_batch b);

/* Plan introspection for tests and benchmarks (host values, no device work). */
typedef struct {
  int32_t n_nodes;       /* n_r * n_theta */
  int32_t band_q;        /* Q: band half-width in fine-grid cells */
  int32_t kernel_width;  /* resolved ES width */
  int32_t precision;
  double  sigma;         /* resolved partition width */
  double  es_beta;       /* ES shape parameter */
  int32_t n_tiles;       /* spreading tiles */
  int32_t max_tile_nodes;
  int32_t n_items;       /* spreading work items (tiles cut into pieces) */
  int32_t spread_tile;   /* spreading configuration chosen at plan creation: */
  int32_t spread_split;  /*   tile edge (cells), threads per cell, entries per item */
  int32_t spread_chunk;
  int32_t row_prefetch;  /* FP32 row passes: bit 0 the forward pass prefetches rho,
                            bit 1 the inverse pass prefetches its spectra, bit 2 also
                            its band values (by grid size and what fits in shared memory) */
  int32_t reserved;
} dsnu_plan_info;

dsnu_status dsnu_plan_get_info(dsnu_plan plan, dsnu_plan_info* info);

#ifdef __cplusplus
}
#endif

#endif /* DSNUFFT_H */
