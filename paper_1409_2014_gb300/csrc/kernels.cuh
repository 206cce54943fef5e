// kernels.cuh -- the split-solver pipeline for one density (Sec. 2.1).
//
// Notation: N x N physical grid (nx, ny), padded/fine grid M = 2N per axis,
// natural frequency index q in [0, M) with signed value q - M for q >= N.
// Per solve, with rho real:
//
//   k_row_fwd : per row, z = rho + i b with b = rho dx(x) dy(y) (ES
//               deconvolution, the type-2 prefactor); one length-M DFT of the
//               zero-padded z (two length-N DFTs: even and odd q); the two
//               real-signal spectra are separated: A = row DFT of rho for q in
//               [0, N], B = row DFT of b for q in [0, Q].   [I1 and eq. 2.2 prep]
//   k_col_main: per column q_x in [0, N] of A: column DFT (length M, N inputs),
//               times m1 = (1 - p) (-k_x^2/|k|^2) (eq. SubInt1), inverse
//               column DFT keeping N rows; in place.               [I1]
//   k_band_fwd: per column q_x in [0, Q] of B: column DFT, keep |q_y| <= Q.
//   k_interp_tile: rho_hat(k_j) = sum over the w x w ES stencil of the band
//               (type-2 NUFFT, eq. 2.2); c_j = D_j rho_hat_j with the polar
//               weights of eq. I2PolarDisc (FP64 multiply); per tile of
//               stencil origins, the band values it reaches staged in shared
//               memory.
//   k_spread  : S(q) = sum_j c_j phi(u_j - q) on the band (type-1 NUFFT
//               spreading, eq. 2.1), gathered per tile from a node list
//               (no atomics).
//   k_band_inv: per band column: inverse column DFT of S, N rows.
//   k_row_inv : per row: one inverse length-M DFT of W = Y + i S
//               (Hermitian extension of both), keeping N points;
//               Phi = [Re T + Im T dx dy] / (Mx My)   (I1 + I2, eq. PotSplitWhoSpace;
//               in mixed plans each term widened to FP64 and the sum formed in FP64).
//
// Intermediate spectra (A, B and the inverse band columns) are stored
// row-tiled: element (row iy, column q) at [iy / TR][q][iy % TR] with TR rows
// of 32 bytes per tile segment (TR = 4 complex floats or 2 complex doubles),
// so that the row passes (TR rows per CTA) and the column passes (one column
// per CTA) both move whole 32-byte sectors.
//
// `cj` = 1 runs the same pipeline with every complex constant conjugated
// (DFT signs, the packing unit i, the centring phases): for real input this is
// the transposed operator (type-1 <-> type-2 transposed pair), see
// dsnu_solve_adjoint.
#pragma once

#include "common.cuh"
#include "internal.h"

// Occupancy targets (minimum resident CTAs per SM) and rows per CTA of the
// FP32 row passes; overridable at compile time for tuning sweeps.
#ifndef DSNU_ROW_MINB
#define DSNU_ROW_MINB 2
#endif
#ifndef DSNU_COL_MINB
#define DSNU_COL_MINB 2
#endif
#ifndef DSNU_ROWF_RB32
#define DSNU_ROWF_RB32 2
#endif
#ifndef DSNU_ROWI_RB32
#define DSNU_ROWI_RB32 2
#endif
// Forward row pass: bulk prefetch of the next rows of rho (FP32 plans), with
// the landing rows N + DSNU_ROWF_LPAD doubles apart
#ifndef DSNU_ROWF_PF
#define DSNU_ROWF_PF 1
#endif
#ifndef DSNU_ROWF_LPAD
#define DSNU_ROWF_LPAD 8
#endif
// Inverse row pass: the band values prefetched with the row pair when they
// fit (BPF); asynchronous prefetch of the next row pair of A (FP32, PF)
#ifndef DSNU_ROWI_BPF
#define DSNU_ROWI_BPF 1
#endif
#ifndef DSNU_ROWI_PF
#define DSNU_ROWI_PF 1
#endif
// Column pass: the next column loaded into registers during the current
// inverse transform
#ifndef DSNU_COL_REGPF
#define DSNU_COL_REGPF 1
#endif
#ifndef DSNU_TILE_LT32
#define DSNU_TILE_LT32 2
#endif
#ifndef DSNU_COLMAIN_MINB
#define DSNU_COLMAIN_MINB 1
#endif

namespace dsnu {

template <typename R>
struct AxisTabs {
  const cpx<R>* stw;     // FFT stage twiddles (fft_stage_twiddles), copied to shared memory
  const cpx<R>* twm_lo;  // e^{-2 pi i n/M}, n < L  (L = min(64, N))
  const cpx<R>* twm_hi;  // e^{-2 pi i L j/M}, j < N/L
  int log2lo;            // log2 L
  const R* decon;        // phi_hat(0) / phi_hat(2 pi (n - N/2)/M), n < N
  const cpx<R>* stwc;    // compact stage twiddles (fft_stage_tw_elems_ct); x axis only
};

// e^{-2 pi i n/M} for n < N from the two short tables (one complex product).
template <typename R>
__device__ __forceinline__ cpx<R> twm(const AxisTabs<R>& a, int n) {
  return cmul(a.twm_hi[n >> a.log2lo], a.twm_lo[n & ((1 << a.log2lo) - 1)]);
}

template <typename R>
struct MultTabs {
  const R* wx2;       // (q_x dk_x)^2, q_x in [0, nx]
  const R* gx;        // 1 - exp(-(q_x dk_x)^2 / sigma^2)
  int n_gy;           // 1 - exp(-(a dk_y)^2 / sigma^2) rounds to 1 for a = |qbar_y| >= n_gy
  R inv_sigma2;       // 1 / sigma^2
  R neg_dky2_s2_log2e;  // -dk_y^2 / (sigma^2 ln 2)
  R dky2;             // dk_y^2
  int half_my;        // N_y (= M_y / 2)
  int sharp;          // 1: p = indicator of |k| <= P
  R cut2;             // P^2
  // another multiplier |k|^alpha (a0 + ac cos 2theta + as sin 2theta) when
  // `generic` (the DS one, -k_x^2/|k|^2, otherwise)
  int generic, alpha;
  R a0, ac, as2;      // as2 = 2 as
  R dky;              // dk_y
  const R* kx;        // k_x of column q_x for the sin 2theta term (0 at the Nyquist column)
  // plans with the DS multiplier: m1(q_x, a) for a = |qbar_y| <= N_y,
  // computed in FP64 at plan creation (stored in the plan's precision), one
  // row of ldm entries per column with the even a first (a = 2 j at j) and the
  // odd a after them (a = 2 j' + 1 at N_y/2 + 1 + j')
  const R* m1;
  int ldm;
};

// The angular and radial factor of the generic multiplier at (k_x, qbar_y):
// |k|^alpha (a0 + (ac (k_x^2 - k_y^2) + 2 as k_x k_y)/|k|^2), 0 at k = 0.
// qs is the signed row index for the sin 2theta term, 0 at the Nyquist row:
// there the aliases +K and -K are averaged (as the real part of a
// full-spectrum evaluation does), which removes that odd term.
template <typename R>
__device__ __forceinline__ R mult_generic(const MultTabs<R>& mt, R wx2, R wy2, R kx, int qs, R s) {
  if (s == R(0)) return R(0);
  const R ang = mt.a0 + fdiv(mt.ac * (wx2 - wy2) + mt.as2 * kx * (R(qs) * mt.dky), s);
  R rad = R(1);
  if (mt.alpha == 1) rad = sqrt(s);
  else if (mt.alpha == -1) rad = R(1) / sqrt(s);
  return rad * ang;
}

// m1 = -(k_x^2/|k|^2) (1 - p(k)), m1(0) = 0, at column q_x and natural row
// frequency q (signed qbar = q or q - M_y).  With the Gaussian partition
// 1 - p = 1 - e^{-kx^2/s^2} e^{-ky^2/s^2} = gx + gy (1 - gx), a sum of
// non-negative terms (no cancellation near k = 0).
template <bool GEN, typename R>
__device__ __forceinline__ R mult_high(const MultTabs<R>& mt, R wx2, R kx, R gx, int q) {
  const int a = (q < mt.half_my) ? q : 2 * mt.half_my - q;
  const R wy2 = R(a * a) * mt.dky2;
  const R s = wx2 + wy2;
  if (s == R(0)) return R(0);
  R part;
  if (mt.sharp) {
    part = (s > mt.cut2) ? R(1) : R(0);
  } else if constexpr (sizeof(R) == 4) {
    // 1 - e^{-kx^2/s^2} e^{-ky^2/s^2} with e^{-ky^2/s^2} = 2^{-a^2 dk^2 / (s^2 ln 2)}
    // (hardware exp2): absolute error ~1e-7, at the level of FP32 rounding of m1
    const R ey = exp2f(R(a * a) * mt.neg_dky2_s2_log2e);
    part = R(1) - (R(1) - gx) * ey;
  } else {
    // 1 - exp(-ky^2/s^2): below working precision of 1 only for a < n_gy
    const R gy = (a < mt.n_gy) ? -expm1_r(-wy2 * mt.inv_sigma2) : R(1);
    part = gx + gy * (R(1) - gx);
  }
  if constexpr (GEN)
    return mult_generic(mt, wx2, wy2, kx, (q < mt.half_my) ? q : (q == mt.half_my ? 0 : q - 2 * mt.half_my), s) *
           part;
  else
    return -fdiv(wx2, s) * part;
}

// Workspace offsets (bytes) of one member's buffers, and member access.
struct WsOff {
  size_t A, B, Bband, Sband, c, partial, sched;
};
__device__ __forceinline__ Member member_at(const Members& m, int i) { return m.count == 1 ? m.one : m.dev[i]; }
template <typename T>
__device__ __forceinline__ T* ws_ptr(const Member& mb, size_t off) {
  return reinterpret_cast<T*>(mb.ws + off);
}

// Row tiling of the intermediate spectra (see the file comment).
template <typename R>
struct Tile {
  static constexpr int LT = (sizeof(R) == 4) ? DSNU_TILE_LT32 : 1;  // log2 rows per tile
  static constexpr int TR = 1 << LT;
  __device__ __forceinline__ static size_t at(int iy, int q, int ldq) {
    return ((size_t(iy >> LT) * ldq + q) << LT) | size_t(iy & (TR - 1));
  }
};

// Minimum resident CTAs per SM requested from the compiler: the FP64 kernels
// are limited to one CTA per SM by shared memory anyway, so they get the full
// register file.
template <typename R>
constexpr int min_blocks(int fp32_target) { return sizeof(R) == 4 ? fp32_target : 1; }

// Launch geometry shared by the kernels and their launchers.
template <typename R, int LOG2N>
struct Geo {
  static constexpr int N = 1 << LOG2N;
  static constexpr int M = 2 * N;
  static constexpr int G = N / 16;                   // threads per length-N FFT
  static constexpr int FB = fft_buf_elems(N);        // one FFT buffer
  static constexpr int RS = ((FB + 15) & ~15) + 4;   // row-buffer stride (== 4 mod 16)
  static constexpr int TR = Tile<R>::TR;
  // row passes: one group of G threads per row, RB_F / RB_I rows per CTA
  // (more rows for short rows), two transform buffers per row
  static constexpr int RMAX = (sizeof(R) == 4) ? 64 : 32;
  static constexpr int RB_F0 = (sizeof(R) == 4) ? DSNU_ROWF_RB32 : 1;
  static constexpr int RB_F = (RB_F0 * G >= 256) ? RB_F0 : ((256 / G < RMAX) ? 256 / G : RMAX);
  static constexpr int T_RF = RB_F * G;
  static constexpr int RB_I0 = (sizeof(R) == 4) ? DSNU_ROWI_RB32 : 1;
  static constexpr int RB_I = (RB_I0 * G >= 256) ? RB_I0 : ((256 / G < RMAX) ? 256 / G : RMAX);
  static constexpr int T_RI = RB_I * G;
  // column passes: CC columns per CTA
  static constexpr int CC = (G >= 256) ? 1 : 256 / G;
  static constexpr int T_C = CC * G;
  static constexpr int STW = fft_stage_tw_elems(LOG2N) > 0 ? fft_stage_tw_elems(LOG2N) : 1;
  static constexpr int STWP = (STW + 1) & ~1;  // keep the buffers 16-byte aligned
  // FP32 row passes keep e^{-2 pi i n/M} (n < N) in a shared table after the buffers
  static constexpr bool ROW_TAB = sizeof(R) == 4;
  // FP32 forward row pass: the next item's RB_F rows of rho (FP64) are
  // prefetched by a bulk copy into a landing buffer while the current item is
  // transformed; room for it comes from the compact stage table and a half
  // e^{-2 pi i n/M} table (n < N/2; the rest is -i times it).  Used when the
  // CTAs per SM that the registers allow still fit in shared memory.
  static constexpr int STWC = fft_stage_tw_elems_ct(LOG2N) > 0 ? fft_stage_tw_elems_ct(LOG2N) : 1;
  static constexpr int STWCP = (STWC + 1) & ~1;
  // (landing rows N + 8 doubles apart, so that the two rows read by one
  // half-warp fall in different banks)
  static constexpr int LS = N + DSNU_ROWF_LPAD;
  static constexpr size_t smem_row_fwd_pf =
      size_t(STWCP + 2 * RB_F * RS + N / 2 + RB_F * LS * 8 / int(sizeof(cpx<R>)) + 2) * sizeof(cpx<R>);
  static constexpr int MINB_F0 = (T_RF >= 512) ? 1 : DSNU_ROW_MINB;
  static constexpr bool ROW_PF =
      sizeof(R) == 4 && DSNU_ROWF_PF && MINB_F0 * (smem_row_fwd_pf + 1024) <= size_t(233472);
  static constexpr size_t smem_row_fwd =
      ROW_PF ? smem_row_fwd_pf : size_t(STWP + 2 * RB_F * RS + (ROW_TAB ? N : 0)) * sizeof(cpx<R>);
  // FP32 inverse row pass with two rows per CTA: the next row pair of A
  // ((N + 1) 16-byte segments of the row tiles) is prefetched by per-thread
  // asynchronous copies into a landing buffer [q][2], with the same compact
  // stage table and half twiddle table as the forward pass.
  static constexpr size_t smem_row_inv_pf = size_t(STWCP + 2 * RB_I * RS + N / 2 + 2 * (N + 1)) * sizeof(cpx<R>);
  static constexpr int MINB_I0 = (T_RI >= 512) ? 1 : DSNU_ROW_MINB;
  static constexpr bool ROWI_PF = sizeof(R) == 4 && DSNU_ROWI_PF && RB_I == 2 && TR == 4 &&
                                  MINB_I0 * (smem_row_inv_pf + 1024) <= size_t(233472);
  static constexpr size_t smem_row_inv =
      ROWI_PF ? smem_row_inv_pf : size_t(STWP + 2 * RB_I * RS + (ROW_TAB ? N : 0)) * sizeof(cpx<R>);
  // with the prefetch, the band values S(q), q <= Q, of the row pair can be
  // prefetched too, into 16 (Q + 1) more bytes after the landing buffer (the
  // launch then asks for them; the kernel's limit is set to the maximum)
  static constexpr size_t smem_row_inv_limit = ROWI_PF ? size_t(232448) : smem_row_inv;
  // two rows of 512 threads: their threads interleave lane by lane, so that
  // the two rows' elements of a 32-byte row tile are touched by adjacent lanes
  static constexpr bool ILV_F = (RB_F == 2);
  static constexpr bool ILV_I = (RB_I == 2);
  static constexpr int MINB_F = (T_RF >= 512) ? 1 : DSNU_ROW_MINB;
  static constexpr int MINB_I = (T_RI >= 512) ? 1 : DSNU_ROW_MINB;
  static constexpr size_t smem_col = size_t(STWP + 2 * CC * FB) * sizeof(cpx<R>);  // two chains
  // FP32 column pass of I1 with the DS multiplier: two shared tables on top,
  // e^{-2 pi i n/M} (n < N) and {(a dk_y)^2, e^{-(a dk_y)^2/sigma^2}} (a <= N)
  static constexpr bool COL_TAB = sizeof(R) == 4;
  // and two buffers of CC multiplier rows (N + 4 floats each), the current
  // item's and the next one's
  static constexpr int LDM = N + 4;
  static constexpr size_t smem_col_main = smem_col + (COL_TAB ? size_t(N) * 8 + size_t(2 * CC * LDM) * 4 : 0);
  static_assert(LOG2N >= 4 && LOG2N <= 12, "grid size 16..4096");
};

// Every FFT kernel is persistent: a grid of at most (SMs x resident CTAs)
// loops over its work items (row blocks or column blocks) and keeps the FFT
// stage twiddles in shared memory for the whole launch.  Each kernel's body is
// a device function of the CTA's index vb among vg CTAs that share the work,
// so that one launch can also serve several plans, each on its own range of
// CTAs (batch_ragged.cu).

// ---------------------------------------------------------------------------
// Forward row pass: per row, the even and odd output frequencies of the
// zero-padded length-M DFT of z = rho + i b are computed together (two
// interleaved length-N transforms of z and z w_M^n), then the two real-signal
// spectra are separated at every q in [0, N].
template <typename R, int LOG2N>
__device__ __forceinline__ void row_fwd_body(int vb, int vg, Members mem, WsOff off, int ldqA, int ldqB, int Q,
                                             int ny, AxisTabs<R> ax, const R* __restrict__ decon_y, int cj,
                                             int* status) {
  using GG = Geo<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, RB = GG::RB_F, T = GG::T_RF, RS = GG::RS;
  constexpr bool PF = GG::ROW_PF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* sm = stw + (PF ? GG::STWCP : GG::STWP);
  cpx<R>* wtab = sm + 2 * RB * RS;  // e^{-2 pi i n/M}: n < N/2 (PF) or n < N (FP32)
  double* land = reinterpret_cast<double*>(wtab + N / 2);  // PF: the item's RB rows of rho, LS apart
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(land + RB * GG::LS);
  if constexpr (PF) copy_to_smem(stw, ax.stwc, GG::STWC);
  else copy_to_smem(stw, ax.stw, GG::STW);
  if constexpr (GG::ROW_TAB)
    for (int i = threadIdx.x; i < (PF ? N / 2 : N); i += T) wtab[i] = twm(ax, i);
  if constexpr (PF)
    if (threadIdx.x == 0) mbar_init(bar, 1);
  __syncthreads();
  grid_dep_wait();
  // the column pass that follows hands out its columns from this counter
  if (vb == 0 && threadIdx.x == 0 && mem.count > 0) *ws_ptr<int>(member_at(mem, 0), off.sched) = 0;
  const int tid = threadIdx.x;
  const int rr = GG::ILV_F ? (tid & 1) : tid / G;
  const int t = GG::ILV_F ? (tid >> 1) : tid - rr * G;
  const R isg = cj ? R(-1) : R(1);
  cpx<R>* buf_e = sm + (2 * rr) * RS;
  cpx<R>* buf_o = buf_e + RS;
  const int items = (ny + RB - 1) / RB;
  const int total = items * mem.count;
  // thread 0: the rows of item it2 into the landing buffer, one copy per row
  auto prefetch = [&](int it2) {
    const int mi2 = it2 / items;
    const int r0 = (it2 - mi2 * items) * RB;
    const int nr = min(RB, ny - r0);
    const double* src = member_at(mem, mi2).rho + size_t(r0) * N;
    mbar_expect_tx(bar, unsigned(nr) * unsigned(N * sizeof(double)));
    // rho is read once: its lines go first when L2 needs room (keeps more of A and B resident)
    const unsigned long long pol = l2_evict_first();
    for (int r = 0; r < nr; ++r)
      bulk_load(land + r * GG::LS, src + size_t(r) * N, unsigned(N * sizeof(double)), bar, pol);
  };
  if constexpr (PF)
    if (tid == 0 && vb < total) prefetch(vb);
  unsigned phase = 0;
#pragma unroll 1
  for (int it = vb; it < total; it += vg) {
    if (it + vg >= total) grid_dep_trigger();  // last item of this CTA
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    const double* __restrict__ rho = mb.rho;
    cpx<R>* __restrict__ A = ws_ptr<cpx<R>>(mb, off.A);
    cpx<R>* __restrict__ B = ws_ptr<cpx<R>>(mb, off.B);
    const int row0 = item * RB;
    const int row = row0 + rr;
    const bool valid = row < ny;
    const R dy = valid ? decon_y[row] : R(0);
    bool landed = true;
    if constexpr (PF) {
      // bounded wait (1 s); on expiry the CTA stops after the reads below
      // (cta_timed_out) without writing anything
      landed = mbar_wait(bar, phase, 1000000000ull);
      phase ^= 1u;
    }
    // FP32 with the landing buffer: rho rounded to FP32, half of the 16 values
    // by the conversion instruction and half by integer instructions
    // (f32_of_f64_int, the same result bit for bit): the instruction runs on
    // GB300's narrow FP64 pipe, the integer form on the integer pipe, and the
    // two halves overlap (all by the instruction cost this pass 19 us, all by
    // integers about as much; half and half 15 us).  One vote of the warp
    // sends the rare values outside the integer form's range to the
    // instruction, out of line.
    R xs[PF ? 16 : 1];
    if constexpr (PF) {
      unsigned oddm = 0u;
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        if (m & 1) {
          bool odd;
          xs[m] = f32_of_f64_int(land[rr * GG::LS + t + G * m], odd);
          oddm |= (odd && valid) ? (1u << m) : 0u;
        } else {
          xs[m] = __double2float_rn(land[rr * GG::LS + t + G * m]);
        }
      }
      if (__any_sync(0xffffffffu, oddm != 0u)) {
        for (int m = 1; m < 16; m += 2)
          if ((oddm >> m) & 1u) xs[m] = f32_of_f64_hw(land[rr * GG::LS + t + G * m]);
      }
    }
    cpx<R> e[16], o[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = t + G * m;
      R x;
      if constexpr (PF) x = valid ? xs[m] : R(0);
      else x = valid ? from_f64<R>(rho[size_t(row) * N + n]) : R(0);
      const cpx<R> z = mk<R>(x, isg * (x * ax.decon[n] * dy));
      cpx<R> w;
      if constexpr (PF) {
        w = wtab[t + G * (m & 7)];           // n - N/2 for m >= 8, and
        if (m >= 8) w = mk<R>(w.y, -w.x);   // e^{-2 pi i (n' + N/2)/M} = -i e^{-2 pi i n'/M}
      } else if constexpr (GG::ROW_TAB) {
        w = wtab[n];
      } else {
        w = twm(ax, n);
      }
      w.y *= isg;
      e[m] = z;
      o[m] = cmul(z, w);
    }
    if constexpr (PF) {
      // every thread has read the landing buffer (a barrier); stop if a wait expired
      if (cta_timed_out(landed, bar, phase ^ 1u, status)) return;
      if (tid == 0 && it + vg < total) prefetch(it + vg);
    }
    block_fft2_regs<R, LOG2N, PF>(e, o, buf_e, buf_o, t, stw, cj != 0);
    __syncthreads();  // last-stage loads (and the previous unpack) finished
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      buf_e[pad16(t + G * m)] = e[m];
      buf_o[pad16(t + G * m)] = o[m];
    }
    __syncthreads();
    // separate the spectra at every q in [0, N] (rows fastest):
    // Z(q) = E[q/2] (q even) or O[(q-1)/2] (q odd); Z(M - q) has the same parity.
    // Element idx = tid + T i of the RB (N + 1) is row r2 = tid % RB (T is a
    // multiple of RB) at q = tid / RB + G i: 16 steps for every thread, a 17th
    // (q = N) for tid < RB; the row, and for G even the parity, stay fixed
    {
      const int r2 = tid & (RB - 1), q0 = tid / RB, row2 = row0 + r2;
      const cpx<R>* be = sm + (2 * r2) * RS;
      const cpx<R>* bo = be + RS;
      cpx<R>* Ar = A + Tile<R>::at(row2, 0, ldqA);
      cpx<R>* Br = B + Tile<R>::at(row2, 0, ldqB);
      if (row2 < ny) {
#pragma unroll 4
        for (int i = 0; i < 17; ++i) {
          const int q = q0 + G * i;
          if (i == 16 && q > N) break;
          const int k = q >> 1;
          cpx<R> zq, zm;
          if (q & 1) {
            zq = bo[pad16(k)];
            zm = bo[pad16(N - 1 - k)];
          } else {
            zq = be[pad16(k)];
            zm = be[pad16(k == 0 ? 0 : N - k)];
          }
          Ar[q * Tile<R>::TR] = mk<R>(R(0.5) * (zq.x + zm.x), R(0.5) * (zq.y - zm.y));
          if (q <= Q) {
            const cpx<R> d = mk<R>(zq.x - zm.x, zq.y + zm.y);  // Z(q) - conj Z(M - q)
            // divided by 2 i (by 2 (-i) in the conjugated pipeline)
            Br[q * Tile<R>::TR] = cj ? mk<R>(R(-0.5) * d.y, R(0.5) * d.x) : mk<R>(R(0.5) * d.y, R(-0.5) * d.x);
          }
        }
      }
    }
  }
}

template <typename R, int LOG2N>
__global__ void __launch_bounds__(Geo<R, LOG2N>::T_RF, min_blocks<R>(Geo<R, LOG2N>::MINB_F))
k_row_fwd(Members mem, WsOff off, int ldqA, int ldqB, int Q, int ny, AxisTabs<R> ax,
          const R* __restrict__ decon_y, int cj, int* status) {
  row_fwd_body<R, LOG2N>(blockIdx.x, gridDim.x, mem, off, ldqA, ldqB, Q, ny, ax, decon_y, cj, status);
}

// ---------------------------------------------------------------------------
// Column pass of I1: per column, both chains (even/odd output rows of the
// padded column DFT) go forward together, are multiplied by m1 and come back
// together; their sum is the column of I1's inverse.  All loads of a column
// precede the first barrier, so the in-place update is safe.
template <typename R, int LOG2N, bool GEN>
__device__ __forceinline__ void col_main_body(int vb, int vg, Members mem, WsOff off, int ldqA, int ncols,
                                              AxisTabs<R> ay, MultTabs<R> mt, int cj, int* ctr) {
  using GG = Geo<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, CC = GG::CC, FB = GG::FB;
  // FP32 with the DS multiplier: the e^{-2 pi i n/M} factors of the odd chain
  // come from a shared table filled once per CTA with the arithmetic of twm(),
  // and m1 of the item's columns from the plan's FP64-computed table, copied
  // row by row into shared memory (cp.async) one item ahead
  constexpr bool TAB = GG::COL_TAB && !GEN;
  constexpr int LDM = GG::LDM;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* sm = stw + GG::STWP;
  copy_to_smem(stw, ay.stw, GG::STW);
  const int tid = threadIdx.x;
  const int cl = tid / G, t = tid - cl * G;
  const R isg = cj ? R(-1) : R(1);
  cpx<R>* buf_e = sm + (2 * cl) * FB;
  cpx<R>* buf_o = buf_e + FB;
  cpx<R>* wtab = sm + 2 * CC * FB;                       // N entries (TAB only)
  // TAB: buffer b holds the m1 rows of an item's CC columns; a warp reads a's
  // of one parity (a = |qbar| of the rows 2 (t + G m) + h), so consecutive
  // entries of the parity-split rows
  float* mrow = reinterpret_cast<float*>(wtab + N);
  constexpr int MH = N / 2 + 1;  // even entries
  const int items = (ncols + CC - 1) / CC;
  const int total = items * mem.count;
  // every thread: its share of the m1 rows of item it2 into buffer b
  auto fetch_mult = [&](int it2, int b) {
    const int item2 = it2 % items;
    for (int i = tid; i < CC * (LDM / 4); i += GG::T_C) {
      const int c = i / (LDM / 4), k = i - c * (LDM / 4);
      const int col2 = item2 * CC + c;
      if (col2 < ncols) cp_async16(mrow + (b * CC + c) * LDM + 4 * k, mt.m1 + size_t(col2) * mt.ldm + 4 * k);
    }
    cp_async_commit();
  };
  if constexpr (TAB) {
    for (int i = tid; i < N; i += GG::T_C) wtab[i] = twm(ay, i);
    if (vb < total) fetch_mult(vb, 0);  // (a plan table: no wait needed)
    __syncthreads();
  }
  grid_dep_wait();
  // the next item's column values are loaded into registers before the
  // current item's inverse transform (PF), hiding their latency
  constexpr bool PF = TAB && DSNU_COL_REGPF;
  cpx<R> xn[PF ? 16 : 1];
  auto load_col = [&](int it2, cpx<R>(&x)[PF ? 16 : 1]) {
    const int mi2 = it2 / items;
    const int col2 = (it2 - mi2 * items) * CC + cl;
    const cpx<R>* A2 = ws_ptr<cpx<R>>(member_at(mem, mi2), off.A);
#pragma unroll
    for (int m = 0; m < (PF ? 16 : 1); ++m)
      x[m] = (col2 < ncols) ? A2[Tile<R>::at(t + G * m, col2, ldqA)] : mk<R>(R(0), R(0));
  };
  // Items: CTA vb starts with items vb and vb + vg; with a work counter
  // (`ctr`, zeroed by the row pass before) each CTA then takes the next free
  // item, item 2 vg + c for the counter's value c, else items vb + 2 vg,
  // vb + 3 vg, ...  Taken from a counter, a CTA that runs slower than the
  // others (persistent CTAs that a programmatic launch placed as the previous
  // kernel's CTAs drained ran up to 15 % slower, leaving the last ones 40 us
  // behind) takes fewer columns; the first two items need no atomic, so the
  // first answer is ready within the first item.  s_next[(kk + 1) & 1]
  // carries the item after `nxt` from thread 0 to the others across the
  // inverse transform's barriers.
  __shared__ int s_next[2];
  int nxt = vb + vg;  // the item after `it`
  if constexpr (PF)
    if (vb < total) load_col(vb, xn);
  int kk = 0;  // items done by this CTA (the multiplier buffer is kk & 1)
#pragma unroll 1
  for (int it = vb; it < total; ++kk) {
    if (nxt >= total) grid_dep_trigger();  // last item of this CTA
    // (thread 0 stores the counter's answer only after the forward transform,
    // so that its warp does not wait for the atomic at the start of the item)
    int grabbed = total;
    if (ctr && tid == 0 && nxt < total) grabbed = 2 * vg + atomicAdd(ctr, 1);
    const int mi = it / items, item = it - mi * items;
    cpx<R>* __restrict__ A = ws_ptr<cpx<R>>(member_at(mem, mi), off.A);
    const int col = item * CC + cl;
    const bool valid = col < ncols;
    const R wx2 = (!TAB && valid) ? mt.wx2[col] : R(0);
    const R gx = (!TAB && valid) ? mt.gx[col] : R(0);
    const R kxc = (GEN && valid) ? mt.kx[col] : R(0);
    // this thread's copies of the item's m1 rows have landed; the barriers of
    // the forward transform below make every thread's copies visible
    if constexpr (TAB) cp_async_wait_all();
    const float* mr = mrow + ((kk & 1) * CC + cl) * LDM;
    cpx<R> e[16], o[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = t + G * m;
      cpx<R> x;
      if constexpr (PF) x = xn[m];
      else x = valid ? A[Tile<R>::at(n, col, ldqA)] : mk<R>(R(0), R(0));
      cpx<R> w;
      if constexpr (TAB) w = wtab[n];
      else w = twm(ay, n);
      w.y *= isg;
      e[m] = x;
      o[m] = cmul(x, w);
    }
    block_fft2_regs<R, LOG2N>(e, o, buf_e, buf_o, t, stw, cj != 0);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = 2 * (t + G * m);
      if constexpr (TAB) {
        // m1 at rows q and q + 1 (a = |qbar|, of the parity of q + h)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int qq = q + h;
          const int a = (qq < N) ? qq : 2 * N - qq;
          const R mv = valid ? mr[(h ? MH : 0) + (a >> 1)] : R(0);
          if (h == 0) e[m] = e[m] * mv;
          else o[m] = o[m] * mv;
        }
      } else if constexpr (!GEN) {
        // FP64: m1 read from the plan's table in global memory (the pass is
        // bound by FP64 arithmetic, which the table saves; the loads overlap it)
        const R* mg = mt.m1 + size_t(valid ? col : 0) * mt.ldm;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int qq = q + h;
          const int a = (qq < N) ? qq : 2 * N - qq;
          const R mv = valid ? mg[(h ? MH : 0) + (a >> 1)] : R(0);
          if (h == 0) e[m] = e[m] * mv;
          else o[m] = o[m] * mv;
        }
      } else {
        e[m] = e[m] * (valid ? mult_high<GEN>(mt, wx2, kxc, gx, q) : R(0));
        o[m] = o[m] * (valid ? mult_high<GEN>(mt, wx2, kxc, gx, q + 1) : R(0));
      }
    }
    if (ctr && tid == 0) s_next[(kk + 1) & 1] = grabbed;
    if constexpr (PF)
      if (nxt < total) load_col(nxt, xn);
    // the next item's m1 rows into the other buffer (last read by the item
    // before this one, whose reads the barriers since then have completed)
    if constexpr (TAB)
      if (nxt < total) fetch_mult(nxt, (kk + 1) & 1);
    block_fft2_regs<R, LOG2N>(e, o, buf_e, buf_o, t, stw, cj == 0);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int n = t + G * m;
        cpx<R> w;
        if constexpr (TAB) w = wtab[n];
        else w = twm(ay, n);
        A[Tile<R>::at(n, col, ldqA)] = cj ? e[m] + cmul(o[m], w) : e[m] + cmulc(o[m], w);
      }
    }
    it = nxt;
    nxt = ctr ? s_next[(kk + 1) & 1] : nxt + vg;
  }
}

template <typename R, int LOG2N, bool GEN>
__global__ void __launch_bounds__(Geo<R, LOG2N>::T_C, min_blocks<R>(DSNU_COLMAIN_MINB))
k_col_main(Members mem, WsOff off, int ldqA, int ncols, AxisTabs<R> ay, MultTabs<R> mt, int cj) {
  col_main_body<R, LOG2N, GEN>(blockIdx.x, gridDim.x, mem, off, ldqA, ncols, ay, mt, cj,
                               ws_ptr<int>(member_at(mem, 0), off.sched));
}


// ---------------------------------------------------------------------------
// Band columns of the type-2 spectrum: per column of B, both output parities
// of the padded column DFT in one paired transform; rows |qbar| <= Q kept.
template <typename R, int LOG2N>
__device__ __forceinline__ void band_fwd_body(int vb, int vg, Members mem, WsOff off, int ldqB, int ncols, int ldq,
                                              int Q, AxisTabs<R> ay, int cj) {
  using GG = Geo<R, LOG2N>;
  constexpr int N = GG::N, M = GG::M, G = GG::G, CC = GG::CC, FB = GG::FB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* sm = stw + GG::STWP;
  copy_to_smem(stw, ay.stw, GG::STW);
  const int tid = threadIdx.x;
  const int cl = tid / G, t = tid - cl * G;
  const R isg = cj ? R(-1) : R(1);
  cpx<R>* buf_e = sm + (2 * cl) * FB;
  cpx<R>* buf_o = buf_e + FB;
  const int items = (ncols + CC - 1) / CC;
  grid_dep_wait();
#pragma unroll 1
  for (int it = vb; it < items * mem.count; it += vg) {
    if (it + vg >= items * mem.count) grid_dep_trigger();  // last item of this CTA
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    const cpx<R>* __restrict__ B = ws_ptr<cpx<R>>(mb, off.B);
    cpx<R>* __restrict__ Bband = ws_ptr<cpx<R>>(mb, off.Bband);
    const int col = item * CC + cl;
    const bool valid = col < ncols;
    cpx<R> e[16], o[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = t + G * m;
      const cpx<R> x = valid ? B[Tile<R>::at(n, col, ldqB)] : mk<R>(R(0), R(0));
      cpx<R> w = twm(ay, n);
      w.y *= isg;
      e[m] = x;
      o[m] = cmul(x, w);
    }
    block_fft2_regs<R, LOG2N>(e, o, buf_e, buf_o, t, stw, cj != 0);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int q = 2 * (t + G * m);
        const int se = q < N ? q : q - M;
        const int so = q + 1 < N ? q + 1 : q + 1 - M;
        if (se >= -Q && se <= Q) Bband[size_t(col) * ldq + se + Q] = e[m];
        if (so >= -Q && so <= Q) Bband[size_t(col) * ldq + so + Q] = o[m];
      }
    }
  }
}

template <typename R, int LOG2N>
__global__ void __launch_bounds__(Geo<R, LOG2N>::T_C, min_blocks<R>(DSNU_COL_MINB))
k_band_fwd(Members mem, WsOff off, int ldqB, int ncols, int ldq, int Q, AxisTabs<R> ay, int cj) {
  band_fwd_body<R, LOG2N>(blockIdx.x, gridDim.x, mem, off, ldqB, ncols, ldq, Q, ay, cj);
}

// ---------------------------------------------------------------------------
// Type-2 interpolation (eq. 2.2) and the polar weighting c_j = D_j rho_hat_j
// (eq. I2PolarDisc, FP64 multiply), by tiles of stencil origins: the plan
// groups the nodes by the kItile x kItile tile of the (q_x, q_y) plane that
// holds their stencil origin, in work items of at most kItileNodes nodes of
// one tile; one CTA per item copies the (kItile + w - 1)^2 band values its
// stencils reach into shared memory (whole band columns' runs, read
// coalesced once; the Hermitian fold for q_x < 0 and the centring phase
// applied on the way; zero outside the band) and then runs every node's
// stencil sum from there, four threads per node.  The band values are read
// once per item instead of once per stencil that covers them, in runs rather
// than in scattered 8-byte loads (one warp per node gathering them from the
// band array took 79 us on 12 SMs, against 19 us on 6 for this form), and a CTA
// starts all its nodes at once, which is what makes the stage fast on the few
// SMs it gets next to the column pass.
constexpr int kItile = 32;       // tile edge (stencil origins)
constexpr int kItileNodes = 64;  // nodes per work item at most (four threads each: 256)
template <typename R>
__device__ __forceinline__ void interp_tile_body(int tile, int mi, Members mem, WsOff off, int ldq, int Q,
                                                 const int2* __restrict__ q0, const R* __restrict__ wts,
                                                 const double* __restrict__ D, const int* __restrict__ tile_ptr,
                                                 const int2* __restrict__ tile_org,
                                                 const int* __restrict__ tile_nodes, int w, int cj) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* reg = reinterpret_cast<cpx<R>*>(smem_raw);  // [dx][dy], S x S
  const int S = kItile + w - 1;
  const int2 org = tile_org[tile];
  const int n0 = tile_ptr[tile], n1 = tile_ptr[tile + 1];
  // four threads per node (an item holds at most 64), thread h of a node
  // taking the stencil rows b = h, h + 4, ...; the node's plan data are
  // fetched before the wait for the band values
  const int s = threadIdx.x >> 2, h = threadIdx.x & 3;
  const bool have = n0 + s < n1;
  const int j = have ? tile_nodes[n0 + s] : 0;
  const int2 b0 = have ? q0[j] : make_int2(0, 0);
  const double d = have ? D[j] : 0.0;
  grid_dep_wait();
  const Member mb = member_at(mem, mi);
  const cpx<R>* __restrict__ Bband = ws_ptr<cpx<R>>(mb, off.Bband);
  cpx<R>* __restrict__ c = ws_ptr<cpx<R>>(mb, off.c);
  for (int i = threadIdx.x; i < S * S; i += blockDim.x) {
    const int dx = i / S, dy = i - dx * S;
    const int qx = org.x + dx, qy = org.y + dy;
    cpx<R> v = mk<R>(R(0), R(0));
    if (qx <= Q && qx >= -Q && qy <= Q && qy >= -Q) {
      if (qx >= 0) {
        v = Bband[size_t(qx) * ldq + qy + Q];
      } else {
        v = conj(Bband[size_t(-qx) * ldq + (Q - qy)]);
      }
      const int e = qx + qy;
      v = mul_ipow(v, cj ? -e : e);  // centring phase i^{q_x + q_y}
    }
    reg[i] = v;
  }
  __syncthreads();
  R ax = R(0), ay = R(0);
  if (have) {
    const R* wx = wts + size_t(j) * 2 * w;
    const R* wy = wx + w;
    const cpx<R>* rb = reg + (b0.x - org.x) * S + (b0.y - org.y);
    for (int b = h; b < w; b += 4) {
      const R fy = wy[b];
      for (int a = 0; a < w; ++a) {
        const cpx<R> v = rb[a * S + b];
        const R f = wx[a] * fy;
        ax += f * v.x;
        ay += f * v.y;
      }
    }
  }
  ax += __shfl_xor_sync(0xffffffffu, ax, 1);
  ay += __shfl_xor_sync(0xffffffffu, ay, 1);
  ax += __shfl_xor_sync(0xffffffffu, ax, 2);
  ay += __shfl_xor_sync(0xffffffffu, ay, 2);
  // the four partial sums of a node (lanes 4 s' .. 4 s' + 3 of the warp)
  if (have && h == 0) c[j] = mk<R>(R(d * double(ax)), R(d * double(ay)));
}

template <typename R>
__global__ void __launch_bounds__(256)
k_interp_tile(Members mem, WsOff off, int ldq, int Q, const int2* __restrict__ q0, const R* __restrict__ wts,
              const double* __restrict__ D, const int* __restrict__ tile_ptr, const int2* __restrict__ tile_org,
              const int* __restrict__ tile_nodes, int w, int cj) {
  interp_tile_body<R>(blockIdx.x, blockIdx.y, mem, off, ldq, Q, q0, wts, D, tile_ptr, tile_org, tile_nodes, w, cj);
}
inline size_t interp_tile_smem(int w, size_t csz) { return size_t(kItile + w - 1) * size_t(kItile + w - 1) * csz; }

// ---------------------------------------------------------------------------
// Type-1 spreading as a gather over TILE x TILE tiles of band cells.  At plan
// time the (node, stencil origin, ES weights) entries of every node whose
// stencil meets a tile are laid out contiguously per tile and cut into work
// items of at most CHUNK entries.  k_spread: one CTA per work item; each cell
// is served by SPLIT threads that take every SPLIT-th entry; the CTA writes
// the item's partial sums.  k_spread_reduce: per tile, adds its items' partial
// sums in item order (deterministic, no atomics) and applies the centring
// phase.  The (TILE, SPLIT, CHUNK) configuration is chosen per plan by timing
// the candidates below (see autotune_spread in plan.cu).
struct SpreadCfg {
  int tile, split, chunk;
};
constexpr int kNumSpreadCfgs = 4;
constexpr SpreadCfg kSpreadCfgs[kNumSpreadCfgs] = {{8, 4, 128}, {8, 2, 128}, {16, 1, 128}, {16, 2, 64}};

// (item: the work item, mi: the member)
template <typename R, int TILE, int SPLIT, int CHUNK>
__device__ __forceinline__ void spread_body(int item, int mi, Members mem, WsOff off,
                                            const int2* __restrict__ item_range, const int* __restrict__ ent_node,
                                            const int2* __restrict__ ent_q0, const R* __restrict__ ent_w,
                                            const int* __restrict__ item_tile, int w, int tiles_x, int Q) {
  constexpr int CELLS = TILE * TILE, THREADS = CELLS * SPLIT;
  __shared__ int2 s_q0[CHUNK];
  __shared__ cpx<R> s_c[CHUNK];
  __shared__ R s_w[CHUNK * 32];
  __shared__ R s_red[2][SPLIT][CELLS];
  grid_dep_wait();
  const Member mb = member_at(mem, mi);
  const cpx<R>* __restrict__ c = ws_ptr<cpx<R>>(mb, off.c);
  cpx<R>* __restrict__ partial = ws_ptr<cpx<R>>(mb, off.partial);
  const int tile = item_tile[item];
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int cell = threadIdx.x & (CELLS - 1), part = threadIdx.x / CELLS;
  const int qx = tx * TILE + (cell & (TILE - 1));
  const int qy = ty * TILE + (cell / TILE) - Q;
  const int2 rg = item_range[item];
  const int s0 = rg.x, cnt = rg.y - rg.x;  // cnt <= CHUNK
  const int w2 = 2 * w;
  for (int i = threadIdx.x; i < cnt; i += THREADS) {
    s_q0[i] = ent_q0[s0 + i];
    s_c[i] = c[ent_node[s0 + i]];
  }
  const R* src = ent_w + size_t(s0) * w2;
  for (int i = threadIdx.x; i < cnt * w2; i += THREADS) {
    const int e = i / w2;
    s_w[e * 32 + (i - e * w2)] = src[i];
  }
  __syncthreads();
  R ax = R(0), ay = R(0);
  for (int k = part; k < cnt; k += SPLIT) {
    const int a = qx - s_q0[k].x, b = qy - s_q0[k].y;
    if ((unsigned)a < (unsigned)w && (unsigned)b < (unsigned)w) {
      const R f = s_w[k * 32 + a] * s_w[k * 32 + w + b];
      ax += f * s_c[k].x;
      ay += f * s_c[k].y;
    }
  }
  if constexpr (SPLIT > 1) {
    s_red[0][part][cell] = ax;
    s_red[1][part][cell] = ay;
    __syncthreads();
    if (part != 0) return;
#pragma unroll
    for (int p = 1; p < SPLIT; ++p) {
      ax += s_red[0][p][cell];
      ay += s_red[1][p][cell];
    }
  }
  partial[size_t(item) * CELLS + cell] = mk<R>(ax, ay);
}

template <typename R, int TILE, int SPLIT, int CHUNK>
__global__ void __launch_bounds__(TILE * TILE * SPLIT)
k_spread(Members mem, WsOff off, const int2* __restrict__ item_range,
         const int* __restrict__ ent_node, const int2* __restrict__ ent_q0,
         const R* __restrict__ ent_w, const int* __restrict__ item_tile, int w, int tiles_x, int Q) {
  spread_body<R, TILE, SPLIT, CHUNK>(blockIdx.x, blockIdx.y, mem, off, item_range, ent_node, ent_q0, ent_w,
                                     item_tile, w, tiles_x, Q);
}

// (tile: the spreading tile, mi: the member)
template <typename R, int TILE>
__device__ __forceinline__ void spread_reduce_body(int tile, int mi, Members mem, WsOff off,
                                                   const int* __restrict__ tile_items, int tiles_x, int n_tiles,
                                                   int Q, int ldq, int cj) {
  constexpr int CELLS = TILE * TILE;
  grid_dep_wait();
  const Member mb = member_at(mem, mi);
  const cpx<R>* __restrict__ partial = ws_ptr<cpx<R>>(mb, off.partial);
  cpx<R>* __restrict__ Sband = ws_ptr<cpx<R>>(mb, off.Sband);
  if (tile >= n_tiles) return;
  const int cell = threadIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int qx = tx * TILE + (cell & (TILE - 1));
  const int qy = ty * TILE + (cell / TILE) - Q;
  R ax = R(0), ay = R(0);
  for (int it = tile_items[tile]; it < tile_items[tile + 1]; ++it) {
    const cpx<R> v = partial[size_t(it) * CELLS + cell];
    ax += v.x;
    ay += v.y;
  }
  if (qx <= Q && qy <= Q) {
    const int e = qx + qy;
    Sband[size_t(qx) * ldq + qy + Q] = mul_ipow(mk<R>(ax, ay), cj ? e : -e);  // (-i)^{q_x+q_y}
  }
}

template <typename R, int TILE>
__global__ void __launch_bounds__(TILE * TILE)
k_spread_reduce(Members mem, WsOff off, const int* __restrict__ tile_items, int tiles_x,
                int n_tiles, int Q, int ldq, int cj) {
  spread_reduce_body<R, TILE>(blockIdx.x, blockIdx.y, mem, off, tile_items, tiles_x, n_tiles, Q, ldq, cj);
}

// Launch the spreading pair with configuration `cfg`: part 0 = k_spread,
// part 1 = k_spread_reduce, part 2 = both.
// Launch with programmatic stream serialization when `pdl` (see grid_dep_wait).
template <typename... KArgs, typename... Args>
inline void launch_k(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                     Args... args) {
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cfg.attrs = attr;
  cfg.numAttrs = pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
}

template <typename R>
void launch_spread(int cfg, const Members& mem, const WsOff& off, const PlanTables& t, const PlanGeom& g,
                   int ldq, int cj, cudaStream_t st, int part, bool pdl) {
  const R* ew = static_cast<const R*>(t.ent_w);
#define DSNU_SPREAD(TL, SP, CH)                                                                     \
  if (part != 1 && g.n_items > 0)                                                                 \
    launch_k(pdl, k_spread<R, TL, SP, CH>, dim3(g.n_items, mem.count), dim3(TL * TL * SP), 0, st,  \
             mem, off, t.item_range, t.ent_node, t.ent_q0, ew, t.item_tile, g.w, g.tiles_x, g.Q);    \
  if (part != 0)                                                                                    \
    launch_k(pdl, k_spread_reduce<R, TL>, dim3(g.n_tiles, mem.count), dim3(TL * TL), 0, st, mem, off, \
             t.tile_items, g.tiles_x, g.n_tiles, g.Q, ldq, cj)
  switch (cfg) {
    case 1: DSNU_SPREAD(8, 2, 128); break;
    case 2: DSNU_SPREAD(16, 1, 128); break;
    case 3: DSNU_SPREAD(16, 2, 64); break;
    default: DSNU_SPREAD(8, 4, 128); break;
  }
#undef DSNU_SPREAD
}

// ---------------------------------------------------------------------------
// Inverse band columns: the even and odd rows of each band column of S go
// through one paired inverse transform; T = even + e^{+2 pi i n/M} odd, n < N.
template <typename R, int LOG2N>
__device__ __forceinline__ void band_inv_body(int vb, int vg, Members mem, WsOff off, int ldq, int Q, int ncols,
                                              int ldqB, AxisTabs<R> ay, int cj) {
  using GG = Geo<R, LOG2N>;
  constexpr int N = GG::N, M = GG::M, G = GG::G, CC = GG::CC, FB = GG::FB;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* sm = stw + GG::STWP;
  copy_to_smem(stw, ay.stw, GG::STW);
  const int tid = threadIdx.x;
  const int cl = tid / G, t = tid - cl * G;
  cpx<R>* buf_e = sm + (2 * cl) * FB;
  cpx<R>* buf_o = buf_e + FB;
  const int items = (ncols + CC - 1) / CC;
  grid_dep_wait();
#pragma unroll 1
  for (int it = vb; it < items * mem.count; it += vg) {
    if (it + vg >= items * mem.count) grid_dep_trigger();  // last item of this CTA
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    const cpx<R>* __restrict__ Sband = ws_ptr<cpx<R>>(mb, off.Sband);
    cpx<R>* __restrict__ St = ws_ptr<cpx<R>>(mb, off.B);
    const int col = item * CC + cl;
    const bool valid = col < ncols;
    cpx<R> e[16], o[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = 2 * (t + G * m);
      const int se = q < N ? q : q - M;
      const int so = q + 1 < N ? q + 1 : q + 1 - M;
      const cpx<R> z = mk<R>(R(0), R(0));
      e[m] = (valid && se >= -Q && se <= Q) ? Sband[size_t(col) * ldq + se + Q] : z;
      o[m] = (valid && so >= -Q && so <= Q) ? Sband[size_t(col) * ldq + so + Q] : z;
    }
    block_fft2_regs<R, LOG2N>(e, o, buf_e, buf_o, t, stw, cj == 0);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int n = t + G * m;
        const cpx<R> w = twm(ay, n);
        St[Tile<R>::at(n, col, ldqB)] = cj ? e[m] + cmul(o[m], w) : e[m] + cmulc(o[m], w);
      }
    }
  }
}

template <typename R, int LOG2N>
__global__ void __launch_bounds__(Geo<R, LOG2N>::T_C, min_blocks<R>(DSNU_COL_MINB))
k_band_inv(Members mem, WsOff off, int ldq, int Q, int ncols, int ldqB, AxisTabs<R> ay, int cj) {
  band_inv_body<R, LOG2N>(blockIdx.x, gridDim.x, mem, off, ldq, Q, ncols, ldqB, ay, cj);
}

// ---------------------------------------------------------------------------
// Inverse length-M DFT keeping n < N, split by output parity:
//   T(2j)   = IDFT_N[W(q) + W(q + N)](j)
//   T(2j+1) = IDFT_N[(W(q) - W(q + N)) e^{+2 pi i q/M}](j),   q < N,
// with W(q) = Y(q) + i S(q) for q <= N and W(M - q) = conj Y(q) + i conj S(q).
// Both transforms run together; j < N/2 gives the grid points n < N.
// Phi must be 16-byte aligned (checked on the host).  With acc64 (FP32 plans)
// Phi = I1 + I2 is added in FP64: I1 = Re T / (Mx My) and I2 = Im T dx dy /
// (Mx My) are each formed in FP32 (1/(Mx My) is a power of two, so the
// scaling is exact), and their FP64 sum is formed by add_f32_f64 (bitwise
// the FP64 addition of the two widened terms).
template <typename R, int LOG2N>
__device__ __forceinline__ void row_inv_body(int vb, int vg, Members mem, WsOff off, int ldqA, int ldqB, int Q,
                                             int ny, AxisTabs<R> ax, const R* __restrict__ decon_y, R scale, int cj,
                                             int bpf, int acc64) {
  using GG = Geo<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, RB = GG::RB_I, RS = GG::RS, T = GG::T_RI;
  constexpr bool PF = GG::ROWI_PF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* sm = stw + (PF ? GG::STWCP : GG::STWP);
  cpx<R>* wtab = sm + 2 * RB * RS;  // e^{-2 pi i q/M}: q < N/2 (PF) or q < N (FP32)
  cpx<R>* land = wtab + N / 2;      // PF: Y(q) of the item's two rows at [2 q + row], q <= N
  cpx<R>* land_s = land + 2 * (N + 1);  // PF and bpf: S(q) likewise, q <= Q
  if constexpr (PF) copy_to_smem(stw, ax.stwc, GG::STWC);
  else copy_to_smem(stw, ax.stw, GG::STW);
  if constexpr (GG::ROW_TAB)
    for (int i = threadIdx.x; i < (PF ? N / 2 : N); i += T) wtab[i] = twm(ax, i);
  const int tid = threadIdx.x;
  const int rr = GG::ILV_I ? (tid & 1) : tid / G;
  const int t = GG::ILV_I ? (tid >> 1) : tid - rr * G;
  // FP32: the deconvolution factors of the outputs n = 2 (t + G m) + {0, 1}
  // this thread writes, the same for every row: kept in registers for the
  // whole launch (loaded per item, at the end of each transform, they came
  // from L2 and stalled the stores)
  constexpr int ND = sizeof(R) == 4 ? 8 : 1;
  float2 dec[ND];
  if constexpr (sizeof(R) == 4) {
#pragma unroll
    for (int m = 0; m < 8; ++m) dec[m] = *reinterpret_cast<const float2*>(ax.decon + 2 * (t + G * m));
  }
  __syncthreads();
  grid_dep_wait();
  const int si = cj ? -1 : 1;
  cpx<R>* buf_u = sm + (2 * rr) * RS;
  cpx<R>* buf_v = buf_u + RS;
  const int items = (ny + RB - 1) / RB;
  const int total = items * mem.count;
  // every thread: its share of the (N + 1) 16-byte segments (both rows at one
  // q) of item it2's row pair
  auto prefetch = [&](int it2) {
    const int mi2 = it2 / items;
    const cpx<R>* src = ws_ptr<cpx<R>>(member_at(mem, mi2), off.A) +
                        Tile<R>::at((it2 - mi2 * items) * RB, 0, ldqA);
    for (int q = tid; q <= N; q += T) cp_async16(land + 2 * q, src + size_t(q) * Tile<R>::TR);
    if (bpf) {
      const cpx<R>* srs = ws_ptr<cpx<R>>(member_at(mem, mi2), off.B) +
                          Tile<R>::at((it2 - mi2 * items) * RB, 0, ldqB);
      for (int q = tid; q <= Q; q += T) cp_async16(land_s + 2 * q, srs + size_t(q) * Tile<R>::TR);
    }
    cp_async_commit();
  };
  if constexpr (PF)
    if (vb < total) prefetch(vb);
#pragma unroll 1
  for (int it = vb; it < total; it += vg) {
    if (it + vg >= total) grid_dep_trigger();  // last item of this CTA
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    const cpx<R>* __restrict__ A = ws_ptr<cpx<R>>(mb, off.A);
    const cpx<R>* __restrict__ St = ws_ptr<cpx<R>>(mb, off.B);
    const int row0 = item * RB;
    const int row = row0 + rr;
    const bool valid = row < ny;
    const R dy = valid ? decon_y[row] : R(0);
    // U(q) = W(q) + W(q + N) and V(q) = (W(q) - W(q + N)) e^{+2 pi i q/M} for
    // the q = t + G m this thread owns in the first FFT stage, formed in
    // registers.  W(q + N) is W(N) for q = 0 and built from the conjugates at
    // the mirror N - q otherwise.  Without the prefetch each Y(q), q < N, is
    // loaded once (all loads of the row are issued together) and its mirror is
    // taken from the other thread through shared memory; with it both come
    // from the landing buffer.  The few band values S are loaded directly.
    const cpx<R> z = mk<R>(R(0), R(0));
    cpx<R> a[16], b[16];
    // e^{-2 pi i q/M} for q = t + G m (the inverse uses its conjugate)
    auto twq = [&](int m) {
      cpx<R> w;
      if constexpr (PF) {
        w = wtab[t + G * (m & 7)];
        if (m >= 8) w = mk<R>(w.y, -w.x);  // -i e^{-2 pi i (q - N/2)/M}
      } else if constexpr (GG::ROW_TAB) {
        w = wtab[t + G * m];
      } else {
        w = twm(ax, t + G * m);
      }
      return w;
    };
    if constexpr (PF) {
      cp_async_wait_all();
      __syncthreads();  // the row pair has landed; the previous transform's last-stage loads are done
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int q = t + G * m;
        const int qm = (q == 0) ? N : N - q;
        // band values: prefetched (bpf) or loaded here
        cpx<R> sv = z, sh = z;
        if (q <= Q) sv = bpf ? land_s[2 * q + rr] : St[Tile<R>::at(row, q, ldqB)];
        if (qm <= Q) sh = bpf ? land_s[2 * qm + rr] : St[Tile<R>::at(row, qm, ldqB)];
        const cpx<R> y = land[2 * q + rr];
        cpx<R> yh = land[2 * qm + rr];
        if (q != 0) {
          yh = conj(yh);
          sh = conj(sh);
        }
        const cpx<R> wlo = y + mul_i(sv, si);
        const cpx<R> whi = yh + mul_i(sh, si);
        a[m] = wlo + whi;
        const cpx<R> d = wlo - whi, w = twq(m);
        b[m] = cj ? cmul(d, w) : cmulc(d, w);
      }
      __syncthreads();  // every thread has read the landing buffer
      if (it + vg < total) prefetch(it + vg);
    } else {
      cpx<R> y[16], s[16], sm2[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int q = t + G * m;
        const int qm = (q == 0) ? N : N - q;
        y[m] = valid ? A[Tile<R>::at(row, q, ldqA)] : z;
        s[m] = (valid && q <= Q) ? St[Tile<R>::at(row, q, ldqB)] : z;
        sm2[m] = (valid && qm <= Q) ? St[Tile<R>::at(row, qm, ldqB)] : z;
      }
      const cpx<R> yN = (valid && t == 0) ? A[Tile<R>::at(row, N, ldqA)] : z;
      __syncthreads();  // the previous transform's last-stage loads of buf_u are done
#pragma unroll
      for (int m = 0; m < 16; ++m) buf_u[pad16(t + G * m)] = y[m];
      __syncthreads();
      cpx<R> ym[16];
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int q = t + G * m;
        ym[m] = (q == 0) ? yN : buf_u[pad16(N - q)];
      }
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int q = t + G * m;
        cpx<R> yh = ym[m], sh = sm2[m];
        if (q != 0) {
          yh = conj(yh);
          sh = conj(sh);
        }
        const cpx<R> wlo = y[m] + mul_i(s[m], si);
        const cpx<R> whi = yh + mul_i(sh, si);
        a[m] = wlo + whi;
        const cpx<R> d = wlo - whi, w = twq(m);
        b[m] = cj ? cmul(d, w) : cmulc(d, w);
      }
    }
    block_fft2_regs<R, LOG2N, PF>(a, b, buf_u, buf_v, t, stw, cj == 0);
    double* __restrict__ phi = mb.phi;
    if (valid) {
      // slot m holds T(2 (t + G m)) in a and T(2 (t + G m) + 1) in b; n < N for m < 8
      if (sizeof(R) == 4 && acc64) {
        const R dys = dy * scale;
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int n = 2 * (t + G * m);
          const R ia = cj ? -a[m].y : a[m].y;
          const R ib = cj ? -b[m].y : b[m].y;
          double2 out;
          out.x = add_f32_f64(float(a[m].x * scale), float(ia * R(dec[m].x) * dys));
          out.y = add_f32_f64(float(b[m].x * scale), float(ib * R(dec[m].y) * dys));
          *reinterpret_cast<double2*>(phi + size_t(row) * N + n) = out;
        }
      } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int n = 2 * (t + G * m);
          const R ia = cj ? -a[m].y : a[m].y;
          const R ib = cj ? -b[m].y : b[m].y;
          double2 out;
          const R d0 = (sizeof(R) == 4) ? R(dec[m & (ND - 1)].x) : ax.decon[n];
          const R d1 = (sizeof(R) == 4) ? R(dec[m & (ND - 1)].y) : ax.decon[n + 1];
          out.x = to_f64<R>((a[m].x + ia * d0 * dy) * scale);
          out.y = to_f64<R>((b[m].x + ib * d1 * dy) * scale);
          *reinterpret_cast<double2*>(phi + size_t(row) * N + n) = out;
        }
      }
    }
  }
}

template <typename R, int LOG2N>
__global__ void __launch_bounds__(Geo<R, LOG2N>::T_RI, min_blocks<R>(Geo<R, LOG2N>::MINB_I))
k_row_inv(Members mem, WsOff off, int ldqA, int ldqB, int Q, int ny, AxisTabs<R> ax,
          const R* __restrict__ decon_y, R scale, int cj, int bpf, int acc64) {
  row_inv_body<R, LOG2N>(blockIdx.x, gridDim.x, mem, off, ldqA, ldqB, Q, ny, ax, decon_y, scale, cj, bpf, acc64);
}

}  // namespace dsnu
