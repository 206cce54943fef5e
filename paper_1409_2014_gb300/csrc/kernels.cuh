// kernels.cuh -- the split-solver pipeline for one density (Sec. 2.1).
//
// Notation: N x N physical grid (nx, ny), padded/fine grid M = 2N per axis,
// natural frequency index q in [0, M) with signed value q - M for q >= N.
// Per solve, with rho real:
//
//   k_row_fwd : per row, z = rho + i b with b = rho * dx(x) dy(y) (ES
//               deconvolution, the type-2 prefactor); one length-M DFT of the
//               zero-padded z; the two real-signal spectra are separated
//               (A = row DFT of rho for q in [0, N], B = row DFT of b for
//               q in [0, Q]).                               [I1 and eq. 2.2 prep]
//   k_col_main: per column q_x in [0, N] of A: column DFT (length M, N inputs),
//               times m1 = (1 - p) (-k_x^2/|k|^2) (eq. SubInt1), inverse
//               column DFT keeping N rows; in place.               [I1]
//   k_band_fwd: per column q_x in [0, Q] of B: column DFT, keep |q_y| <= Q.
//   k_interp  : rho_hat(k_j) = sum over the w x w ES stencil of the band
//               (type-2 NUFFT, eq. 2.2); c_j = D_j rho_hat_j with the polar
//               weights of eq. I2PolarDisc (FP64 multiply).
//   k_spread  : S(q) = sum_j c_j phi(u_j - q) on the band (type-1 NUFFT
//               spreading, eq. 2.1), gathered per tile from a node list
//               (no atomics).
//   k_band_inv: per band column: inverse column DFT of S, N rows.
//   k_row_inv : per row: one inverse length-M DFT of
//               W = Y + i S (Hermitian extension of both), keeping N points;
//               Phi = [Re T + Im T dx dy] / (Mx My)   (I1 + I2, eq. PotSplitWhoSpace).
//
// `cj` = 1 runs the same pipeline with every complex constant conjugated
// (DFT signs, the packing unit i, the centring phases): for real input this is
// the transposed operator (type-1 <-> type-2 transposed pair), see
// dsnu_solve_adjoint.
#pragma once

#include "common.cuh"

namespace dsnu {

constexpr int kThreads = 512;  // every FFT-bearing kernel: 512 threads, 16 values per thread per FFT

template <typename R>
struct AxisTabs {
  const cpx<R>* twN;   // e^{-2 pi i m/N}, m < N
  const cpx<R>* twM;   // e^{-2 pi i n/M}, n < N
  const R* decon;      // phi_hat(0) / phi_hat(2 pi (n - N/2)/M), n < N
};

template <typename R>
struct MultTabs {
  const R* wx2;  // (q_x dk_x)^2, q_x in [0, nx]
  const R* gx;   // 1 - exp(-(q_x dk_x)^2 / sigma^2)
  const R* wy2;  // (qbar_y dk_y)^2, natural q_y in [0, My)
  const R* gy;
  int sharp;     // 1: p = indicator of |k| <= P
  R cut2;        // P^2
};

// m1 = -(k_x^2/|k|^2) (1 - p(k)), m1(0) = 0.  With the Gaussian partition
// 1 - p = 1 - e^{-kx^2/s^2} e^{-ky^2/s^2} = gx + gy (1 - gx), a sum of
// non-negative terms (no cancellation near k = 0).
template <typename R>
__device__ __forceinline__ R mult_high(const MultTabs<R>& mt, int qx, int qy_nat) {
  const R wx2 = mt.wx2[qx], wy2 = mt.wy2[qy_nat];
  const R s = wx2 + wy2;
  if (s == R(0)) return R(0);
  R part;
  if (mt.sharp) {
    part = (s > mt.cut2) ? R(1) : R(0);
  } else {
    const R gx = mt.gx[qx], gy = mt.gy[qy_nat];
    part = gx + gy * (R(1) - gx);
  }
  return -(wx2 / s) * part;
}

template <int LOG2N>
struct Geo {
  static constexpr int N = 1 << LOG2N;
  static constexpr int M = 2 * N;
  static constexpr int G = N / 16;          // threads per length-N FFT
  static constexpr int PER_CTA = 4096 / N;  // rows (or columns) per CTA
  static_assert(LOG2N >= 4 && LOG2N <= 12, "grid size 16..4096");
};

template <typename R>
constexpr size_t fft_smem_bytes() { return size_t(2) * 4096 * sizeof(cpx<R>); }

// ---------------------------------------------------------------------------
template <typename R, int LOG2N>
__global__ void __launch_bounds__(kThreads)
k_row_fwd(const double* __restrict__ rho, cpx<R>* __restrict__ A, int lda,
          cpx<R>* __restrict__ Brow, int ldb, int Q, int ny, AxisTabs<R> ax,
          const R* __restrict__ decon_y, int cj) {
  using GG = Geo<LOG2N>;
  constexpr int N = GG::N, G = GG::G, RPC = GG::PER_CTA;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * RPC;
  const R isg = cj ? R(-1) : R(1);
  for (int idx = tid; idx < RPC * N; idx += kThreads) {
    const int rl = idx >> LOG2N, n = idx & (N - 1), row = row0 + rl;
    R v = R(0), b = R(0);
    if (row < ny) {
      v = R(rho[(size_t)row * N + n]);
      b = v * ax.decon[n] * decon_y[row];
    }
    const cpx<R> z = mk<R>(v, isg * b);
    cpx<R> w = ax.twM[n];
    w.y *= isg;
    sm[(2 * rl) * N + n] = z;
    sm[(2 * rl + 1) * N + n] = cmul(z, w);
  }
  __syncthreads();
  block_fft<R, LOG2N>(sm + (tid / G) * N, tid % G, true, ax.twN, cj != 0);
  for (int idx = tid; idx < RPC * (N + 1); idx += kThreads) {
    const int rl = idx / (N + 1), q = idx - rl * (N + 1), row = row0 + rl;
    if (row >= ny) continue;
    const cpx<R>* E = sm + (2 * rl) * N;
    const cpx<R>* O = E + N;
    const cpx<R> zq = (q & 1) ? O[q >> 1] : E[q >> 1];
    const cpx<R> zm = (q == 0) ? E[0] : ((q & 1) ? O[N - ((q + 1) >> 1)] : E[N - (q >> 1)]);
    A[(size_t)row * lda + q] = mk<R>(R(0.5) * (zq.x + zm.x), R(0.5) * (zq.y - zm.y));
    if (q <= Q) {
      const cpx<R> d = mk<R>(zq.x - zm.x, zq.y + zm.y);  // Z(q) - conj Z(M - q)
      // divide by 2 i (2 (-i) in the conjugated pipeline)
      Brow[(size_t)row * ldb + q] = cj ? mk<R>(R(-0.5) * d.y, R(0.5) * d.x)
                                       : mk<R>(R(0.5) * d.y, R(-0.5) * d.x);
    }
  }
}

// ---------------------------------------------------------------------------
template <typename R, int LOG2N>
__global__ void __launch_bounds__(kThreads)
k_col_main(cpx<R>* __restrict__ A, int lda, int ncols, AxisTabs<R> ay, MultTabs<R> mt, int cj) {
  using GG = Geo<LOG2N>;
  constexpr int N = GG::N, G = GG::G, CPC = GG::PER_CTA;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * CPC;
  const R isg = cj ? R(-1) : R(1);
  for (int idx = tid; idx < CPC * N; idx += kThreads) {
    const int cl = idx & (CPC - 1), n = idx / CPC, col = c0 + cl;
    cpx<R> x = mk<R>(R(0), R(0));
    if (col < ncols) x = A[(size_t)n * lda + col];
    cpx<R> w = ay.twM[n];
    w.y *= isg;
    sm[(2 * cl) * N + n] = x;
    sm[(2 * cl + 1) * N + n] = cmul(x, w);
  }
  __syncthreads();
  block_fft<R, LOG2N>(sm + (tid / G) * N, tid % G, true, ay.twN, cj != 0);
  for (int idx = tid; idx < 2 * CPC * N; idx += kThreads) {
    const int chn = idx >> LOG2N, k = idx & (N - 1);
    const int col = c0 + (chn >> 1);
    const R m = (col < ncols) ? mult_high(mt, col, 2 * k + (chn & 1)) : R(0);
    sm[idx] = sm[idx] * m;
  }
  __syncthreads();
  block_fft<R, LOG2N>(sm + (tid / G) * N, tid % G, true, ay.twN, cj == 0);
  for (int idx = tid; idx < CPC * N; idx += kThreads) {
    const int cl = idx & (CPC - 1), n = idx / CPC, col = c0 + cl;
    if (col >= ncols) continue;
    const cpx<R> e = sm[(2 * cl) * N + n], o = sm[(2 * cl + 1) * N + n];
    const cpx<R> w = ay.twM[n];
    A[(size_t)n * lda + col] = cj ? e + cmul(o, w) : e + cmulc(o, w);
  }
}

// ---------------------------------------------------------------------------
template <typename R, int LOG2N>
__global__ void __launch_bounds__(kThreads)
k_band_fwd(const cpx<R>* __restrict__ Brow, int ldb, int ncols, cpx<R>* __restrict__ Bband,
           int ldq, int Q, AxisTabs<R> ay, int cj) {
  using GG = Geo<LOG2N>;
  constexpr int N = GG::N, M = GG::M, G = GG::G, CPC = GG::PER_CTA;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * CPC;
  const R isg = cj ? R(-1) : R(1);
  for (int idx = tid; idx < CPC * N; idx += kThreads) {
    const int cl = idx & (CPC - 1), n = idx / CPC, col = c0 + cl;
    cpx<R> x = mk<R>(R(0), R(0));
    if (col < ncols) x = Brow[(size_t)n * ldb + col];
    cpx<R> w = ay.twM[n];
    w.y *= isg;
    sm[(2 * cl) * N + n] = x;
    sm[(2 * cl + 1) * N + n] = cmul(x, w);
  }
  __syncthreads();
  block_fft<R, LOG2N>(sm + (tid / G) * N, tid % G, true, ay.twN, cj != 0);
  const int nq = 2 * Q + 1;
  for (int idx = tid; idx < CPC * nq; idx += kThreads) {
    const int cl = idx / nq, s = idx - cl * nq - Q, col = c0 + cl;
    if (col >= ncols) continue;
    const int q = s < 0 ? s + M : s;
    const cpx<R>* E = sm + (2 * cl) * N;
    Bband[(size_t)col * ldq + s + Q] = (q & 1) ? E[N + (q >> 1)] : E[q >> 1];
  }
}

// ---------------------------------------------------------------------------
// Type-2 interpolation: one warp per polar node.
template <typename R>
__global__ void __launch_bounds__(256)
k_interp(const cpx<R>* __restrict__ Bband, int ldq, int Q, const int2* __restrict__ q0,
         const R* __restrict__ wts, const double* __restrict__ D, int n_nodes, int w,
         cpx<R>* __restrict__ c, int cj) {
  const int lane = threadIdx.x & 31;
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (j >= n_nodes) return;
  const int2 b0 = q0[j];
  const R* wx = wts + (size_t)j * 2 * w;
  const R* wy = wx + w;
  R ax = R(0), ay = R(0);
  for (int p = lane; p < w * w; p += 32) {
    const int b = p / w, a = p - b * w;
    const int qx = b0.x + a, qy = b0.y + b;
    cpx<R> v;
    if (qx >= 0) {
      v = Bband[(size_t)qx * ldq + qy + Q];
    } else {
      v = conj(Bband[(size_t)(-qx) * ldq + (Q - qy)]);
    }
    const int e = qx + qy;
    v = mul_ipow(v, cj ? -e : e);  // centring phase i^{q_x + q_y}
    const R f = wx[a] * wy[b];
    ax += f * v.x;
    ay += f * v.y;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ax += __shfl_xor_sync(0xffffffffu, ax, off);
    ay += __shfl_xor_sync(0xffffffffu, ay, off);
  }
  if (lane == 0) {
    const double d = D[j];
    c[j] = mk<R>(R(d * double(ax)), R(d * double(ay)));
  }
}

// ---------------------------------------------------------------------------
// Type-1 spreading as a gather: one CTA per 16 x 16 tile of band cells; the
// nodes whose stencil meets the tile are listed at plan time.
constexpr int kTile = 16;
constexpr int kSpreadChunk = 64;

template <typename R>
__global__ void __launch_bounds__(256)
k_spread(const cpx<R>* __restrict__ c, const int2* __restrict__ q0, const R* __restrict__ wts,
         int w, const int* __restrict__ tile_ptr, const int* __restrict__ tile_nodes,
         int tiles_x, int Q, cpx<R>* __restrict__ Sband, int ldq, int cj) {
  __shared__ int2 s_q0[kSpreadChunk];
  __shared__ cpx<R> s_c[kSpreadChunk];
  __shared__ R s_w[kSpreadChunk * 32];
  const int tile = blockIdx.x;
  const int tx = tile % tiles_x, ty = tile / tiles_x;
  const int qx = tx * kTile + (threadIdx.x & (kTile - 1));
  const int qy = ty * kTile + (threadIdx.x / kTile) - Q;
  R ax = R(0), ay = R(0);
  const int beg = tile_ptr[tile], end = tile_ptr[tile + 1];
  const int w2 = 2 * w;
  for (int s0 = beg; s0 < end; s0 += kSpreadChunk) {
    const int cnt = min(kSpreadChunk, end - s0);
    for (int i = threadIdx.x; i < cnt; i += 256) {
      const int j = tile_nodes[s0 + i];
      s_q0[i] = q0[j];
      s_c[i] = c[j];
    }
    for (int i = threadIdx.x; i < cnt * w2; i += 256) {
      const int jj = i / w2, a = i - jj * w2;
      s_w[jj * 32 + a] = wts[(size_t)tile_nodes[s0 + jj] * w2 + a];
    }
    __syncthreads();
    for (int i = 0; i < cnt; ++i) {
      const int a = qx - s_q0[i].x, b = qy - s_q0[i].y;
      if ((unsigned)a < (unsigned)w && (unsigned)b < (unsigned)w) {
        const R f = s_w[i * 32 + a] * s_w[i * 32 + w + b];
        ax += f * s_c[i].x;
        ay += f * s_c[i].y;
      }
    }
    __syncthreads();
  }
  if (qx <= Q && qy <= Q) {
    const int e = qx + qy;
    Sband[(size_t)qx * ldq + qy + Q] = mul_ipow(mk<R>(ax, ay), cj ? e : -e);  // (-i)^{q_x+q_y}
  }
}

// ---------------------------------------------------------------------------
template <typename R, int LOG2N>
__global__ void __launch_bounds__(kThreads)
k_band_inv(const cpx<R>* __restrict__ Sband, int ldq, int Q, int ncols, cpx<R>* __restrict__ Scol,
           int ldb, AxisTabs<R> ay, int cj) {
  using GG = Geo<LOG2N>;
  constexpr int N = GG::N, M = GG::M, G = GG::G, CPC = GG::PER_CTA;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * CPC;
  for (int idx = tid; idx < 2 * CPC * N; idx += kThreads) {
    const int chn = idx >> LOG2N, k = idx & (N - 1);
    const int col = c0 + (chn >> 1);
    const int q = 2 * k + (chn & 1);
    const int s = q < N ? q : q - M;
    cpx<R> v = mk<R>(R(0), R(0));
    if (col < ncols && s >= -Q && s <= Q) v = Sband[(size_t)col * ldq + s + Q];
    sm[idx] = v;
  }
  __syncthreads();
  block_fft<R, LOG2N>(sm + (tid / G) * N, tid % G, true, ay.twN, cj == 0);
  for (int idx = tid; idx < CPC * N; idx += kThreads) {
    const int cl = idx & (CPC - 1), n = idx / CPC, col = c0 + cl;
    if (col >= ncols) continue;
    const cpx<R> e = sm[(2 * cl) * N + n], o = sm[(2 * cl + 1) * N + n];
    const cpx<R> w = ay.twM[n];
    Scol[(size_t)n * ldb + col] = cj ? e + cmul(o, w) : e + cmulc(o, w);
  }
}

// ---------------------------------------------------------------------------
template <typename R, int LOG2N>
__global__ void __launch_bounds__(kThreads)
k_row_inv(const cpx<R>* __restrict__ A, int lda, const cpx<R>* __restrict__ Scol, int ldb, int Q,
          double* __restrict__ phi, int ny, AxisTabs<R> ax, const R* __restrict__ decon_y, R scale,
          int cj) {
  using GG = Geo<LOG2N>;
  constexpr int N = GG::N, M = GG::M, G = GG::G, RPC = GG::PER_CTA;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* sm = reinterpret_cast<cpx<R>*>(smem_raw);
  const int tid = threadIdx.x;
  const int row0 = blockIdx.x * RPC;
  const int si = cj ? -1 : 1;
  for (int idx = tid; idx < RPC * M; idx += kThreads) {
    const int rl = idx >> (LOG2N + 1), q = idx & (M - 1), row = row0 + rl;
    cpx<R> W = mk<R>(R(0), R(0));
    if (row < ny) {
      const bool lo = q <= N;
      const int qq = lo ? q : M - q;
      cpx<R> y = A[(size_t)row * lda + qq];
      cpx<R> s = (qq <= Q) ? Scol[(size_t)row * ldb + qq] : mk<R>(R(0), R(0));
      if (!lo) { y = conj(y); s = conj(s); }
      W = y + mul_i(s, si);
    }
    sm[(2 * rl + (q & 1)) * N + (q >> 1)] = W;
  }
  __syncthreads();
  block_fft<R, LOG2N>(sm + (tid / G) * N, tid % G, true, ax.twN, cj == 0);
  for (int idx = tid; idx < RPC * N; idx += kThreads) {
    const int rl = idx >> LOG2N, n = idx & (N - 1), row = row0 + rl;
    if (row >= ny) continue;
    const cpx<R> e = sm[(2 * rl) * N + n], o = sm[(2 * rl + 1) * N + n];
    const cpx<R> w = ax.twM[n];
    const cpx<R> T = cj ? e + cmul(o, w) : e + cmulc(o, w);
    const R im = cj ? -T.y : T.y;
    const R val = (T.x + im * ax.decon[n] * decon_y[row]) * scale;
    phi[(size_t)row * N + n] = double(val);
  }
}

}  // namespace dsnu
