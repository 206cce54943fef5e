// standard.cuh -- the standard periodic FFT solver that the paper compares the
// split solver against (Sec. 2.1 and Table 1): on the unpadded N_x x N_y grid,
//     Phi = IDFT[ m(k) DFT[rho] ],   m(k) = -k_x^2/|k|^2,  m(0) = 0,
// with k the FFT frequencies of the periodic box (dk = pi/l per axis).  No
// splitting, no padding (kappa = 1, p = 0): its error is set by the domain
// truncation, which is what Table 1 shows.
//
// Three kernels, all length-N transforms from common.cuh:
//   k_std_row_fwd : two real rows per transform (z = rho_a + i rho_b), the two
//                   half spectra q in [0, N_x/2] separated by Hermitian
//                   symmetry and stored row-tiled (both rows in one store);
//   k_std_col     : per half-spectrum column: DFT along y, times m / (N_x N_y),
//                   inverse DFT along y, in place (m: the DS multiplier or
//                   the generic family of MultTabs);
//   k_std_row_inv : two rows per transform again (W = Y_a + i Y_b, each
//                   extended to q > N_x/2 by conjugate symmetry); the real and
//                   imaginary parts of the inverse are the two rows of Phi.
// `cj` = 1 conjugates every transform (the transposed operator, equal to the
// operator itself since m is real and even).
//
// FP32 plans (PF): the row passes read their inputs from shared-memory
// landing buffers filled while the previous item is transformed (a bulk copy
// of the item's rows of rho; cp.async of the row pairs' 16-byte segments of the
// half spectrum), with the compact stage table making room; the column pass
// (N >= 512) loads its next column into registers during the current inverse
// transform.
// All three are launched with programmatic stream serialization.
#pragma once

#include "kernels.cuh"

namespace dsnu {

template <typename R, int LOG2N>
struct GeoStd {
  static constexpr int N = 1 << LOG2N;
  static constexpr int G = N / 16;                       // threads per transform
  static constexpr int FB = fft_buf_elems(N);
  static constexpr int PER = (G >= 256) ? 1 : 256 / G;   // row pairs or columns per CTA
  static constexpr int T = PER * G;
  static constexpr int STW = fft_stage_tw_elems(LOG2N) > 0 ? fft_stage_tw_elems(LOG2N) : 1;
  static constexpr int STWP = (STW + 1) & ~1;
  static constexpr size_t smem = size_t(STWP + PER * FB) * sizeof(cpx<R>);
  static constexpr bool PF = sizeof(R) == 4;
  static constexpr int STWC = fft_stage_tw_elems_ct(LOG2N) > 0 ? fft_stage_tw_elems_ct(LOG2N) : 1;
  static constexpr int STWCP = (STWC + 1) & ~1;
  // forward rows: 2 PER rows of rho (FP64) and an mbarrier after the buffers
  static constexpr size_t smem_rowf =
      PF ? size_t(STWCP + PER * FB) * sizeof(cpx<R>) + size_t(2 * PER) * N * sizeof(double) + 16 : smem;
  // inverse rows: PER row pairs x (N/2 + 1) segments of 16 bytes
  static constexpr size_t smem_rowi =
      PF ? size_t(STWCP + PER * FB) * sizeof(cpx<R>) + size_t(PER) * (N / 2 + 1) * 16 : smem;
};

template <typename R, int LOG2N>
__global__ void __launch_bounds__(GeoStd<R, LOG2N>::T, min_blocks<R>(2))
k_std_row_fwd(Members mem, size_t offH, int ldq, int ny, const cpx<R>* __restrict__ stw_g, int cj, int* status) {
  using GG = GeoStd<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, PER = GG::PER;
  constexpr bool PF = GG::PF;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  copy_to_smem(stw, stw_g, PF ? GG::STWC : GG::STW);
  const int tid = threadIdx.x;
  const int rr = tid / G, t = tid - rr * G;
  cpx<R>* buf = stw + (PF ? GG::STWCP : GG::STWP) + rr * GG::FB;
  double* land = reinterpret_cast<double*>(stw + (PF ? GG::STWCP : GG::STWP) + PER * GG::FB);  // PF: 2 PER rows
  unsigned long long* bar = reinterpret_cast<unsigned long long*>(land + 2 * PER * N);
  if constexpr (PF)
    if (tid == 0) mbar_init(bar, 1);
  __syncthreads();
  grid_dep_wait();
  const int pairs = ny / 2;
  const int items = (pairs + PER - 1) / PER;
  const int total = items * mem.count;
  // thread 0: the 2 PER rows of item it2 (contiguous in rho) in one bulk copy
  auto prefetch = [&](int it2) {
    const int mi2 = it2 / items;
    const int r0 = 2 * (it2 - mi2 * items) * PER;
    const unsigned bytes = unsigned(min(2 * PER, ny - r0)) * unsigned(N * sizeof(double));
    mbar_expect_tx(bar, bytes);
    bulk_load(land, member_at(mem, mi2).rho + size_t(r0) * N, bytes, bar, l2_evict_first());
  };
  if constexpr (PF)
    if (tid == 0 && int(blockIdx.x) < total) prefetch(blockIdx.x);
  unsigned phase = 0;
#pragma unroll 1
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    if (it + int(gridDim.x) >= total) grid_dep_trigger();  // last item of this CTA
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    cpx<R>* __restrict__ H = ws_ptr<cpx<R>>(mb, offH);
    const int pr = item * PER + rr;
    const bool valid = pr < pairs;
    const int row = 2 * pr;
    bool landed = true;
    if constexpr (PF) {
      // bounded wait (1 s); on expiry the CTA stops after the reads below
      landed = mbar_wait(bar, phase, 1000000000ull);
      phase ^= 1u;
    }
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = t + G * m;
      R a = R(0), b = R(0);
      if (valid) {
        if constexpr (PF) {
          a = from_f64<R>(land[(2 * rr) * N + n]);
          b = from_f64<R>(land[(2 * rr + 1) * N + n]);
        } else {
          a = from_f64<R>(mb.rho[size_t(row) * N + n]);
          b = from_f64<R>(mb.rho[size_t(row + 1) * N + n]);
        }
      }
      v[m] = mk<R>(a, b);
    }
    if constexpr (PF) {
      // every thread has read the landing buffer (a barrier); stop if a wait expired
      if (cta_timed_out(landed, bar, phase ^ 1u, status)) return;
      if (tid == 0 && it + int(gridDim.x) < total) prefetch(it + gridDim.x);
    }
    block_fft_regs<R, LOG2N, PF>(v, buf, t, stw, cj != 0);
    __syncthreads();  // the last stage's loads of buf are done
#pragma unroll
    for (int m = 0; m < 16; ++m) buf[pad16(t + G * m)] = v[m];
    __syncthreads();
    if (valid) {
      for (int q = t; q <= N / 2; q += G) {
        const cpx<R> zq = buf[pad16(q)];
        const cpx<R> zm = buf[pad16((N - q) & (N - 1))];
        // X_a = (Z(q) + conj Z(N - q)) / 2,  X_b = (Z(q) - conj Z(N - q)) / (2i)
        const cpx<R> xa = mk<R>(R(0.5) * (zq.x + zm.x), R(0.5) * (zq.y - zm.y));
        const cpx<R> xb = mk<R>(R(0.5) * (zq.y + zm.y), R(-0.5) * (zq.x - zm.x));
        cpx<R>* dst = H + Tile<R>::at(row, q, ldq);  // row + 1 is the next element
        if constexpr (sizeof(R) == 4) {              // (16-byte aligned: row is even)
          *reinterpret_cast<float4*>(dst) = make_float4(xa.x, xa.y, xb.x, xb.y);
        } else {
          dst[0] = xa;
          dst[1] = xb;
        }
      }
    }
  }
}

template <typename R, int LOG2N>
__global__ void __launch_bounds__(GeoStd<R, LOG2N>::T, min_blocks<R>(2))
k_std_col(Members mem, size_t offH, int ldq, int ncols, const cpx<R>* __restrict__ stw_g,
          MultTabs<R> mt, R scale, int cj) {
  using GG = GeoStd<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, PER = GG::PER;
  constexpr bool PF = GG::PF && LOG2N >= 9;  // (below, the registers for it are not there)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  copy_to_smem(stw, stw_g, GG::STW);
  const int tid = threadIdx.x;
  const int cl = tid / G, t = tid - cl * G;
  cpx<R>* buf = stw + GG::STWP + cl * GG::FB;
  __syncthreads();
  grid_dep_wait();
  const int items = (ncols + PER - 1) / PER;
  const int total = items * mem.count;
  // PF: the next column's values are loaded into registers before the
  // current column's inverse transform
  cpx<R> xn[PF ? 16 : 1];
  auto load_col = [&](int it2) {
    const int mi2 = it2 / items;
    const int col2 = (it2 - mi2 * items) * PER + cl;
    const cpx<R>* H2 = ws_ptr<cpx<R>>(member_at(mem, mi2), offH);
#pragma unroll
    for (int m = 0; m < (PF ? 16 : 1); ++m)
      xn[m] = (col2 < ncols) ? H2[Tile<R>::at(t + G * m, col2, ldq)] : mk<R>(R(0), R(0));
  };
  if constexpr (PF)
    if (int(blockIdx.x) < total) load_col(blockIdx.x);
#pragma unroll 1
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    if (it + int(gridDim.x) >= total) grid_dep_trigger();  // last item of this CTA
    const int mi = it / items, item = it - mi * items;
    cpx<R>* __restrict__ H = ws_ptr<cpx<R>>(member_at(mem, mi), offH);
    const int col = item * PER + cl;
    const bool valid = col < ncols;
    const R kx2 = valid ? mt.wx2[col] : R(0);
    const R kxc = (valid && mt.generic) ? mt.kx[col] : R(0);
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      if constexpr (PF) v[m] = xn[m];
      else v[m] = valid ? H[Tile<R>::at(t + G * m, col, ldq)] : mk<R>(R(0), R(0));
    }
    block_fft_regs<R, LOG2N>(v, buf, t, stw, cj != 0);
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = t + G * m;  // natural order after the transform
      const int a = (q <= N / 2) ? q : N - q;
      const R wy2 = R(a * a) * mt.dky2;
      const R s = kx2 + wy2;
      R mlt;
      if (mt.generic)  // signed qbar for the sin 2theta term, 0 at the Nyquist row
        mlt = mult_generic(mt, kx2, wy2, kxc, (q < N / 2) ? q : (q == N / 2 ? 0 : q - N), s) * scale;
      else
        mlt = (s == R(0)) ? R(0) : -fdiv(kx2, s) * scale;
      v[m] = v[m] * mlt;
    }
    if constexpr (PF)
      if (it + int(gridDim.x) < total) load_col(it + gridDim.x);
    block_fft_regs<R, LOG2N>(v, buf, t, stw, cj == 0);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 16; ++m) H[Tile<R>::at(t + G * m, col, ldq)] = v[m];
    }
  }
}

template <typename R, int LOG2N>
__global__ void __launch_bounds__(GeoStd<R, LOG2N>::T, min_blocks<R>(2))
k_std_row_inv(Members mem, size_t offH, int ldq, int ny, const cpx<R>* __restrict__ stw_g, int cj) {
  using GG = GeoStd<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, PER = GG::PER, T = GG::T;
  constexpr bool PF = GG::PF;
  constexpr int HS = N / 2 + 1;  // segments per row pair
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  copy_to_smem(stw, stw_g, PF ? GG::STWC : GG::STW);
  const int tid = threadIdx.x;
  const int rr = tid / G, t = tid - rr * G;
  cpx<R>* buf = stw + (PF ? GG::STWCP : GG::STWP) + rr * GG::FB;
  // PF: Y_a(q), Y_b(q) of each row pair of the item at [2 (pair HS + q) + row]
  cpx<R>* land = stw + (PF ? GG::STWCP : GG::STWP) + PER * GG::FB;
  __syncthreads();
  grid_dep_wait();
  const int pairs = ny / 2;
  const int items = (pairs + PER - 1) / PER;
  const int total = items * mem.count;
  // every thread: its share of the item's PER x (N/2 + 1) 16-byte segments
  auto prefetch = [&](int it2) {
    const int mi2 = it2 / items;
    const int p0 = (it2 - mi2 * items) * PER;
    const cpx<R>* H2 = ws_ptr<cpx<R>>(member_at(mem, mi2), offH);
    for (int i = tid; i < PER * HS; i += T) {
      const int p = i / HS, q = i - p * HS;
      if (p0 + p < pairs) cp_async16(land + 2 * i, H2 + Tile<R>::at(2 * (p0 + p), q, ldq));
    }
    cp_async_commit();
  };
  if constexpr (PF)
    if (int(blockIdx.x) < total) prefetch(blockIdx.x);
#pragma unroll 1
  for (int it = blockIdx.x; it < total; it += gridDim.x) {
    if (it + int(gridDim.x) >= total) grid_dep_trigger();  // last item of this CTA
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    const cpx<R>* __restrict__ H = ws_ptr<cpx<R>>(mb, offH);
    const int pr = item * PER + rr;
    const bool valid = pr < pairs;
    const int row = 2 * pr;
    if constexpr (PF) {
      cp_async_wait_all();
      __syncthreads();  // the item's segments have landed
    }
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = t + G * m;
      const bool hi = q > N / 2;
      const int qq = hi ? N - q : q;
      cpx<R> ya = mk<R>(R(0), R(0)), yb = ya;
      if (valid) {
        const cpx<R>* src = PF ? land + 2 * (rr * HS + qq) : H + Tile<R>::at(row, qq, ldq);
        ya = src[0];
        yb = src[1];
      }
      if (hi) {
        ya = conj(ya);
        yb = conj(yb);
      }
      v[m] = mk<R>(ya.x - yb.y, ya.y + yb.x);  // Y_a + i Y_b
    }
    if constexpr (PF) {
      __syncthreads();  // every thread has read the landing buffer
      if (it + int(gridDim.x) < total) prefetch(it + gridDim.x);
    }
    block_fft_regs<R, LOG2N, PF>(v, buf, t, stw, cj == 0);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 16; ++m) {
        const int n = t + G * m;
        mb.phi[size_t(row) * N + n] = to_f64<R>(v[m].x);
        mb.phi[size_t(row + 1) * N + n] = to_f64<R>(v[m].y);
      }
    }
  }
}

}  // namespace dsnu
