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
};

template <typename R, int LOG2N>
__global__ void __launch_bounds__(GeoStd<R, LOG2N>::T, min_blocks<R>(2))
k_std_row_fwd(Members mem, size_t offH, int ldq, int ny, const cpx<R>* __restrict__ stw_g, int cj) {
  using GG = GeoStd<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, PER = GG::PER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  copy_to_smem(stw, stw_g, GG::STW);
  const int tid = threadIdx.x;
  const int rr = tid / G, t = tid - rr * G;
  cpx<R>* buf = stw + GG::STWP + rr * GG::FB;
  const int pairs = ny / 2;
  const int items = (pairs + PER - 1) / PER;
#pragma unroll 1
  for (int it = blockIdx.x; it < items * mem.count; it += gridDim.x) {
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    cpx<R>* __restrict__ H = ws_ptr<cpx<R>>(mb, offH);
    const int pr = item * PER + rr;
    const bool valid = pr < pairs;
    const int row = 2 * pr;
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int n = t + G * m;
      const R a = valid ? from_f64<R>(mb.rho[size_t(row) * N + n]) : R(0);
      const R b = valid ? from_f64<R>(mb.rho[size_t(row + 1) * N + n]) : R(0);
      v[m] = mk<R>(a, b);
    }
    block_fft_regs<R, LOG2N>(v, buf, t, stw, cj != 0);
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
        dst[0] = xa;
        dst[1] = xb;
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
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  copy_to_smem(stw, stw_g, GG::STW);
  const int tid = threadIdx.x;
  const int cl = tid / G, t = tid - cl * G;
  cpx<R>* buf = stw + GG::STWP + cl * GG::FB;
  const int items = (ncols + PER - 1) / PER;
#pragma unroll 1
  for (int it = blockIdx.x; it < items * mem.count; it += gridDim.x) {
    const int mi = it / items, item = it - mi * items;
    cpx<R>* __restrict__ H = ws_ptr<cpx<R>>(member_at(mem, mi), offH);
    const int col = item * PER + cl;
    const bool valid = col < ncols;
    const R kx2 = valid ? mt.wx2[col] : R(0);
    const R kxc = (valid && mt.generic) ? mt.kx[col] : R(0);
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = valid ? H[Tile<R>::at(t + G * m, col, ldq)] : mk<R>(R(0), R(0));
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
  constexpr int N = GG::N, G = GG::G, PER = GG::PER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  copy_to_smem(stw, stw_g, GG::STW);
  const int tid = threadIdx.x;
  const int rr = tid / G, t = tid - rr * G;
  cpx<R>* buf = stw + GG::STWP + rr * GG::FB;
  const int pairs = ny / 2;
  const int items = (pairs + PER - 1) / PER;
#pragma unroll 1
  for (int it = blockIdx.x; it < items * mem.count; it += gridDim.x) {
    const int mi = it / items, item = it - mi * items;
    const Member mb = member_at(mem, mi);
    const cpx<R>* __restrict__ H = ws_ptr<cpx<R>>(mb, offH);
    const int pr = item * PER + rr;
    const bool valid = pr < pairs;
    const int row = 2 * pr;
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      const int q = t + G * m;
      const bool hi = q > N / 2;
      const int qq = hi ? N - q : q;
      cpx<R> ya = mk<R>(R(0), R(0)), yb = ya;
      if (valid) {
        const cpx<R>* src = H + Tile<R>::at(row, qq, ldq);
        ya = src[0];
        yb = src[1];
      }
      if (hi) {
        ya = conj(ya);
        yb = conj(yb);
      }
      v[m] = mk<R>(ya.x - yb.y, ya.y + yb.x);  // Y_a + i Y_b
    }
    block_fft_regs<R, LOG2N>(v, buf, t, stw, cj == 0);
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
