// common.cuh -- complex type and the in-CTA FFT used by every pipeline kernel.
//
// The split solver (Sec. 2.1 of the paper) needs, per grid row or column, a
// length-M = 2N DFT of data that is non-zero on N points only (the kappa = 2
// zero padding of I1, which is also the upsampling-2 fine grid of both NUFFTs),
// or an inverse length-M DFT of which only N outputs are kept.  Both reduce to
// two length-N DFTs (the even and the odd output frequencies):
//     Z(2k)   = DFT_N[z](k),     Z(2k+1) = DFT_N[z(n) w_M^n](k),   w_M = e^{-2 pi i/M}
//     T(n)    = IDFT_N[W(2k)](n) + w_M^{-n} IDFT_N[W(2k+1)](n),      n < N
// so the only transform primitive is a length-N complex DFT (Sec. 2.2, the
// uniform DFT pair), done here by a group of N/16 threads of one CTA with the
// data in shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dsnufft.h"

namespace dsnu {

template <typename R>
struct alignas(2 * sizeof(R)) cpx {
  R x, y;
};

template <typename R>
__host__ __device__ __forceinline__ cpx<R> mk(R x, R y) { cpx<R> c; c.x = x; c.y = y; return c; }
template <typename R>
__device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return mk<R>(a.x + b.x, a.y + b.y); }
template <typename R>
__device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return mk<R>(a.x - b.x, a.y - b.y); }
template <typename R>
__device__ __forceinline__ cpx<R> operator*(cpx<R> a, R s) { return mk<R>(a.x * s, a.y * s); }
template <typename R>
__device__ __forceinline__ cpx<R> cmul(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename R>
__device__ __forceinline__ cpx<R> cmulc(cpx<R> a, cpx<R> b) {
  return mk<R>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename R>
__device__ __forceinline__ cpx<R> conj(cpx<R> a) { return mk<R>(a.x, -a.y); }
// multiply by +i (s = +1) or -i (s = -1)
template <typename R>
__device__ __forceinline__ cpx<R> mul_i(cpx<R> a, int s) { return s > 0 ? mk<R>(-a.y, a.x) : mk<R>(a.y, -a.x); }
// multiply by i^e, e taken mod 4
template <typename R>
__device__ __forceinline__ cpx<R> mul_ipow(cpx<R> a, int e) {
  switch (e & 3) {
    case 0: return a;
    case 1: return mk<R>(-a.y, a.x);
    case 2: return mk<R>(-a.x, -a.y);
    default: return mk<R>(a.y, -a.x);
  }
}

// ---------------------------------------------------------------------------
// Small forward DFTs in registers (e^{-2 pi i jk/RAD}), RAD = 2, 4, 8, 16,
// by radix-2 decimation in time with the constant twiddles of the 16th roots
// of unity written out: cos(pi/8) = sqrt(2+sqrt 2)/2, sin(pi/8) =
// sqrt(2-sqrt 2)/2, cos(pi/4) = sqrt(1/2).
// ---------------------------------------------------------------------------
constexpr double kC1_16 = 0.92387953251128675613;  // cos(2 pi/16)
constexpr double kS1_16 = 0.38268343236508977173;  // sin(2 pi/16)
constexpr double kR2 = 0.70710678118654752440;     // sqrt(1/2)

// x * e^{-2 pi i m/16}, m in [0, 8)
template <int M16, typename R>
__device__ __forceinline__ cpx<R> rot16(cpx<R> a) {
  if constexpr (M16 == 0) {
    return a;
  } else if constexpr (M16 == 4) {          // -i
    return mk<R>(a.y, -a.x);
  } else if constexpr (M16 == 2) {          // (1 - i)/sqrt2
    return mk<R>(R(kR2) * (a.x + a.y), R(kR2) * (a.y - a.x));
  } else if constexpr (M16 == 6) {          // (-1 - i)/sqrt2
    return mk<R>(R(kR2) * (a.y - a.x), R(-kR2) * (a.x + a.y));
  } else {
    // cos/sin of 2 pi m/16 for m = 1, 3, 5, 7
    constexpr double c = (M16 == 1) ? kC1_16 : (M16 == 3) ? kS1_16 : (M16 == 5) ? -kS1_16 : -kC1_16;
    constexpr double s = (M16 == 1) ? kS1_16 : (M16 == 3) ? kC1_16 : (M16 == 5) ? kC1_16 : kS1_16;
    // (x + i y)(c - i s)
    return mk<R>(a.x * R(c) + a.y * R(s), a.y * R(c) - a.x * R(s));
  }
}

// In-place forward DFT of v[0..RAD) (natural order in and out).
template <int RAD, typename R>
__device__ __forceinline__ void dft_rec(cpx<R> (&v)[RAD]) {
  if constexpr (RAD == 1) {
    return;
  } else if constexpr (RAD == 2) {
    cpx<R> a = v[0], b = v[1];
    v[0] = a + b;
    v[1] = a - b;
  } else {
    constexpr int H = RAD / 2;
    cpx<R> e[H], o[H];
#pragma unroll
    for (int i = 0; i < H; ++i) { e[i] = v[2 * i]; o[i] = v[2 * i + 1]; }
    dft_rec<H, R>(e);
    dft_rec<H, R>(o);
    constexpr int step = 16 / RAD;
    // twiddle o[k] by e^{-2 pi i k/RAD} = rot16<k*step>
    // (for the factor -i the sum and difference are written out: no multiply)
#define DSNU_TW(K)                                                         \
  if constexpr ((K) < H) {                                                 \
    constexpr int RK = ((K) * step) & 15;                                  \
    if constexpr (RK == 4) {                                               \
      v[(K)] = mk<R>(e[(K)].x + o[(K)].y, e[(K)].y - o[(K)].x);            \
      v[(K) + H] = mk<R>(e[(K)].x - o[(K)].y, e[(K)].y + o[(K)].x);        \
    } else {                                                               \
      cpx<R> t = rot16<RK, R>(o[(K)]);                                     \
      v[(K)] = e[(K)] + t;                                                 \
      v[(K) + H] = e[(K)] - t;                                             \
    }                                                                      \
  }
    DSNU_TW(0) DSNU_TW(1) DSNU_TW(2) DSNU_TW(3) DSNU_TW(4) DSNU_TW(5) DSNU_TW(6) DSNU_TW(7)
#undef DSNU_TW
  }
}

// ---------------------------------------------------------------------------
// Length-N DFT by a group of G = N/16 threads (t = 0..G-1), data in registers.
//
// On entry thread t holds v[m] = x[t + G m], m = 0..15; on return it holds
// v[m] = X[t + G m] (X = DFT_N[x], e^{-2 pi i nk/N}; with inv = true the
// unnormalised inverse e^{+2 pi i nk/N}, computed as conj(DFT(conj x))).
// Stockham autosort: radix-16 stages, then one radix-2/4/8 stage; the first
// stage reads the registers, the last leaves its outputs in registers, the
// stages in between exchange through `buf` (this group's shared-memory
// buffer of fft_buf_elems(N) elements, index i stored at i + i/16 so that
// every stage is free of bank conflicts).  Every thread of the CTA must call
// it the same number of times (it contains __syncthreads()).
//
// `stw` (normally in shared memory) holds the twiddles of stages 1.. in the
// order stage, r = 1..RAD-1, k = 0..NS-1:  e^{-2 pi i r k / (NS RAD)}, so that
// threads with consecutive k read consecutive entries.  They are generated in
// FP64 on the host (fft_stage_twiddles in plan.cu).
// ---------------------------------------------------------------------------
__host__ __device__ constexpr int fft_buf_elems(int n) { return n + n / 16; }
__device__ __forceinline__ int pad16(int i) { return i + (i >> 4); }

// Offset of stage `stage`'s twiddles in the stage table of a length-2^log2n
// transform (stages >= 1), and the table's total length (host + device).
__host__ __device__ constexpr int fft_stage_tw_offset(int log2n, int stage) {
  int total = 0;
  const int full = log2n / 4;
  for (int s = 1; s < stage; ++s) {
    const int lr = (s < full) ? 4 : (log2n - 4 * full);
    total += ((1 << lr) - 1) * (1 << (4 * s));
  }
  return total;
}
__host__ __device__ constexpr int fft_stage_tw_elems(int log2n) {
  return fft_stage_tw_offset(log2n, (log2n + 3) / 4);
}

// Compact stage table (the CT form of the transforms below): stage 1 as in
// the full table, then for the stage with NS = 256 (the third stage of
// N >= 512, radix RAD = N/256) two factors of (RAD - 1) x 16 entries each,
//   hi[r][k1] = e^{-2 pi i 16 r k1/(NS RAD)},  lo[r][k0] = e^{-2 pi i r k0/(NS RAD)},
// whose product is the twiddle of k = 16 k1 + k0: 720 entries at N = 4096
// instead of 4080.
__host__ __device__ constexpr int fft_stage_tw_elems_ct(int log2n) {
  return log2n <= 8 ? fft_stage_tw_elems(log2n) : 15 * 16 + 2 * 16 * ((1 << (log2n - 8)) - 1);
}

template <int LOG2N, int S>
struct StageInfo {
  static constexpr int full = LOG2N / 4;
  static constexpr int lr = (S < full) ? 4 : (LOG2N - 4 * full);
  static constexpr int nstages = (LOG2N + 3) / 4;
  static constexpr int log2ns = 4 * S;  // product of the previous radices
  static constexpr int tw_off = fft_stage_tw_offset(LOG2N, S);
};

template <typename R, int LOG2N, int S, bool CT = false>
__device__ __forceinline__ void fft_stage_regs(cpx<R> (&v)[16], cpx<R>* buf, int t,
                                               const cpx<R>* __restrict__ stw) {
  using SI = StageInfo<LOG2N, S>;
  constexpr int N = 1 << LOG2N;
  constexpr int LR = SI::lr;
  constexpr int RAD = 1 << LR;
  constexpr int NB = N / RAD;
  constexpr int G = N / 16;
  constexpr int PER = 16 / RAD;
  constexpr int LOG2NS = SI::log2ns;
  constexpr int NS = 1 << LOG2NS;
  constexpr bool FIRST = (S == 0);
  constexpr bool LAST = (S == SI::nstages - 1);
  if constexpr (!FIRST) {
    __syncthreads();  // previous stage's stores visible
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int j = t + b * G;
#pragma unroll
      for (int r = 0; r < RAD; ++r) v[b * RAD + r] = buf[pad16(j + r * NB)];
    }
  }
  // (stage 0 has RAD = 16, PER = 1 and v[r] = x[t + G r] = x[j + r NB] already)
#pragma unroll
  for (int b = 0; b < PER; ++b) {
    const int j = t + b * G;
    const int k = j & (NS - 1);
    if constexpr (CT && LOG2NS == 8) {  // compact table: w = hi[r][k >> 4] lo[r][k & 15]
      const cpx<R>* hi = stw + 15 * 16 + (k >> 4);
      const cpx<R>* lo = stw + 15 * 16 + (RAD - 1) * 16 + (k & 15);
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[b * RAD + r] = cmul(v[b * RAD + r], cmul(hi[(r - 1) * 16], lo[(r - 1) * 16]));
    } else if constexpr (LOG2NS > 0) {
      const cpx<R>* tws = stw + SI::tw_off + k;
#pragma unroll
      for (int r = 1; r < RAD; ++r) v[b * RAD + r] = cmul(v[b * RAD + r], tws[(r - 1) * NS]);
    }
    cpx<R> u[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) u[r] = v[b * RAD + r];
    dft_rec<RAD, R>(u);
#pragma unroll
    for (int r = 0; r < RAD; ++r) v[b * RAD + r] = u[r];
  }
  if constexpr (!LAST) {
    __syncthreads();  // every load of this buffer done (in place)
#pragma unroll
    for (int b = 0; b < PER; ++b) {
      const int j = t + b * G;
      const int k = j & (NS - 1);
      const int base = (j - k) * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) buf[pad16(base + r * NS)] = v[b * RAD + r];
    }
  } else {
    // slot b*RAD + r holds X[j_b + r NS] = X[t + G (b + r PER)]
    cpx<R> o[16];
#pragma unroll
    for (int b = 0; b < PER; ++b)
#pragma unroll
      for (int r = 0; r < RAD; ++r) o[b + r * PER] = v[b * RAD + r];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = o[m];
  }
}

template <typename R, int LOG2N, int S, bool CT = false>
__device__ __forceinline__ void fft_stages_regs(cpx<R> (&v)[16], cpx<R>* buf, int t,
                                                const cpx<R>* __restrict__ stw) {
  if constexpr (S < StageInfo<LOG2N, 0>::nstages) {
    fft_stage_regs<R, LOG2N, S, CT>(v, buf, t, stw);
    fft_stages_regs<R, LOG2N, S + 1, CT>(v, buf, t, stw);
  }
}

// CT = true: `stw` is the compact stage table (fft_stage_tw_elems_ct).
template <typename R, int LOG2N, bool CT = false>
__device__ __forceinline__ void block_fft_regs(cpx<R> (&v)[16], cpx<R>* buf, int t,
                                               const cpx<R>* __restrict__ stw, bool inv) {
  static_assert(LOG2N >= 4 && LOG2N <= 12, "FFT length 16..4096");
  if (inv) {
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m].y = -v[m].y;
  }
  fft_stages_regs<R, LOG2N, 0, CT>(v, buf, t, stw);
  if (inv) {
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m].y = -v[m].y;
  }
}

// ---------------------------------------------------------------------------
// Two independent length-N DFTs (same direction) by the same group of threads:
// a[m] and b[m] hold x_a[t + G m] and x_b[t + G m]; buffers buf_a and buf_b
// (fft_buf_elems(N) each).  The stages of both transforms are interleaved, so
// they share the barriers and every twiddle load, and each thread has two
// independent butterflies in flight per stage.
// ---------------------------------------------------------------------------
template <typename R, int LOG2N, int S, bool CT>
__device__ __forceinline__ void fft2_stage_regs(cpx<R> (&a)[16], cpx<R> (&b)[16], cpx<R>* buf_a,
                                                cpx<R>* buf_b, int t, const cpx<R>* __restrict__ stw) {
  using SI = StageInfo<LOG2N, S>;
  constexpr int N = 1 << LOG2N;
  constexpr int LR = SI::lr;
  constexpr int RAD = 1 << LR;
  constexpr int NB = N / RAD;
  constexpr int G = N / 16;
  constexpr int PER = 16 / RAD;
  constexpr int LOG2NS = SI::log2ns;
  constexpr int NS = 1 << LOG2NS;
  constexpr bool FIRST = (S == 0);
  constexpr bool LAST = (S == SI::nstages - 1);
  if constexpr (!FIRST) {
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < PER; ++bb) {
      const int j = t + bb * G;
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        a[bb * RAD + r] = buf_a[pad16(j + r * NB)];
        b[bb * RAD + r] = buf_b[pad16(j + r * NB)];
      }
    }
  }
#pragma unroll
  for (int bb = 0; bb < PER; ++bb) {
    const int j = t + bb * G;
    const int k = j & (NS - 1);
    if constexpr (CT && LOG2NS == 8) {  // compact table: w = hi[r][k >> 4] lo[r][k & 15]
      const cpx<R>* hi = stw + 15 * 16 + (k >> 4);
      const cpx<R>* lo = stw + 15 * 16 + (RAD - 1) * 16 + (k & 15);
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const cpx<R> w = cmul(hi[(r - 1) * 16], lo[(r - 1) * 16]);
        a[bb * RAD + r] = cmul(a[bb * RAD + r], w);
        b[bb * RAD + r] = cmul(b[bb * RAD + r], w);
      }
    } else if constexpr (LOG2NS > 0) {
      const cpx<R>* tws = stw + SI::tw_off + k;
#pragma unroll
      for (int r = 1; r < RAD; ++r) {
        const cpx<R> w = tws[(r - 1) * NS];
        a[bb * RAD + r] = cmul(a[bb * RAD + r], w);
        b[bb * RAD + r] = cmul(b[bb * RAD + r], w);
      }
    }
    cpx<R> ua[RAD], ub[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      ua[r] = a[bb * RAD + r];
      ub[r] = b[bb * RAD + r];
    }
    dft_rec<RAD, R>(ua);
    dft_rec<RAD, R>(ub);
#pragma unroll
    for (int r = 0; r < RAD; ++r) {
      a[bb * RAD + r] = ua[r];
      b[bb * RAD + r] = ub[r];
    }
  }
  if constexpr (!LAST) {
    __syncthreads();
#pragma unroll
    for (int bb = 0; bb < PER; ++bb) {
      const int j = t + bb * G;
      const int k = j & (NS - 1);
      const int base = (j - k) * RAD + k;
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        buf_a[pad16(base + r * NS)] = a[bb * RAD + r];
        buf_b[pad16(base + r * NS)] = b[bb * RAD + r];
      }
    }
  } else {
    cpx<R> oa[16], ob[16];
#pragma unroll
    for (int bb = 0; bb < PER; ++bb)
#pragma unroll
      for (int r = 0; r < RAD; ++r) {
        oa[bb + r * PER] = a[bb * RAD + r];
        ob[bb + r * PER] = b[bb * RAD + r];
      }
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      a[m] = oa[m];
      b[m] = ob[m];
    }
  }
}

template <typename R, int LOG2N, int S, bool CT>
__device__ __forceinline__ void fft2_stages_regs(cpx<R> (&a)[16], cpx<R> (&b)[16], cpx<R>* buf_a,
                                                 cpx<R>* buf_b, int t, const cpx<R>* __restrict__ stw) {
  if constexpr (S < StageInfo<LOG2N, 0>::nstages) {
    fft2_stage_regs<R, LOG2N, S, CT>(a, b, buf_a, buf_b, t, stw);
    fft2_stages_regs<R, LOG2N, S + 1, CT>(a, b, buf_a, buf_b, t, stw);
  }
}

// CT = true: `stw` is the compact stage table (fft_stage_tw_elems_ct).
template <typename R, int LOG2N, bool CT = false>
__device__ __forceinline__ void block_fft2_regs(cpx<R> (&a)[16], cpx<R> (&b)[16], cpx<R>* buf_a,
                                                cpx<R>* buf_b, int t, const cpx<R>* __restrict__ stw,
                                                bool inv) {
  static_assert(LOG2N >= 4 && LOG2N <= 12, "FFT length 16..4096");
  if (inv) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      a[m].y = -a[m].y;
      b[m].y = -b[m].y;
    }
  }
  fft2_stages_regs<R, LOG2N, 0, CT>(a, b, buf_a, buf_b, t, stw);
  if (inv) {
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      a[m].y = -a[m].y;
      b[m].y = -b[m].y;
    }
  }
}

// ---------------------------------------------------------------------------
// Programmatic dependent launch.  A kernel launched with programmatic stream
// serialization may start while its predecessor in the stream is still
// running: grid_dep_wait() blocks until the predecessor has completed and its
// writes are visible (a no-op for a normally launched kernel), so a kernel
// touches only its constant plan tables and shared memory before it.
// grid_dep_trigger() lets the successor launch once every CTA has called it
// or exited.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;\n" ::: "memory"); }
__device__ __forceinline__ void grid_dep_trigger() { asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory"); }

// Bulk copies from global to shared memory completing on an mbarrier (one
// arrival with the expected byte count per phase) under an L2 eviction-priority
// policy, and a wait on a phase bounded by wall time (%globaltimer): false
// after `ns` nanoseconds.
__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}
// L2 eviction priority "evict first" for data read once
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, unsigned bytes, unsigned long long* bar,
                                          unsigned long long pol) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;\n" ::
          "r"(smem_addr(sdst)),
      "l"(gsrc), "r"(bytes), "r"(smem_addr(bar)), "l"(pol)
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, unsigned long long ns) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  while (!mbar_try_wait(bar, parity))
    if (global_ns() - t0 > ns) return false;
  return true;
}

// The way out of a prefetching loop after a bounded wait expired in some
// thread of the CTA (every thread calls it, with its own wait's outcome): the
// status word records the timeout, thread 0 waits (bounded again) for the copy
// still in flight on phase `parity` of `bar`, so that the CTA does not exit
// while data lands in its shared memory, and the caller returns without
// writing results.  Returns true when the CTA must stop; it is a barrier for
// the whole CTA either way.
__device__ __forceinline__ bool cta_timed_out(bool ok, unsigned long long* bar, unsigned parity, int* status,
                                              unsigned long long drain_ns = 1000000000ull) {
  if (!__syncthreads_or(!ok)) return false;
  if (threadIdx.x == 0) {
    atomicExch(status, int(DSNU_ETIMEOUT));
    mbar_wait(bar, parity, drain_ns);
  }
  return true;
}

// Per-thread asynchronous 16-byte copies global -> shared (through L2 only);
// cp_async_wait_all() returns once this thread's copies have landed (a
// barrier then makes them visible to the block).
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(sdst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Cooperative copy of `n` table entries from global to shared memory.
template <typename T>
__device__ __forceinline__ void copy_to_smem(T* __restrict__ dst, const T* __restrict__ src, int n) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Conversions used at the FP64 boundary of the pipeline (identity for double).
// (round to nearest; FP32 -> FP64 is exact)
template <typename R>
__device__ __forceinline__ R from_f64(double d) {
  if constexpr (sizeof(R) == 4) return __double2float_rn(d);
  else return d;
}
template <typename R>
__device__ __forceinline__ double to_f64(R v) {
  return static_cast<double>(v);
}

// double(a) + double(b) rounded to FP64 (round to nearest even), bit for bit,
// for FP32 a and b, without FP64 instructions on the common path (this GPU
// runs FP64 at 1/63 of its FP32 rate):
//  * TwoSum (Knuth): s = fl32(a + b) and the exact remainder e, s + e = a + b,
//    |e| <= half an FP32 ulp of s;
//  * double(s) has 29 zero low fraction bits, so the FP64 sum is the FP64 bit
//    pattern of s plus e counted in FP64 ulps of s, rounded to the nearest
//    integer, ties to even (the pattern's last bit being 0); s + e stays in
//    the binade of s, except below a power of two s when e has the other
//    sign, where the count is in the lower binade's ulps (half as large) and
//    the pattern steps down into that binade;
//  * the count is e scaled by a power of two (exact) and converted with
//    round-to-nearest-even; it is at most 2^29 in magnitude.
// s with a biased exponent below 53 (|s| < 2^-74, where the scale would leave
// the float range), infinite or NaN takes the FP64 addition, in a branch that
// a warp enters only when one of its lanes needs it, through an out-of-line
// function: the compiler would otherwise turn the branch into predicated
// instructions, and a predicated-off FP64 instruction still occupies the
// narrow FP64 pipe.
static __device__ __noinline__ double add_f64_of_f32(float a, float b) {
  return static_cast<double>(a) + static_cast<double>(b);
}

__device__ __forceinline__ double add_f32_f64(float a, float b) {
  const float s = a + b;
  const float bv = s - a;
  const float av = s - bv;
  const float e = (a - av) + (b - bv);
  const unsigned u = __float_as_uint(s), v = __float_as_uint(e);
  const unsigned es = (u >> 23) & 0xFFu;
  const bool down = ((u & 0x7FFFFFu) == 0u) && ((u ^ v) & 0x80000000u) && (e != 0.0f);
  const float scale = __uint_as_float((306u - es + (down ? 1u : 0u)) << 23);  // 2^(52 - E) or 2^(53 - E)
  const int r = __float2int_rn(e * scale);
  const long long d = (u & 0x80000000u) ? -(long long)r : (long long)r;  // along the magnitude of s
  const unsigned hi = (u & 0x80000000u) | (((u & 0x7FFFFFFFu) >> 3) + 0x38000000u);
  double out = __longlong_as_double((long long)(((unsigned long long)hi << 32) | (u << 29)) + d);
  const bool slow = es < 53u || es == 255u;
  if (__any_sync(__activemask(), slow))
    if (slow) out = add_f64_of_f32(a, b);
  return out;
}

// FP64 -> FP32, rounded to nearest with ties to even, by integer instructions.
// For a double whose rounded value is a normal float, or that is a zero: the
// exponent is rebiased (1023 -> 127) and the top 23 fraction bits kept, which
// is the value truncated toward zero; adding 1 when the first dropped bit is
// set and either a later dropped bit or the kept last bit is set rounds it to
// nearest, ties to even (a carry out of the fraction steps the exponent, up to
// the infinity pattern past the largest float, as the rounding does).  `odd`
// is set for the other doubles (subnormal or too small results, infinities,
// NaNs, magnitudes from 2^128 up), which the caller converts with the hardware
// instruction, out of line (f32_of_f64_hw).
__device__ __forceinline__ float f32_of_f64_int(double d, bool& odd) {
  const unsigned hi = unsigned(__double2hiint(d)), lo = unsigned(__double2loint(d));
  const unsigned ha = hi & 0x7FFFFFFFu;
  unsigned f = __funnelshift_l(lo, ha - 0x38000000u, 3);  // exponent - 896, 20 + 3 fraction bits
  f += ((lo >> 28) & 1u) & ((((lo & 0x0FFFFFFFu) != 0u) ? 1u : 0u) | (f & 1u));
  const bool zero = (ha | lo) == 0u;
  odd = !zero && (ha - 0x38100000u > 0x47EFFFFFu - 0x38100000u);
  return __uint_as_float((zero ? 0u : f) | (hi & 0x80000000u));
}
static __device__ __noinline__ float f32_of_f64_hw(double d) { return __double2float_rn(d); }

// expm1 in the working precision (library function).
template <typename R>
__device__ __forceinline__ R expm1_r(R x) {
  if constexpr (sizeof(R) == 4) return expm1f(x);
  else return expm1(x);
}

// 1/b in FP64 by Newton-Raphson: the hardware's approximate reciprocal
// (rcp.approx.ftz.f64, about 2^-20 relative) refined twice by
// r <- r + r (1 - b r), which squares the relative error each step, so the
// result is within a couple of ulp of 1/b.  Five FP64 operations instead of
// an IEEE division; b must be a normal number (here b >= dk^2 > 0).
__device__ __forceinline__ double rcp_nr(double b) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(b));
  double e = fma(-b, r, 1.0);
  r = fma(r, e, r);
  e = fma(-b, r, 1.0);
  return fma(r, e, r);
}

// a / b: fast reciprocal path in FP32 (<= 2 ulp), a * rcp_nr(b) in FP64.
template <typename R>
__device__ __forceinline__ R fdiv(R a, R b) {
  if constexpr (sizeof(R) == 4) return __fdividef(a, b);
  else return a * rcp_nr(b);
}

}  // namespace dsnu
