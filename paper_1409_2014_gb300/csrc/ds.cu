// ds.cu -- split-step (time-splitting spectral) pieces of the DS time loop.
//
// Sec. 2.3 of the paper advances i u_t = -u_xx + alpha u_yy - 2 beta |u|^2 u
// - 4 beta Phi u (eq. DSII_exact) by composing
//   * the linear flow (eqs. 1st_tssp, 1st_tssp_more), exact in Fourier space on
//     the periodic N x N grid:  v_hat <- exp(-i tau (k_x^2 - alpha k_y^2)) v_hat;
//   * the nonlinear flow (eqs. 2nd_tssp, 2nd_tssp_more), pointwise with the
//     density and Phi frozen:  w <- w exp(i tau (2 beta |w|^2 + 4 beta Phi)).
// This file provides both flows on the GPU plus the pieces of their
// vector-Jacobian products; Phi itself comes from the potential solver.
// Complex fields are interleaved (re, im) [ny][nx]: complex64 for a DSNU_MIXED
// plan, complex128 for DSNU_FP64.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace dsnu {

// Geometry of the unpadded 2D transform (rows: length nx; columns: length ny).
template <typename R, int LOG2N>
struct GeoC2C {
  static constexpr int N = 1 << LOG2N;
  static constexpr int G = N / 16;
  static constexpr int FB = fft_buf_elems(N);
  static constexpr int PER = (G >= 256) ? 1 : 256 / G;  // rows or columns per CTA
  static constexpr int T = PER * G;
  static constexpr int STW = fft_stage_tw_elems(LOG2N) > 0 ? fft_stage_tw_elems(LOG2N) : 1;
  static constexpr int STWP = (STW + 1) & ~1;
  static constexpr size_t smem = size_t(STWP + PER * FB) * sizeof(cpx<R>);
};

// In-place length-nx DFT of every row (inv: unnormalised inverse).
template <typename R, int LOG2N>
__global__ void __launch_bounds__(GeoC2C<R, LOG2N>::T)
k_c2c_rows(cpx<R>* __restrict__ u, int ny, const cpx<R>* __restrict__ stw_g, int inv) {
  using GG = GeoC2C<R, LOG2N>;
  constexpr int N = GG::N, G = GG::G, PER = GG::PER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* sm = stw + GG::STWP;
  copy_to_smem(stw, stw_g, GG::STW);
  const int tid = threadIdx.x;
  const int rr = tid / G, t = tid - rr * G;
  cpx<R>* buf = sm + rr * GG::FB;
  const int items = (ny + PER - 1) / PER;
#pragma unroll 1
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int row = item * PER + rr;
    const bool valid = row < ny;
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m) v[m] = valid ? u[size_t(row) * N + t + G * m] : mk<R>(R(0), R(0));
    block_fft_regs<R, LOG2N>(v, buf, t, stw, inv != 0);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 16; ++m) u[size_t(row) * N + t + G * m] = v[m];
    }
  }
}

// Per column: DFT along y, multiply by px[col] py[k] * scale (conjugated when
// adj), inverse DFT along y; in place.  px, py: the separable linear-flow
// phases e^{-i tau k_x^2} and e^{+i tau alpha k_y^2} in FFT order.
template <typename R, int LOG2N>
__global__ void __launch_bounds__(GeoC2C<R, LOG2N>::T)
k_c2c_cols_phase(cpx<R>* __restrict__ u, int nx, const cpx<R>* __restrict__ stw_g,
                 const cpx<R>* __restrict__ px, const cpx<R>* __restrict__ py, R scale, int adj) {
  using GG = GeoC2C<R, LOG2N>;
  constexpr int G = GG::G, PER = GG::PER;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cpx<R>* stw = reinterpret_cast<cpx<R>*>(smem_raw);
  cpx<R>* sm = stw + GG::STWP;
  copy_to_smem(stw, stw_g, GG::STW);
  const int tid = threadIdx.x;
  const int cl = tid / G, t = tid - cl * G;
  cpx<R>* buf = sm + cl * GG::FB;
  const int items = (nx + PER - 1) / PER;
#pragma unroll 1
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int col = item * PER + cl;
    const bool valid = col < nx;
    cpx<R> v[16];
#pragma unroll
    for (int m = 0; m < 16; ++m)
      v[m] = valid ? u[size_t(t + G * m) * nx + col] : mk<R>(R(0), R(0));
    block_fft_regs<R, LOG2N>(v, buf, t, stw, false);
    cpx<R> pxc = valid ? px[col] : mk<R>(R(0), R(0));
    if (adj) pxc.y = -pxc.y;
#pragma unroll
    for (int m = 0; m < 16; ++m) {
      cpx<R> p = py[t + G * m];
      if (adj) p.y = -p.y;
      v[m] = cmul(v[m], cmul(pxc, p)) * scale;
    }
    block_fft_regs<R, LOG2N>(v, buf, t, stw, true);
    if (valid) {
#pragma unroll
      for (int m = 0; m < 16; ++m) u[size_t(t + G * m) * nx + col] = v[m];
    }
  }
}

// rho = |u|^2 (FP64 out).
template <typename R>
__global__ void k_abs2(const cpx<R>* __restrict__ u, double* __restrict__ rho, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const cpx<R> a = u[i];
    rho[i] = to_f64<R>(a.x * a.x + a.y * a.y);
  }
}

// Vector-Jacobian product of rho = |u|^2 for a real loss (gradients in the
// d/dRe + i d/dIm convention): grad_u = 2 g_rho u, g_rho FP64.
template <typename R>
__global__ void k_abs2_vjp(const cpx<R>* __restrict__ u, const double* __restrict__ g_rho,
                           cpx<R>* __restrict__ grad, size_t n) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const cpx<R> a = u[i];
    const R g2 = R(2) * from_f64<R>(g_rho[i]);
    grad[i] = mk<R>(g2 * a.x, g2 * a.y);
  }
}

template <typename R>
__device__ __forceinline__ void sincos_r(R a, R* s, R* c) {
  if constexpr (sizeof(R) == 4) sincosf(a, s, c);
  else sincos(a, s, c);
}

// theta = tau (2 beta |u|^2 + 4 beta Phi) at a point.
template <typename R>
__device__ __forceinline__ R nl_angle(cpx<R> a, double phi, R tau, R beta) {
  return tau * (R(2) * beta * (a.x * a.x + a.y * a.y) + R(4) * beta * from_f64<R>(phi));
}

// u <- u e^{i theta}.
template <typename R>
__global__ void k_nonlinear(cpx<R>* __restrict__ u, const double* __restrict__ phi, size_t n, R tau,
                            R beta) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const cpx<R> a = u[i];
    R s, c;
    sincos_r(nl_angle(a, phi[i], tau, beta), &s, &c);
    u[i] = cmul(a, mk<R>(c, s));
  }
}

// Backward of u' = u e^{i theta(|u|^2)} for a real loss, gradients in the
// (d/dRe + i d/dIm) convention:  given g' at u', returns
//   part = g' e^{-i theta}        (the direct term)
//   sfld = Im(g' conj(u'))        (so that dL = <tau (2 beta s + 4 beta A^T s), d rho> + ...)
template <typename R>
__global__ void k_nonlinear_vjp(const cpx<R>* __restrict__ u, const double* __restrict__ phi,
                                const cpx<R>* __restrict__ g, size_t n, R tau, R beta,
                                double* __restrict__ sfld, cpx<R>* __restrict__ part) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const cpx<R> a = u[i];
    R s, c;
    sincos_r(nl_angle(a, phi[i], tau, beta), &s, &c);
    const cpx<R> e = mk<R>(c, s);
    const cpx<R> up = cmul(a, e);
    const cpx<R> gi = g[i];
    part[i] = cmulc(gi, e);                              // g' e^{-i theta}
    sfld[i] = to_f64<R>(gi.y * up.x - gi.x * up.y);      // Im(g' conj u')
  }
}

// grad_u = part + 2 tau (2 beta s + 4 beta (A^T s)) u   (in place on part)
template <typename R>
__global__ void k_nonlinear_vjp_finish(const cpx<R>* __restrict__ u, const double* __restrict__ sfld,
                                       const double* __restrict__ ats, size_t n, R tau, R beta,
                                       cpx<R>* __restrict__ part) {
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n; i += size_t(gridDim.x) * blockDim.x) {
    const R grho = tau * (R(2) * beta * from_f64<R>(sfld[i]) + R(4) * beta * from_f64<R>(ats[i]));
    const cpx<R> a = u[i];
    const cpx<R> p = part[i];
    part[i] = mk<R>(p.x + R(2) * grho * a.x, p.y + R(2) * grho * a.y);
  }
}

// Linear-flow phase tables in FFT order: px[q] = e^{-i tau k_x^2} and
// py[q] = e^{+i tau alpha k_y^2}, k = qs dk with qs the signed index.  The
// angles and their sine/cosine are formed in FP64 and rounded to the plan's
// precision; launched on the caller's stream, so a change of step size needs
// no host round trip.
template <typename R>
__global__ void k_phase_tables(cpx<R>* __restrict__ px, cpx<R>* __restrict__ py, int nx, int ny, double dkx,
                               double dky, double tau, double alpha) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nx) {
    const double k = double(i < nx / 2 ? i : i - nx) * dkx;
    double s, c;
    sincos(-tau * k * k, &s, &c);
    px[i] = mk<R>(R(c), R(s));
  }
  if (i < ny) {
    const double k = double(i < ny / 2 ? i : i - ny) * dky;
    double s, c;
    sincos(tau * alpha * k * k, &s, &c);
    py[i] = mk<R>(R(c), R(s));
  }
}

}  // namespace dsnu

using namespace dsnu;

struct dsnu_ds_plan_s {
  dsnu_ds_params prm;
  int log2nx, log2ny;
  void* block;       // stage twiddles of both axes + phase tables
  void* stw_x;
  void* stw_y;
  void* px;          // nx complex
  void* py;          // ny complex
  double tau, alpha; // phases currently loaded
  bool has_phase;
  int grid_rows, grid_cols;
};

namespace {

dsnu_status ds_fail(dsnu_status s, const std::string& m) {
  dsnu::set_last_error(m);
  return s;
}

void stage_twiddles(int log2n, std::vector<double>& out) {
  out.clear();
  const int full = log2n / 4;
  const int nst = (log2n + 3) / 4;
  for (int s = 1; s < nst; ++s) {
    const int lr = (s < full) ? 4 : (log2n - 4 * full);
    const int rad = 1 << lr, ns = 1 << (4 * s);
    for (int r = 1; r < rad; ++r)
      for (int k = 0; k < ns; ++k) {
        const double a = -2.0 * M_PI * double(r) * double(k) / double(ns * rad);
        out.push_back(std::cos(a));
        out.push_back(std::sin(a));
      }
  }
  if (out.empty()) out.assign(2, 0.0);
}

template <typename R>
void upload(void* dst, const std::vector<double>& v, cudaStream_t st, cudaError_t* e) {
  std::vector<R> tmp(v.begin(), v.end());
  if (*e == cudaSuccess) *e = cudaMemcpyAsync(dst, tmp.data(), tmp.size() * sizeof(R), cudaMemcpyHostToDevice, st);
  if (*e == cudaSuccess) *e = cudaStreamSynchronize(st);
}

template <typename R, typename K>
int grid_for(K kernel, int threads, size_t smem, int items) {
  int dev = 0, sms = 1, per = 1;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, threads, smem);
  if (per < 1) per = 1;
  const int cap = sms * per;
  return items < cap ? (items > 0 ? items : 1) : cap;
}

#define DSNU_C2C_CASES(CALL) \
  case 4: CALL(4); break;    \
  case 5: CALL(5); break;    \
  case 6: CALL(6); break;    \
  case 7: CALL(7); break;    \
  case 8: CALL(8); break;    \
  case 9: CALL(9); break;    \
  case 10: CALL(10); break;  \
  case 11: CALL(11); break;  \
  case 12: CALL(12); break;

template <typename R>
cudaError_t prepare(dsnu_ds_plan_s* P) {
  cudaError_t e = cudaSuccess;
  const cudaFuncAttribute A = cudaFuncAttributeMaxDynamicSharedMemorySize;
#define DSNU_PR(L2)                                                                                 \
  e = cudaFuncSetAttribute(k_c2c_rows<R, L2>, A, int(GeoC2C<R, L2>::smem));                        \
  if (e == cudaSuccess)                                                                             \
    P->grid_rows = grid_for<R>(k_c2c_rows<R, L2>, GeoC2C<R, L2>::T, GeoC2C<R, L2>::smem,            \
                               (P->prm.ny + GeoC2C<R, L2>::PER - 1) / GeoC2C<R, L2>::PER)
#define DSNU_PC(L2)                                                                                 \
  e = cudaFuncSetAttribute(k_c2c_cols_phase<R, L2>, A, int(GeoC2C<R, L2>::smem));                  \
  if (e == cudaSuccess)                                                                             \
    P->grid_cols = grid_for<R>(k_c2c_cols_phase<R, L2>, GeoC2C<R, L2>::T, GeoC2C<R, L2>::smem,      \
                               (P->prm.nx + GeoC2C<R, L2>::PER - 1) / GeoC2C<R, L2>::PER)
  switch (P->log2nx) {
    DSNU_C2C_CASES(DSNU_PR)
    default: return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess) return e;
  switch (P->log2ny) {
    DSNU_C2C_CASES(DSNU_PC)
    default: return cudaErrorInvalidValue;
  }
#undef DSNU_PR
#undef DSNU_PC
  return e;
}

template <typename R>
dsnu_status linear(dsnu_ds_plan_s* P, void* uv, int adjoint, cudaStream_t st) {
  cpx<R>* u = static_cast<cpx<R>*>(uv);
  const R scale = R(1.0 / (double(P->prm.nx) * double(P->prm.ny)));
  const cpx<R>* sx = static_cast<const cpx<R>*>(P->stw_x);
  const cpx<R>* sy = static_cast<const cpx<R>*>(P->stw_y);
  const cpx<R>* px = static_cast<const cpx<R>*>(P->px);
  const cpx<R>* py = static_cast<const cpx<R>*>(P->py);
#define DSNU_ROWS(L2, INV)                                                                   \
  k_c2c_rows<R, L2><<<P->grid_rows, GeoC2C<R, L2>::T, GeoC2C<R, L2>::smem, st>>>(u, P->prm.ny, sx, INV)
#define DSNU_RF(L2) DSNU_ROWS(L2, 0)
#define DSNU_RI(L2) DSNU_ROWS(L2, 1)
#define DSNU_CP(L2)                                                                          \
  k_c2c_cols_phase<R, L2><<<P->grid_cols, GeoC2C<R, L2>::T, GeoC2C<R, L2>::smem, st>>>(     \
      u, P->prm.nx, sy, px, py, scale, adjoint)
  switch (P->log2nx) {
    DSNU_C2C_CASES(DSNU_RF)
    default: return DSNU_EUNSUPPORTED;
  }
  switch (P->log2ny) {
    DSNU_C2C_CASES(DSNU_CP)
    default: return DSNU_EUNSUPPORTED;
  }
  switch (P->log2nx) {
    DSNU_C2C_CASES(DSNU_RI)
    default: return DSNU_EUNSUPPORTED;
  }
#undef DSNU_ROWS
#undef DSNU_RF
#undef DSNU_RI
#undef DSNU_CP
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DSNU_OK : ds_fail(DSNU_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
}

int grid_1d(size_t n) {
  const size_t b = (n + 255) / 256;
  return int(b < 4096 ? b : 4096);
}

dsnu_status check_launch() {
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DSNU_OK : ds_fail(DSNU_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
}

int ilog2i(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

}  // namespace

extern "C" {

dsnu_status dsnu_ds_plan_create(const dsnu_ds_params* params, void* stream, dsnu_ds_plan* out) {
  if (!params || !out) return ds_fail(DSNU_EINVAL, "NULL params or out");
  const dsnu_ds_params p = *params;
  auto pow2 = [](int v) { return v >= 16 && v <= 4096 && (v & (v - 1)) == 0; };
  if (!pow2(p.nx) || !pow2(p.ny)) return ds_fail(DSNU_EINVAL, "nx, ny must be powers of two in [16, 4096]");
  if (!(p.lx > 0.0) || !(p.ly > 0.0) || !std::isfinite(p.lx) || !std::isfinite(p.ly))
    return ds_fail(DSNU_EINVAL, "lx, ly must be positive and finite");
  if (p.precision != DSNU_FP64 && p.precision != DSNU_MIXED) return ds_fail(DSNU_EINVAL, "unknown precision");
  dsnu_ds_plan_s* P = new (std::nothrow) dsnu_ds_plan_s();
  if (!P) return ds_fail(DSNU_ENOMEM, "host allocation failed");
  P->prm = p;
  P->log2nx = ilog2i(p.nx);
  P->log2ny = ilog2i(p.ny);
  const size_t rsz = p.precision == DSNU_MIXED ? 4 : 8;
  std::vector<double> sx, sy;
  stage_twiddles(P->log2nx, sx);
  stage_twiddles(P->log2ny, sy);
  auto al = [](size_t v) { return (v + 255) & ~size_t(255); };
  const size_t o_sx = 0, o_sy = al(sx.size() * rsz), o_px = o_sy + al(sy.size() * rsz);
  const size_t o_py = o_px + al(2 * size_t(p.nx) * rsz), total = o_py + al(2 * size_t(p.ny) * rsz);
  cudaError_t e = cudaMalloc(&P->block, total);
  if (e != cudaSuccess) {
    delete P;
    return ds_fail(DSNU_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  char* d = static_cast<char*>(P->block);
  P->stw_x = d + o_sx;
  P->stw_y = d + o_sy;
  P->px = d + o_px;
  P->py = d + o_py;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (p.precision == DSNU_MIXED) {
    upload<float>(P->stw_x, sx, st, &e);
    upload<float>(P->stw_y, sy, st, &e);
    if (e == cudaSuccess) e = prepare<float>(P);
  } else {
    upload<double>(P->stw_x, sx, st, &e);
    upload<double>(P->stw_y, sy, st, &e);
    if (e == cudaSuccess) e = prepare<double>(P);
  }
  if (e != cudaSuccess) {
    cudaFree(P->block);
    delete P;
    return ds_fail(DSNU_ECUDA, std::string("DS plan set-up: ") + cudaGetErrorString(e));
  }
  P->has_phase = false;
  *out = P;
  return DSNU_OK;
}

dsnu_status dsnu_ds_set_linear_step(dsnu_ds_plan plan, double tau, double alpha, void* stream) {
  if (!plan) return ds_fail(DSNU_EINVAL, "NULL plan");
  if (!std::isfinite(tau) || !std::isfinite(alpha)) return ds_fail(DSNU_EINVAL, "tau, alpha must be finite");
  if (plan->has_phase && plan->tau == tau && plan->alpha == alpha) return DSNU_OK;
  const dsnu_ds_params& p = plan->prm;
  const double dkx = M_PI / p.lx, dky = M_PI / p.ly;  // 2 pi / (n h), h = 2 l / n
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int n = p.nx > p.ny ? p.nx : p.ny;
  if (p.precision == DSNU_MIXED)
    k_phase_tables<float><<<(n + 255) / 256, 256, 0, st>>>(static_cast<cpx<float>*>(plan->px),
                                                           static_cast<cpx<float>*>(plan->py), p.nx, p.ny,
                                                           dkx, dky, tau, alpha);
  else
    k_phase_tables<double><<<(n + 255) / 256, 256, 0, st>>>(static_cast<cpx<double>*>(plan->px),
                                                            static_cast<cpx<double>*>(plan->py), p.nx, p.ny,
                                                            dkx, dky, tau, alpha);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ds_fail(DSNU_ECUDA, std::string("phase tables: ") + cudaGetErrorString(e));
  plan->tau = tau;
  plan->alpha = alpha;
  plan->has_phase = true;
  return DSNU_OK;
}

dsnu_status dsnu_ds_linear(dsnu_ds_plan plan, void* u_dev, int32_t adjoint, void* stream) {
  if (!plan || !u_dev) return ds_fail(DSNU_EINVAL, "NULL plan or field");
  if (!plan->has_phase) return ds_fail(DSNU_EINVAL, "no linear step set (dsnu_ds_set_linear_step)");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return plan->prm.precision == DSNU_MIXED ? linear<float>(plan, u_dev, adjoint, st)
                                           : linear<double>(plan, u_dev, adjoint, st);
}

dsnu_status dsnu_ds_abs2(dsnu_ds_plan plan, const void* u_dev, double* rho_dev, void* stream) {
  if (!plan || !u_dev || !rho_dev) return ds_fail(DSNU_EINVAL, "NULL argument");
  const size_t n = size_t(plan->prm.nx) * plan->prm.ny;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->prm.precision == DSNU_MIXED)
    k_abs2<float><<<grid_1d(n), 256, 0, st>>>(static_cast<const cpx<float>*>(u_dev), rho_dev, n);
  else
    k_abs2<double><<<grid_1d(n), 256, 0, st>>>(static_cast<const cpx<double>*>(u_dev), rho_dev, n);
  return check_launch();
}

dsnu_status dsnu_ds_abs2_vjp(dsnu_ds_plan plan, const void* u_dev, const double* g_rho_dev, void* grad_dev,
                             void* stream) {
  if (!plan || !u_dev || !g_rho_dev || !grad_dev) return ds_fail(DSNU_EINVAL, "NULL argument");
  const size_t n = size_t(plan->prm.nx) * plan->prm.ny;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->prm.precision == DSNU_MIXED)
    k_abs2_vjp<float><<<grid_1d(n), 256, 0, st>>>(static_cast<const cpx<float>*>(u_dev), g_rho_dev,
                                                 static_cast<cpx<float>*>(grad_dev), n);
  else
    k_abs2_vjp<double><<<grid_1d(n), 256, 0, st>>>(static_cast<const cpx<double>*>(u_dev), g_rho_dev,
                                                  static_cast<cpx<double>*>(grad_dev), n);
  return check_launch();
}

dsnu_status dsnu_ds_nonlinear(dsnu_ds_plan plan, void* u_dev, const double* phi_dev, double tau, double beta,
                              void* stream) {
  if (!plan || !u_dev || !phi_dev) return ds_fail(DSNU_EINVAL, "NULL argument");
  const size_t n = size_t(plan->prm.nx) * plan->prm.ny;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->prm.precision == DSNU_MIXED)
    k_nonlinear<float><<<grid_1d(n), 256, 0, st>>>(static_cast<cpx<float>*>(u_dev), phi_dev, n, float(tau),
                                                  float(beta));
  else
    k_nonlinear<double><<<grid_1d(n), 256, 0, st>>>(static_cast<cpx<double>*>(u_dev), phi_dev, n, tau, beta);
  return check_launch();
}

dsnu_status dsnu_ds_nonlinear_vjp(dsnu_ds_plan plan, const void* u_dev, const double* phi_dev, const void* g_dev,
                                  double tau, double beta, double* s_dev, void* part_dev, void* stream) {
  if (!plan || !u_dev || !phi_dev || !g_dev || !s_dev || !part_dev) return ds_fail(DSNU_EINVAL, "NULL argument");
  const size_t n = size_t(plan->prm.nx) * plan->prm.ny;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->prm.precision == DSNU_MIXED)
    k_nonlinear_vjp<float><<<grid_1d(n), 256, 0, st>>>(
        static_cast<const cpx<float>*>(u_dev), phi_dev, static_cast<const cpx<float>*>(g_dev), n, float(tau),
        float(beta), s_dev, static_cast<cpx<float>*>(part_dev));
  else
    k_nonlinear_vjp<double><<<grid_1d(n), 256, 0, st>>>(
        static_cast<const cpx<double>*>(u_dev), phi_dev, static_cast<const cpx<double>*>(g_dev), n, tau, beta,
        s_dev, static_cast<cpx<double>*>(part_dev));
  return check_launch();
}

dsnu_status dsnu_ds_nonlinear_vjp_finish(dsnu_ds_plan plan, const void* u_dev, const double* s_dev,
                                         const double* ats_dev, double tau, double beta, void* grad_dev,
                                         void* stream) {
  if (!plan || !u_dev || !s_dev || !ats_dev || !grad_dev) return ds_fail(DSNU_EINVAL, "NULL argument");
  const size_t n = size_t(plan->prm.nx) * plan->prm.ny;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (plan->prm.precision == DSNU_MIXED)
    k_nonlinear_vjp_finish<float><<<grid_1d(n), 256, 0, st>>>(
        static_cast<const cpx<float>*>(u_dev), s_dev, ats_dev, n, float(tau), float(beta),
        static_cast<cpx<float>*>(grad_dev));
  else
    k_nonlinear_vjp_finish<double><<<grid_1d(n), 256, 0, st>>>(
        static_cast<const cpx<double>*>(u_dev), s_dev, ats_dev, n, tau, beta, static_cast<cpx<double>*>(grad_dev));
  return check_launch();
}

dsnu_status dsnu_ds_plan_destroy(dsnu_ds_plan plan) {
  if (!plan) return DSNU_OK;
  const cudaError_t e = cudaFree(plan->block);
  delete plan;
  return e == cudaSuccess ? DSNU_OK : ds_fail(DSNU_ECUDA, std::string("cudaFree: ") + cudaGetErrorString(e));
}

}  // extern "C"
