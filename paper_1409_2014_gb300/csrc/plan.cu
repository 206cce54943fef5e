// plan.cu -- host side: parameter checks, FP64 plan tables, the C ABI.
//
// Plan tables (Sec. 2.1 of the paper, all generated in FP64 here):
//   * radial Gauss-Legendre nodes/weights on [0, P] (Newton iteration on the
//     Legendre three-term recurrence) and the uniform angular rule
//     theta_j = 2 pi j / N_theta  -> polar nodes k_ij = r_i (cos, sin) theta_j;
//   * weights D_ij = -(2 pi)^-2 r_i w_i (2 pi/N_theta) cos^2(theta_j) p(r_i)
//     (eq. I2PolarDisc with the Jacobian r and the angular-frequency
//     normalisation written in);
//   * the exponential-of-semicircle (ES) kernel phi(z) = exp(beta (sqrt(1 -
//     (2z/w)^2) - 1)) on |z| <= w/2 fine-grid cells, beta = 2.30 w (Barnett,
//     Magland, af Klinteberg 2019, upsampling 2), its per-node separable
//     weights and its Fourier transform phi_hat (deconvolution);
//   * twiddles e^{-2 pi i m/N} and e^{-2 pi i n/M}, and the axis tables of the
//     high-frequency multiplier (1 - p) (-k_x^2/|k|^2);
//   * the spreading tiles' node lists (nodes are fixed per plan).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "internal.h"
#include "kernels.cuh"

namespace dsnu {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

static dsnu_status fail(dsnu_status st, const std::string& msg) {
  set_last_error(msg);
  return st;
}

static bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
static int ilog2(int v) {
  int l = 0;
  while ((1 << l) < v) ++l;
  return l;
}

// Gauss-Legendre nodes (ascending) and weights on [-1, 1].
static void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = (n == 1) ? 1.0 : n * (z * p1 - p0) / (z * z - 1.0);
    }
    x[n - 1 - i] = z;
    w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// P_n and P_{n-1} of the Jacobi polynomials P^{(a,b)} with a = 0, b = 1 at t,
// from the three-term recurrence
//   2(k+1)(k+a+b+1)(2k+a+b) P_{k+1}
//     = (2k+a+b+1)[(2k+a+b+2)(2k+a+b) t + a^2 - b^2] P_k - 2(k+a)(k+b)(2k+a+b+2) P_{k-1},
// P_0 = 1, P_1 = (3t - 1)/2.
static void jacobi01(int n, double t, double* pn, double* pn1) {
  double p0 = 1.0, p1 = 0.5 * (3.0 * t - 1.0);
  if (n == 0) {
    *pn = 1.0;
    *pn1 = 0.0;
    return;
  }
  for (int k = 1; k < n; ++k) {
    const double c1 = 2.0 * (k + 1) * (k + 2) * (2.0 * k + 1);
    const double c2 = -(2.0 * k + 2);
    const double c3 = (2.0 * k + 1) * (2.0 * k + 2) * (2.0 * k + 3);
    const double c4 = 2.0 * k * (k + 1) * (2.0 * k + 3);
    const double p2 = ((c2 + c3 * t) * p1 - c4 * p0) / c1;
    p0 = p1;
    p1 = p2;
  }
  *pn = p1;
  *pn1 = p0;
}

// Gauss-Jacobi nodes (ascending) and weights on [-1, 1] for the weight
// function (1 + t): Newton on P_n^{(0,1)} with the roots already found divided
// out, started from cos(pi (i - 1/4)/(n + 1)); the derivative from
//   (2n+1)(1 - t^2) P_n' = n[-1 - (2n+1) t] P_n + 2n(n+1) P_{n-1},
// the weights 4 / ((1 - t^2) P_n'(t)^2).
static void gauss_jacobi01(int n, std::vector<double>& x, std::vector<double>& w) {
  std::vector<double> roots;
  auto deriv = [n](double t, double pn, double pn1) {
    return (n * (-1.0 - (2.0 * n + 1) * t) * pn + 2.0 * n * (n + 1) * pn1) / ((2.0 * n + 1) * (1.0 - t * t));
  };
  for (int i = 1; i <= n; ++i) {
    double z = std::cos(M_PI * (i - 0.25) / (n + 1.0));
    for (int it = 0; it < 200; ++it) {
      double pn, pn1;
      jacobi01(n, z, &pn, &pn1);
      double defl = 0.0;
      for (double r : roots) defl += 1.0 / (z - r);
      const double dz = pn / (deriv(z, pn, pn1) - pn * defl);
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    roots.push_back(z);
  }
  std::sort(roots.begin(), roots.end());
  x = roots;
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double pn, pn1;
    jacobi01(n, x[i], &pn, &pn1);
    const double d = deriv(x[i], pn, pn1);
    w[i] = 4.0 / ((1.0 - x[i] * x[i]) * d * d);
  }
}

// Radial nodes r_i in (0, P) (ascending) and weights W_i with
// sum_i W_i f(r_i) ~ int_0^P f(r) r dr (the polar Jacobian r, Sec. 2.1):
// Gauss-Legendre mapped to [0, P] with r multiplied into the weight, or the
// Gauss-Jacobi(0, 1) rule whose weight function is that Jacobian
// (r = P (1 + t)/2, r dr = (P/2)^2 (1 + t) dt).
static void radial_nodes(int n, int rule, double P, std::vector<double>& r, std::vector<double>& w) {
  std::vector<double> t, v;
  if (rule == DSNU_RADIAL_JACOBI) {
    gauss_jacobi01(n, t, v);
    for (double& x : v) x *= 0.25 * P * P;
  } else {
    gauss_legendre(n, t, v);
    for (int i = 0; i < n; ++i) v[i] *= 0.5 * P * (0.5 * P * (t[i] + 1.0));
  }
  r.resize(n);
  for (int i = 0; i < n; ++i) r[i] = 0.5 * P * (t[i] + 1.0);
  w = v;
}

static double es_kernel(double z, int w, double beta) {
  const double t = 2.0 * z / w;
  const double u = 1.0 - t * t;
  if (u < 0.0) return 0.0;
  return std::exp(beta * (std::sqrt(u) - 1.0));
}

// phi_hat(xi) = int_{-w/2}^{w/2} phi(z) e^{-i xi z} dz, by Gauss-Legendre in
// t with z = (w/2) sin t (smooth integrand on [0, pi/2]).
struct EsFourier {
  std::vector<double> t, v;
  int w;
  double beta;
  EsFourier(int w_, double beta_) : w(w_), beta(beta_) {
    std::vector<double> x, ww;
    gauss_legendre(200, x, ww);
    t.resize(x.size());
    v.resize(x.size());
    for (size_t i = 0; i < x.size(); ++i) {
      t[i] = (x[i] + 1.0) * M_PI / 4.0;
      v[i] = ww[i] * M_PI / 4.0;
    }
  }
  double operator()(double xi) const {
    const double hw = 0.5 * w;
    double s = 0.0;
    for (size_t i = 0; i < t.size(); ++i) {
      const double z = hw * std::sin(t[i]);
      s += v[i] * std::exp(beta * (std::cos(t[i]) - 1.0)) * hw * std::cos(t[i]) * std::cos(xi * z);
    }
    return 2.0 * s;
  }
};

template <typename R>
struct HostTables {
  // complex tables interleaved (re, im)
  std::vector<R> stw_x, stwc_x, twm_lo_x, twm_hi_x, decon_x, stw_y, twm_lo_y, twm_hi_y, decon_y;
  std::vector<R> m_wx2, m_gx, m_gy, m_kx;
  std::vector<int2> node_q0;
  std::vector<int> itile_ptr, itile_nodes;
  std::vector<int2> itile_org;
  std::vector<R> node_w;
  std::vector<double> node_D;
};

// Spreading tables for one tile configuration (see k_spread).
template <typename R>
struct HostSpread {
  std::vector<int> tile_ptr, ent_node, tile_items, item_tile;
  std::vector<int2> ent_q0, item_range;
  std::vector<R> ent_w;
  int tiles_x = 0, tiles_y = 0, n_tiles = 0, n_items = 0, max_tile = 0;
};

// Bin the nodes into cfg.tile x cfg.tile tiles of band cells over q_x in
// [0, Q], q_y in [-Q, Q]; per tile, the entries of every node whose stencil
// meets it, cut into work items of at most cfg.chunk entries.
template <typename R>
static void bin_spread(const std::vector<int2>& q0, const std::vector<R>& nw, int w, int Q, const SpreadCfg& cfg,
                       HostSpread<R>& H) {
  const int TS = cfg.tile, nn = int(q0.size());
  H.tiles_x = (Q + 1 + TS - 1) / TS;
  H.tiles_y = (2 * Q + 1 + TS - 1) / TS;
  H.n_tiles = H.tiles_x * H.tiles_y;
  std::vector<std::vector<int>> lists(H.n_tiles);
  for (int j = 0; j < nn; ++j) {
    const int xlo = std::max(q0[j].x, 0), xhi = std::min(q0[j].x + w - 1, Q);
    if (xhi < xlo) continue;
    const int ylo = q0[j].y + Q, yhi = q0[j].y + w - 1 + Q;
    for (int ty = ylo / TS; ty <= yhi / TS; ++ty)
      for (int tx = xlo / TS; tx <= xhi / TS; ++tx) lists[ty * H.tiles_x + tx].push_back(j);
  }
  H.tile_ptr.assign(H.n_tiles + 1, 0);
  H.max_tile = 0;
  for (int i = 0; i < H.n_tiles; ++i) {
    H.tile_ptr[i + 1] = H.tile_ptr[i] + int(lists[i].size());
    H.max_tile = std::max(H.max_tile, int(lists[i].size()));
  }
  for (auto& l : lists)
    for (int j : l) {
      H.ent_node.push_back(j);
      H.ent_q0.push_back(q0[j]);
      H.ent_w.insert(H.ent_w.end(), nw.begin() + size_t(j) * 2 * w, nw.begin() + size_t(j + 1) * 2 * w);
    }
  if (H.ent_node.empty()) {
    H.ent_node.push_back(0);
    H.ent_q0.push_back(make_int2(0, 0));
    H.ent_w.resize(2 * w, R(0));
  }
  H.tile_items.assign(H.n_tiles + 1, 0);
  for (int i = 0; i < H.n_tiles; ++i) {
    for (int b = H.tile_ptr[i]; b < H.tile_ptr[i + 1]; b += cfg.chunk) {
      H.item_range.push_back(make_int2(b, std::min(b + cfg.chunk, H.tile_ptr[i + 1])));
      H.item_tile.push_back(i);
    }
    H.tile_items[i + 1] = int(H.item_range.size());
  }
  H.n_items = int(H.item_range.size());
  if (H.item_range.empty()) {
    H.item_range.push_back(make_int2(0, 0));
    H.item_tile.push_back(0);
  }
}

static void twiddles(int n, int m, std::vector<double>& out) {
  out.resize(2 * n);
  for (int i = 0; i < n; ++i) {
    const double a = -2.0 * M_PI * double(i) / double(m);
    out[2 * i] = std::cos(a);
    out[2 * i + 1] = std::sin(a);
  }
}

// FFT stage twiddles of a length-2^log2n transform in the order the device
// FFT reads them: stage s >= 1 (radix RAD, NS = product of the earlier
// radices), r = 1..RAD-1, k = 0..NS-1: e^{-2 pi i r k / (NS RAD)}.
static void fft_stage_twiddles(int log2n, std::vector<double>& out) {
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

// The compact form (fft_stage_tw_elems_ct): stage 1 as above, then the two
// factor tables of the stage with NS = 256 (N >= 512).
static void fft_stage_twiddles_ct(int log2n, std::vector<double>& out) {
  if (log2n <= 8) {
    fft_stage_twiddles(log2n, out);
    return;
  }
  out.clear();
  auto put = [&](double a) {
    out.push_back(std::cos(a));
    out.push_back(std::sin(a));
  };
  for (int r = 1; r < 16; ++r)
    for (int k = 0; k < 16; ++k) put(-2.0 * M_PI * double(r) * double(k) / 256.0);
  const int rad = 1 << (log2n - 8);
  const double span = 256.0 * double(rad);
  for (int r = 1; r < rad; ++r)
    for (int k1 = 0; k1 < 16; ++k1) put(-2.0 * M_PI * double(r) * double(16 * k1) / span);
  for (int r = 1; r < rad; ++r)
    for (int k0 = 0; k0 < 16; ++k0) put(-2.0 * M_PI * double(r) * double(k0) / span);
}

// e^{-2 pi i n/M}, n < N, as a product of two short tables:
// lo[i] = e^{-2 pi i i/M} (i < L), hi[j] = e^{-2 pi i L j/M} (j < N/L), L = min(64, N).
static int half_angle_tables(int n, std::vector<double>& lo, std::vector<double>& hi) {
  const int L = n < 64 ? n : 64;
  twiddles(L, 2 * n, lo);
  hi.resize(2 * (n / L));
  for (int j = 0; j < n / L; ++j) {
    const double a = -2.0 * M_PI * double(L) * double(j) / double(2 * n);
    hi[2 * j] = std::cos(a);
    hi[2 * j + 1] = std::sin(a);
  }
  int l = 0;
  while ((1 << l) < L) ++l;
  return l;
}

template <typename R>
static std::vector<R> cast(const std::vector<double>& v) {
  return std::vector<R>(v.begin(), v.end());
}

struct Builder {
  std::vector<unsigned char> bytes;
  size_t add(const void* p, size_t n) {
    const size_t off = (bytes.size() + 255) & ~size_t(255);
    bytes.resize(off + n);
    if (n) std::memcpy(bytes.data() + off, p, n);
    return off;
  }
  template <typename T>
  size_t add(const std::vector<T>& v) { return add(v.data(), v.size() * sizeof(T)); }
};


template <typename R>
static dsnu_status upload_spread(const HostSpread<R>& H, cudaStream_t st, void** block, PlanTables& t) {
  Builder b;
  const size_t o_ti = b.add(H.tile_items), o_ir = b.add(H.item_range), o_it = b.add(H.item_tile);
  const size_t o_en = b.add(H.ent_node), o_eq = b.add(H.ent_q0), o_ew = b.add(H.ent_w);
  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, b.bytes.size());
  if (e != cudaSuccess) return fail(DSNU_ENOMEM, std::string("cudaMalloc(spread tables): ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(dev, b.bytes.data(), b.bytes.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return fail(DSNU_ECUDA, std::string("spread table upload: ") + cudaGetErrorString(e));
  }
  char* d = static_cast<char*>(dev);
  t.tile_items = reinterpret_cast<int*>(d + o_ti);
  t.item_range = reinterpret_cast<int2*>(d + o_ir);
  t.item_tile = reinterpret_cast<int*>(d + o_it);
  t.ent_node = reinterpret_cast<int*>(d + o_en);
  t.ent_q0 = reinterpret_cast<int2*>(d + o_eq);
  t.ent_w = d + o_ew;
  *block = dev;
  return DSNU_OK;
}

static void set_spread_geom(PlanGeom& g, int cfg, int tiles_x, int tiles_y, int n_items, int max_tile) {
  g.spread_cfg = cfg;
  g.spread_tile = kSpreadCfgs[cfg].tile;
  g.tiles_x = tiles_x;
  g.tiles_y = tiles_y;
  g.n_tiles = tiles_x * tiles_y;
  g.n_items = n_items;
  g.max_tile_nodes = max_tile;
}

static void layout_workspace(dsnu_plan_s* P);

static std::mutex g_tune_mutex;
static std::map<std::string, int> g_tune_cache;

// Choose the spreading configuration: DSNU_AUTOTUNE=0 in the environment
// keeps the first candidate; otherwise every candidate of kSpreadCfgs is
// timed on scratch buffers (values do not change its cost) and the fastest is
// kept, cached per device and plan geometry for the process.
template <typename R>
static dsnu_status setup_spread(dsnu_plan_s* P, const std::vector<int2>& q0, const std::vector<R>& nw,
                                cudaStream_t st) {
  PlanGeom& g = P->geom;
  const dsnu_params& p = P->prm;
  int dev = 0;
  cudaGetDevice(&dev);
  // The spreading work depends on the node stencils on the fine grid, i.e. on
  // the polar rule, the disk, the ES width and the fine-grid spacing
  // pi/(2 l) per axis -- not on the number of grid points -- so plans that
  // share these share one tuned configuration (a batch of several grid sizes
  // then has one spreading configuration).
  char key[256];
  std::snprintf(key, sizeof(key), "%d|%.17g|%.17g|%.17g|%d|%d|%d|%d|%d", dev, p.lx, p.ly, p.cut_radius, p.n_r,
                p.n_theta, p.kernel_width, p.precision, p.radial_rule);
  const char* env = std::getenv("DSNU_AUTOTUNE");
  const bool tune = !(env && env[0] == '0');
  int choice = 0;
  bool have = !tune;
  // DSNU_SPREAD_CFG=<k> fixes candidate k of kSpreadCfgs (no timing)
  if (const char* fix = std::getenv("DSNU_SPREAD_CFG")) {
    const int k = std::atoi(fix);
    if (k >= 0 && k < kNumSpreadCfgs) {
      choice = k;
      have = true;
    }
  }
  if (tune && !have) {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      choice = it->second;
      have = true;
    }
  }
  if (!have) {
    float best = 1e30f;
    for (int c = 0; c < kNumSpreadCfgs; ++c) {
      HostSpread<R> H;
      bin_spread<R>(q0, nw, g.w, g.Q, kSpreadCfgs[c], H);
      void* blk = nullptr;
      PlanTables t = P->tab;
      dsnu_status s = upload_spread<R>(H, st, &blk, t);
      if (s != DSNU_OK) return s;
      set_spread_geom(g, c, H.tiles_x, H.tiles_y, H.n_items, H.max_tile);
      layout_workspace(P);
      void* ws = nullptr;
      cudaError_t e = cudaMalloc(&ws, P->ws_layout.total);
      if (e == cudaSuccess) e = cudaMemset(ws, 0, P->ws_layout.total);
      float ms = 0.f;
      if (e == cudaSuccess)
        e = (g.precision == DSNU_MIXED) ? time_spread_f32(g, t, P->ws_layout, ws, 5, &ms)
                                        : time_spread_f64(g, t, P->ws_layout, ws, 5, &ms);
      if (ws) cudaFree(ws);
      cudaFree(blk);
      if (e != cudaSuccess) return fail(DSNU_ECUDA, std::string("spread autotune: ") + cudaGetErrorString(e));
      if (ms < best) {
        best = ms;
        choice = c;
      }
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = choice;
  }
  HostSpread<R> H;
  bin_spread<R>(q0, nw, g.w, g.Q, kSpreadCfgs[choice], H);
  const dsnu_status s = upload_spread<R>(H, st, &P->spread_block, P->tab);
  if (s != DSNU_OK) return s;
  set_spread_geom(g, choice, H.tiles_x, H.tiles_y, H.n_items, H.max_tile);
  return DSNU_OK;
}

// The column multiplier of I1 (eq. SubInt1) on the padded grid,
//   m1(q_x, a) = -(q_x dk_x)^2 / s * (1 - p),  s = (q_x dk_x)^2 + (a dk_y)^2,
// with p = e^{-s/sigma^2} (Gaussian partition) or the indicator of s <= P^2
// (sharp), m1 = 0 at s = 0; computed in FP64 and stored in the plan's
// precision (one rounding for FP32).  Row q_x holds a = 2 j at j <= ny/2 and
// a = 2 j' + 1 at ny/2 + 1 + j', then zeros up to its ldm = ny + 4 entries.
template <typename T>
__global__ void k_fill_m1(T* tab, int nx1, int ny, int ldm, double dkx, double dky, double inv_sigma2, int sharp,
                          double cut2) {
  const long long n = (long long)nx1 * ldm;
  const int mh = ny / 2 + 1;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const int col = int(i / ldm), j = int(i - (long long)col * ldm);
    T v = T(0);
    if (j <= ny) {
      const int a = (j < mh) ? 2 * j : 2 * (j - mh) + 1;
      const double wx = col * dkx, wy = a * dky;
      const double wx2 = wx * wx, s = wx2 + wy * wy;
      if (s > 0.0) {
        const double part = sharp ? (s > cut2 ? 1.0 : 0.0) : -expm1(-s * inv_sigma2);
        v = T(-wx2 / s * part);
      }
    }
    tab[i] = v;
  }
}

template <typename R>
static dsnu_status build_m1_table(dsnu_plan_s* P, double dkx, double dky, cudaStream_t st) {
  const PlanGeom& g = P->geom;
  const int ldm = g.ny + 4;
  const size_t bytes = size_t(g.nx + 1) * ldm * sizeof(R);
  void* m = nullptr;
  cudaError_t e = cudaMalloc(&m, bytes);
  if (e != cudaSuccess) return fail(DSNU_ENOMEM, std::string("cudaMalloc(multiplier table): ") + cudaGetErrorString(e));
  k_fill_m1<R><<<1024, 256, 0, st>>>(static_cast<R*>(m), g.nx + 1, g.ny, ldm, dkx, dky, 1.0 / (g.sigma * g.sigma),
                                     g.sharp, g.cut_radius * g.cut_radius);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(m);
    return fail(DSNU_ECUDA, std::string("multiplier table: ") + cudaGetErrorString(e));
  }
  P->m1_block = m;
  P->tab.m1tab = m;
  return DSNU_OK;
}

template <typename R>
static dsnu_status build_tables(dsnu_plan_s* P, cudaStream_t st) {
  const dsnu_params& p = P->prm;
  PlanGeom& g = P->geom;
  const int nx = g.nx, ny = g.ny, Mx = g.mx, My = g.my, w = g.w;
  const double hx = 2.0 * p.lx / nx, hy = 2.0 * p.ly / ny;
  const double dkx = 2.0 * M_PI / (Mx * hx), dky = 2.0 * M_PI / (My * hy);
  const double sigma = g.sigma, beta = g.beta;

  // polar nodes and weights
  std::vector<double> rn, rw;
  radial_nodes(p.n_r, p.radial_rule, p.cut_radius, rn, rw);
  const int nn = p.n_r * p.n_theta;
  std::vector<double> kx(nn), ky(nn), D(nn);
  for (int i = 0; i < p.n_r; ++i) {
    const double r = rn[i];
    const double pr = g.sharp ? 1.0 : std::exp(-r * r / (sigma * sigma));
    for (int j = 0; j < p.n_theta; ++j) {
      const double th = 2.0 * M_PI * j / p.n_theta;
      const double c = std::cos(th), s = std::sin(th);
      kx[i * p.n_theta + j] = r * c;
      ky[i * p.n_theta + j] = r * s;
      if (g.m_generic)  // r^alpha (a0 + ac cos 2theta + as sin 2theta) in place of -cos^2 theta
        D[i * p.n_theta + j] = (rw[i] * std::pow(r, double(g.m_alpha)) *
                                (g.m_a0 + g.m_ac * (c * c - s * s) + g.m_as * 2.0 * s * c) *
                                (2.0 * M_PI / p.n_theta) * pr) / (4.0 * M_PI * M_PI);
      else
        D[i * p.n_theta + j] = -(rw[i] * (2.0 * M_PI / p.n_theta) * c * c * pr) / (4.0 * M_PI * M_PI);
    }
  }

  // ES kernel tables
  EsFourier fh(w, beta);
  const double ph0 = fh(0.0);
  HostTables<R> T;
  std::vector<double> tmp, tmp2;
  fft_stage_twiddles(g.log2nx, tmp); T.stw_x = cast<R>(tmp);
  fft_stage_twiddles(g.log2ny, tmp); T.stw_y = cast<R>(tmp);
  fft_stage_twiddles_ct(g.log2nx, tmp); T.stwc_x = cast<R>(tmp);
  if (int(T.stw_x.size()) != 2 * std::max(1, fft_stage_tw_elems(g.log2nx)) ||
      int(T.stw_y.size()) != 2 * std::max(1, fft_stage_tw_elems(g.log2ny)) ||
      int(T.stwc_x.size()) != 2 * std::max(1, fft_stage_tw_elems_ct(g.log2nx)))
    return fail(DSNU_EINVAL, "internal: stage twiddle table size mismatch");
  g.log2lo_x = half_angle_tables(nx, tmp, tmp2); T.twm_lo_x = cast<R>(tmp); T.twm_hi_x = cast<R>(tmp2);
  g.log2lo_y = half_angle_tables(ny, tmp, tmp2); T.twm_lo_y = cast<R>(tmp); T.twm_hi_y = cast<R>(tmp2);
  T.decon_x.resize(nx);
  for (int n = 0; n < nx; ++n) T.decon_x[n] = R(ph0 / fh(2.0 * M_PI * (n - nx / 2) / Mx));
  T.decon_y.resize(ny);
  for (int n = 0; n < ny; ++n) T.decon_y[n] = R(ph0 / fh(2.0 * M_PI * (n - ny / 2) / My));

  // multiplier axis tables: per column q_x; along y only the partition factor
  // 1 - exp(-(a dk_y)^2/sigma^2) up to the first |qbar_y| = a where it is 1 in
  // working precision ((a dk_y)^2 itself is formed in the kernel)
  T.m_wx2.resize(nx + 1);
  T.m_gx.resize(nx + 1);
  T.m_kx.resize(nx + 1);
  for (int q = 0; q <= nx; ++q) {
    const double a = q * dkx;
    T.m_wx2[q] = R(a * a);
    T.m_gx[q] = R(-std::expm1(-(a * a) / (sigma * sigma)));
    T.m_kx[q] = R(q < nx ? a : 0.0);  // Nyquist column: +-K averaged, the sin 2theta term vanishes
  }
  g.dky2 = dky * dky;
  T.m_gy.clear();
  if (!g.sharp) {
    for (int a = 0; a <= ny; ++a) {
      const double v = -std::expm1(-(a * dky) * (a * dky) / (sigma * sigma));
      if (R(v) == R(1)) break;
      T.m_gy.push_back(R(v));
    }
  }
  g.n_gy = int(T.m_gy.size());
  if (T.m_gy.empty()) T.m_gy.push_back(R(0));

  // per-node stencils
  T.node_q0.resize(nn);
  T.node_w.resize(size_t(nn) * 2 * w);
  T.node_D.resize(nn);
  int Q = 0;
  for (int j = 0; j < nn; ++j) {
    const double ux = kx[j] / dkx, uy = ky[j] / dky;
    const int q0x = int(std::ceil(ux - 0.5 * w));
    const int q0y = int(std::ceil(uy - 0.5 * w));
    T.node_q0[j] = make_int2(q0x, q0y);
    for (int a = 0; a < w; ++a) {
      T.node_w[size_t(j) * 2 * w + a] = R(es_kernel(ux - (q0x + a), w, beta));
      T.node_w[size_t(j) * 2 * w + w + a] = R(es_kernel(uy - (q0y + a), w, beta));
    }
    Q = std::max({Q, std::abs(q0x), std::abs(q0x + w - 1), std::abs(q0y), std::abs(q0y + w - 1)});
    // rho_hat = hx hy / phi_hat(0)^2 * (stencil sum), then the type-1 scale
    // Mx My / phi_hat(0)^2 so that both halves of the final complex inverse
    // transform carry comparable magnitudes.
    T.node_D[j] = D[j] * (hx * hy / (ph0 * ph0)) * (double(Mx) * double(My) / (ph0 * ph0));
  }
  if (Q > nx - 1 || Q > ny - 1)
    return fail(DSNU_EINVAL, "disk plus ES stencil does not fit the padded grid: need P*h + w*pi/M < pi");
  g.Q = Q;

  // interpolation items: nodes grouped by the kItile x kItile tile of the
  // plane of stencil origins q0 in [-Q, Q]^2 that holds theirs (node order
  // kept within a tile), each tile's nodes cut into items of at most
  // kItileNodes (the polar nodes crowd near the origin: a whole ring of small
  // radius falls in one tile); only tiles with nodes are listed
  {
    const int nt = (2 * Q + 1 + kItile - 1) / kItile;
    std::vector<int> cnt(size_t(nt) * nt, 0);
    std::vector<int> tix(nn);
    for (int j = 0; j < nn; ++j) {
      const int tx = (T.node_q0[j].x + Q) / kItile, ty = (T.node_q0[j].y + Q) / kItile;
      tix[j] = tx * nt + ty;
      ++cnt[tix[j]];
    }
    std::vector<int> first(size_t(nt) * nt, -1);
    T.itile_ptr.assign(1, 0);
    T.itile_org.clear();
    for (int t = 0; t < nt * nt; ++t)
      if (cnt[t] > 0) {
        first[t] = T.itile_ptr.back();
        for (int k = 0; k < cnt[t]; k += kItileNodes) {
          T.itile_ptr.push_back(T.itile_ptr.back() + std::min(kItileNodes, cnt[t] - k));
          T.itile_org.push_back(make_int2(-Q + (t / nt) * kItile, -Q + (t % nt) * kItile));
        }
      }
    T.itile_nodes.assign(nn, 0);
    for (int j = 0; j < nn; ++j) T.itile_nodes[first[tix[j]]++] = j;
    g.n_itiles = int(T.itile_org.size());
  }

  // one device block for every table
  Builder b;
  const size_t o_stx = b.add(T.stw_x), o_tlx = b.add(T.twm_lo_x), o_thx = b.add(T.twm_hi_x);
  const size_t o_dx = b.add(T.decon_x), o_scx = b.add(T.stwc_x);
  const size_t o_sty = b.add(T.stw_y), o_tly = b.add(T.twm_lo_y), o_thy = b.add(T.twm_hi_y);
  const size_t o_dy = b.add(T.decon_y);
  const size_t o_wx2 = b.add(T.m_wx2), o_gx = b.add(T.m_gx), o_gy = b.add(T.m_gy), o_kx = b.add(T.m_kx);
  const size_t o_q0 = b.add(T.node_q0), o_w = b.add(T.node_w), o_D = b.add(T.node_D);
  const size_t o_itp = b.add(T.itile_ptr), o_ito = b.add(T.itile_org), o_itn = b.add(T.itile_nodes);
  const int zero = 0;
  const size_t o_st = b.add(&zero, sizeof(int));
  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, b.bytes.size());
  if (e != cudaSuccess) return fail(DSNU_ENOMEM, std::string("cudaMalloc(plan tables): ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(dev, b.bytes.data(), b.bytes.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return fail(DSNU_ECUDA, std::string("plan table upload: ") + cudaGetErrorString(e));
  }
  char* d = static_cast<char*>(dev);
  PlanTables& t = P->tab;
  t.stw_x = d + o_stx; t.twm_lo_x = d + o_tlx; t.twm_hi_x = d + o_thx; t.decon_x = d + o_dx;
  t.stwc_x = d + o_scx;
  t.stw_y = d + o_sty; t.twm_lo_y = d + o_tly; t.twm_hi_y = d + o_thy; t.decon_y = d + o_dy;
  t.m_wx2 = d + o_wx2; t.m_gx = d + o_gx; t.m_gy = d + o_gy; t.m_kx = d + o_kx;
  t.node_q0 = reinterpret_cast<int2*>(d + o_q0);
  t.itile_ptr = reinterpret_cast<int*>(d + o_itp);
  t.itile_org = reinterpret_cast<int2*>(d + o_ito);
  t.itile_nodes = reinterpret_cast<int*>(d + o_itn);
  t.node_w = d + o_w;
  t.node_D = reinterpret_cast<double*>(d + o_D);
  t.status = reinterpret_cast<int*>(d + o_st);
  P->table_block = dev;
  P->table_bytes = b.bytes.size();
  if (!g.m_generic) {
    const dsnu_status sm = build_m1_table<R>(P, dkx, dky, st);
    if (sm != DSNU_OK) return sm;
  }
  return setup_spread<R>(P, T.node_q0, T.node_w, st);
}

// Tables of the standard periodic FFT solver: the stage twiddles of both
// axes and (q_x dk_x)^2 for q_x in [0, nx/2], dk = 2 pi/(2 l) (no padding).
template <typename R>
static dsnu_status build_tables_standard(dsnu_plan_s* P, cudaStream_t st) {
  const dsnu_params& p = P->prm;
  PlanGeom& g = P->geom;
  std::vector<double> tmp;
  fft_stage_twiddles(g.log2nx, tmp);
  const std::vector<R> stw_x = cast<R>(tmp);
  fft_stage_twiddles(g.log2ny, tmp);
  const std::vector<R> stw_y = cast<R>(tmp);
  fft_stage_twiddles_ct(g.log2nx, tmp);
  const std::vector<R> stwc_x = cast<R>(tmp);
  const double dkx = M_PI / p.lx, dky = M_PI / p.ly;
  std::vector<R> wx2(g.nx / 2 + 1), kx(g.nx / 2 + 1);
  for (int q = 0; q <= g.nx / 2; ++q) {
    wx2[q] = R((q * dkx) * (q * dkx));
    kx[q] = R(q < g.nx / 2 ? q * dkx : 0.0);  // Nyquist column: +-K averaged (no sin 2theta term)
  }
  g.dky2 = dky * dky;
  Builder b;
  const size_t o_stx = b.add(stw_x), o_sty = b.add(stw_y), o_wx2 = b.add(wx2), o_kx = b.add(kx);
  const size_t o_scx = b.add(stwc_x);
  const int zero = 0;
  const size_t o_st = b.add(&zero, sizeof(int));
  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, b.bytes.size());
  if (e != cudaSuccess) return fail(DSNU_ENOMEM, std::string("cudaMalloc(plan tables): ") + cudaGetErrorString(e));
  e = cudaMemcpyAsync(dev, b.bytes.data(), b.bytes.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(dev);
    return fail(DSNU_ECUDA, std::string("plan table upload: ") + cudaGetErrorString(e));
  }
  char* d = static_cast<char*>(dev);
  PlanTables& t = P->tab;
  t.stw_x = d + o_stx;
  t.stwc_x = d + o_scx;
  t.stw_y = d + o_sty;
  t.m_wx2 = d + o_wx2;
  t.m_kx = d + o_kx;
  t.status = reinterpret_cast<int*>(d + o_st);
  P->table_block = dev;
  P->table_bytes = b.bytes.size();
  return DSNU_OK;
}

static void layout_workspace(dsnu_plan_s* P) {  // defined after the autotuner, which uses it
  const PlanGeom& g = P->geom;
  const size_t csz = (g.precision == DSNU_MIXED) ? 8 : 16;
  WsLayout& L = P->ws_layout;
  if (g.standard) {  // one row-tiled half spectrum, q_x in [0, nx/2]
    L = WsLayout{};
    L.ldqA = g.nx / 2 + 1;
    L.total = (size_t(g.ny) * L.ldqA * csz + 255) & ~size_t(255);
    return;
  }
  L.ldqA = g.nx + 1;
  L.ldqB = g.Q + 1;
  L.ldq = 2 * g.Q + 1;
  size_t off = 0;
  auto take = [&](size_t n) {
    const size_t o = off;
    off = (off + n + 255) & ~size_t(255);
    return o;
  };
  L.off_A = take(size_t(g.ny) * L.ldqA * csz);
  L.off_B = take(size_t(g.ny) * L.ldqB * csz);
  L.off_Bband = take(size_t(g.Q + 1) * L.ldq * csz);
  L.off_Sband = take(size_t(g.Q + 1) * L.ldq * csz);
  L.off_c = take(size_t(g.n_nodes) * csz);
  L.off_partial = take(size_t(std::max(g.n_items, 1)) * g.spread_tile * g.spread_tile * csz);
  L.off_sched = take(sizeof(int));
  L.total = off;
}

}  // namespace dsnu

using namespace dsnu;

extern "C" {

const char* dsnu_last_error(void) { return g_last_error.c_str(); }

dsnu_status dsnu_plan_create(const dsnu_params* params, void* stream, dsnu_plan* out) {
  return dsnu_plan_create_multiplier(params, nullptr, stream, out);
}

dsnu_status dsnu_plan_create_multiplier(const dsnu_params* params, const dsnu_multiplier* mult, void* stream,
                                        dsnu_plan* out) {
  if (!params || !out) return fail(DSNU_EINVAL, "NULL params or out");
  if (mult) {
    if (mult->alpha < -1 || mult->alpha > 1) return fail(DSNU_EINVAL, "multiplier alpha must be -1, 0 or 1");
    if (!std::isfinite(mult->a0) || !std::isfinite(mult->a_cos) || !std::isfinite(mult->a_sin))
      return fail(DSNU_EINVAL, "multiplier coefficients must be finite");
  }
  dsnu_params p = *params;
  if (!is_pow2(p.nx) || !is_pow2(p.ny) || p.nx < 16 || p.ny < 16 || p.nx > 4096 || p.ny > 4096)
    return fail(DSNU_EINVAL, "nx, ny must be powers of two in [16, 4096]");
  if (!(p.lx > 0.0) || !(p.ly > 0.0) || !std::isfinite(p.lx) || !std::isfinite(p.ly))
    return fail(DSNU_EINVAL, "lx, ly must be positive and finite");
  if (p.precision != DSNU_FP64 && p.precision != DSNU_MIXED) return fail(DSNU_EINVAL, "unknown precision");
  if (p.accumulation != DSNU_ACCUM_FP64 && p.accumulation != DSNU_ACCUM_WORKING)
    return fail(DSNU_EINVAL, "unknown accumulation");
  if (p.partition != DSNU_PARTITION_GAUSS && p.partition != DSNU_PARTITION_SHARP &&
      p.partition != DSNU_PARTITION_NONE)
    return fail(DSNU_EINVAL, "unknown partition");
  const bool standard = (p.partition == DSNU_PARTITION_NONE);
  if (standard) {
    // the standard periodic FFT solver: no polar part, no padding
    if (p.pad_factor != 1) return fail(DSNU_EINVAL, "partition NONE (standard FFT solver) needs pad_factor = 1");
    p.cut_radius = 0.0;
    p.sigma = 0.0;
    p.n_r = p.n_theta = p.kernel_width = 0;
  } else {
    if (p.pad_factor == 1) return fail(DSNU_EINVAL, "pad_factor = 1 is the standard solver: partition NONE");
    if (p.pad_factor != 0 && p.pad_factor != 2) return fail(DSNU_EUNSUPPORTED, "only pad_factor = 2 is supported");
    if (!(p.cut_radius > 0.0) || !std::isfinite(p.cut_radius))
      return fail(DSNU_EINVAL, "cut_radius must be positive");
    if (p.sigma < 0.0 || !std::isfinite(p.sigma)) return fail(DSNU_EINVAL, "sigma must be >= 0");
    if (p.n_r < 1 || p.n_r > 4096) return fail(DSNU_EINVAL, "n_r must be in [1, 4096]");
    if (p.n_theta < 2 || (p.n_theta & 1) || p.n_theta > 65536)
      return fail(DSNU_EINVAL, "n_theta must be even, >= 2");
    if (p.radial_rule != DSNU_RADIAL_LEGENDRE && p.radial_rule != DSNU_RADIAL_JACOBI)
      return fail(DSNU_EINVAL, "unknown radial_rule");
    if (p.kernel_width == 0) p.kernel_width = (p.precision == DSNU_FP64) ? 15 : 8;
    if (p.kernel_width < 2 || p.kernel_width > 16) return fail(DSNU_EINVAL, "kernel_width must be in [2, 16]");
    if (p.sigma == 0.0) p.sigma = p.cut_radius / 6.0;
    p.pad_factor = 2;
    if (long(p.n_r) * long(p.n_theta) > (1L << 24)) return fail(DSNU_EINVAL, "too many polar nodes");
  }

  dsnu_plan_s* P = new (std::nothrow) dsnu_plan_s();
  if (!P) return fail(DSNU_ENOMEM, "host allocation failed");
  P->prm = p;
  PlanGeom& g = P->geom;
  g.nx = p.nx;
  g.ny = p.ny;
  g.standard = standard ? 1 : 0;
  {
    const char* env = std::getenv("DSNU_PDL");  // DSNU_PDL=0: plain stream-ordered launches
    g.pdl = (env && env[0] == '0') ? 0 : 1;
  }
  if (mult) {
    g.m_generic = 1;
    g.m_alpha = mult->alpha;
    g.m_a0 = mult->a0;
    g.m_ac = mult->a_cos;
    g.m_as = mult->a_sin;
  }
  g.mx = p.pad_factor * p.nx;
  g.my = p.pad_factor * p.ny;
  g.log2nx = ilog2(p.nx);
  g.log2ny = ilog2(p.ny);
  g.w = p.kernel_width;
  g.beta = 2.30 * p.kernel_width;
  g.sigma = p.sigma;
  g.cut_radius = p.cut_radius;
  g.n_nodes = p.n_r * p.n_theta;
  g.precision = p.precision;
  g.acc64 = (p.precision == DSNU_MIXED && p.accumulation == DSNU_ACCUM_FP64) ? 1 : 0;
  g.sharp = (p.partition == DSNU_PARTITION_SHARP);
  g.scale = 1.0 / (double(g.mx) * double(g.my));
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  dsnu_status s;
  if (standard)
    s = (p.precision == DSNU_MIXED) ? build_tables_standard<float>(P, st) : build_tables_standard<double>(P, st);
  else
    s = (p.precision == DSNU_MIXED) ? build_tables<float>(P, st) : build_tables<double>(P, st);
  if (s != DSNU_OK) {
    if (P->spread_block) cudaFree(P->spread_block);
    if (P->m1_block) cudaFree(P->m1_block);
    if (P->table_block) cudaFree(P->table_block);
    delete P;
    return s;
  }
  const cudaError_t e = (p.precision == DSNU_MIXED) ? prepare_kernels_f32(g) : prepare_kernels_f64(g);
  if (e != cudaSuccess) {
    if (P->spread_block) cudaFree(P->spread_block);
    if (P->m1_block) cudaFree(P->m1_block);
    cudaFree(P->table_block);
    delete P;
    return fail(DSNU_ECUDA, std::string("kernel attributes: ") + cudaGetErrorString(e));
  }
  layout_workspace(P);
  // mixed plans on large grids: the band chain runs next to the column pass
  // on a low-priority side stream, the column pass leaving it 16 of every 152
  // SMs at 4096^2 and a share growing as 1/sqrt(nx ny) for smaller grids,
  // whose band chain (its node work is the same) is larger next to their
  // column pass: measured best on GB300 16 SMs at 4096^2 (0.5137 ms against
  // 0.5226 with 12 and 0.534 with the band chain in line) and 32 at 2048^2
  // (0.131-0.134 ms against 0.139 with 16 and 0.150 in line);
  // DSNU_BAND_SMS=<n> sets the number of SMs, 0 turns it off
  if (p.precision == DSNU_MIXED && !standard) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int reserve = 0;
    if (p.nx >= 2048 && p.ny >= 2048)
      reserve = std::max(1, int(std::lround(sms * (16.0 / 152.0) * 4096.0 / std::sqrt(double(p.nx) * p.ny))));
    const char* env = std::getenv("DSNU_BAND_SMS");
    if (env) reserve = std::atoi(env);
    if (reserve > 0) {
      int lo = 0, hi = 0;
      cudaError_t ce = cudaDeviceGetStreamPriorityRange(&lo, &hi);
      if (ce == cudaSuccess) ce = cudaStreamCreateWithPriority(&P->overlap.side, cudaStreamNonBlocking, lo);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&P->overlap.fork, cudaEventDisableTiming);
      if (ce == cudaSuccess) ce = cudaEventCreateWithFlags(&P->overlap.join, cudaEventDisableTiming);
      if (ce == cudaSuccess) P->overlap.reserve = reserve;
    }
  }
  *out = P;
  return DSNU_OK;
}

size_t dsnu_workspace_bytes(dsnu_plan plan) { return plan ? plan->ws_layout.total : 0; }

dsnu_status dsnu_set_workspace(dsnu_plan plan, void* ws, size_t bytes) {
  if (!plan || !ws) return fail(DSNU_EINVAL, "NULL plan or workspace");
  if (bytes < plan->ws_layout.total) return fail(DSNU_EINVAL, "workspace too small");
  if (reinterpret_cast<uintptr_t>(ws) & 255) return fail(DSNU_EINVAL, "workspace must be 256-byte aligned");
  plan->ws = ws;
  plan->ws_bytes = bytes;
  return DSNU_OK;
}

static dsnu_status run(dsnu_plan plan, const double* in, double* out, void* stream, int cj) {
  if (!plan) return fail(DSNU_EINVAL, "NULL plan");
  if (!in || !out) return fail(DSNU_EINVAL, "NULL input or output");
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) & 15)
    return fail(DSNU_EINVAL, "input and output must be 16-byte aligned");
  if (!plan->ws) return fail(DSNU_EINVAL, "no workspace attached (dsnu_set_workspace)");
  const size_t nbytes = size_t(plan->geom.nx) * plan->geom.ny * sizeof(double);
  const char* a = reinterpret_cast<const char*>(in);
  const char* b = reinterpret_cast<const char*>(out);
  if (a < b + nbytes && b < a + nbytes) return fail(DSNU_EINVAL, "input and output overlap");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaEvent_t* ev = nullptr;
  if (plan->prof_events && plan->prof_used < plan->prof_max)
    ev = plan->prof_events + size_t(plan->prof_used++) * kProfEvents;
  if (plan->geom.precision == DSNU_MIXED)
    return run_pipeline_f32(plan->geom, plan->tab, plan->ws_layout, single_member(in, out, plan->ws), st,
                            cj, ev, plan->overlap.reserve > 0 ? &plan->overlap : nullptr);
  return run_pipeline_f64(plan->geom, plan->tab, plan->ws_layout, single_member(in, out, plan->ws), st, cj,
                          ev);
}

static void free_profile(dsnu_plan plan) {
  if (!plan->prof_events) return;
  for (int i = 0; i < plan->prof_max * kProfEvents; ++i) cudaEventDestroy(plan->prof_events[i]);
  delete[] plan->prof_events;
  plan->prof_events = nullptr;
  plan->prof_max = plan->prof_used = 0;
}

dsnu_status dsnu_solve(dsnu_plan plan, const double* rho, double* phi, void* stream) {
  return run(plan, rho, phi, stream, 0);
}

dsnu_status dsnu_solve_adjoint(dsnu_plan plan, const double* g, double* out, void* stream) {
  return run(plan, g, out, stream, 1);
}

dsnu_status dsnu_status_poll(dsnu_plan plan, void* stream) {
  if (!plan) return fail(DSNU_EINVAL, "NULL plan");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, plan->tab.status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess && h != 0) e = cudaMemsetAsync(plan->tab.status, 0, sizeof(int), st);
  if (e != cudaSuccess) return fail(DSNU_ECUDA, std::string("status poll: ") + cudaGetErrorString(e));
  return static_cast<dsnu_status>(h);
}

dsnu_status dsnu_plan_destroy(dsnu_plan plan) {
  if (!plan) return DSNU_OK;
  free_profile(plan);
  if (plan->overlap.reserve > 0) {
    cudaStreamSynchronize(plan->overlap.side);
    cudaStreamDestroy(plan->overlap.side);
    cudaEventDestroy(plan->overlap.fork);
    cudaEventDestroy(plan->overlap.join);
  }
  if (plan->has_copy_streams) {
    cudaStreamSynchronize(plan->copy_in);
    cudaStreamSynchronize(plan->copy_out);
    cudaStreamDestroy(plan->copy_in);
    cudaStreamDestroy(plan->copy_out);
    cudaEventDestroy(plan->ev_start);
    for (int k = 0; k < 2; ++k) {
      cudaEventDestroy(plan->ev_in[k]);
      cudaEventDestroy(plan->ev_solved[k]);
      cudaEventDestroy(plan->ev_out[k]);
    }
  }
  if (plan->spread_block) cudaFree(plan->spread_block);
  if (plan->m1_block) cudaFree(plan->m1_block);
  cudaError_t e = cudaFree(plan->table_block);
  delete plan;
  if (e != cudaSuccess) return fail(DSNU_ECUDA, std::string("cudaFree: ") + cudaGetErrorString(e));
  return DSNU_OK;
}

dsnu_status dsnu_solve_host(dsnu_plan plan, const double* rho_host, double* phi_host, double* rho_dev,
                            double* phi_dev, void* stream) {
  if (!plan) return fail(DSNU_EINVAL, "NULL plan");
  if (!rho_host || !phi_host || !rho_dev || !phi_dev) return fail(DSNU_EINVAL, "NULL buffer");
  if ((reinterpret_cast<uintptr_t>(rho_dev) | reinterpret_cast<uintptr_t>(phi_dev)) & 15)
    return fail(DSNU_EINVAL, "device buffers must be 16-byte aligned");
  if (!plan->ws) return fail(DSNU_EINVAL, "no workspace attached (dsnu_set_workspace)");
  const size_t nbytes = size_t(plan->geom.nx) * plan->geom.ny * sizeof(double);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemcpyAsync(rho_dev, rho_host, nbytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail(DSNU_ECUDA, std::string("H2D copy: ") + cudaGetErrorString(e));
  const dsnu_status s = run(plan, rho_dev, phi_dev, stream, 0);
  if (s != DSNU_OK) return s;
  e = cudaMemcpyAsync(phi_host, phi_dev, nbytes, cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return fail(DSNU_ECUDA, std::string("D2H copy: ") + cudaGetErrorString(e));
  return DSNU_OK;
}

size_t dsnu_stream_staging_bytes(dsnu_plan plan) {
  return plan ? 4 * ((size_t(plan->geom.nx) * plan->geom.ny * sizeof(double) + 255) & ~size_t(255)) : 0;
}

static cudaError_t make_copy_streams(dsnu_plan p) {
  if (p->has_copy_streams) return cudaSuccess;
  cudaError_t e = cudaStreamCreateWithFlags(&p->copy_in, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&p->copy_out, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_start, cudaEventDisableTiming);
  for (int k = 0; k < 2 && e == cudaSuccess; ++k) {
    e = cudaEventCreateWithFlags(&p->ev_in[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_solved[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->ev_out[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) p->has_copy_streams = true;
  return e;
}

dsnu_status dsnu_solve_host_stream(dsnu_plan plan, int32_t count, const double* const* rho_host,
                                   double* const* phi_host, void* staging_dev, size_t staging_bytes,
                                   void* stream) {
  if (!plan) return fail(DSNU_EINVAL, "NULL plan");
  if (count < 1 || !rho_host || !phi_host || !staging_dev) return fail(DSNU_EINVAL, "count >= 1 and buffers required");
  for (int i = 0; i < count; ++i)
    if (!rho_host[i] || !phi_host[i]) return fail(DSNU_EINVAL, "NULL host buffer");
  if (staging_bytes < dsnu_stream_staging_bytes(plan)) return fail(DSNU_EINVAL, "staging buffer too small");
  if (reinterpret_cast<uintptr_t>(staging_dev) & 255) return fail(DSNU_EINVAL, "staging must be 256-byte aligned");
  if (!plan->ws) return fail(DSNU_EINVAL, "no workspace attached (dsnu_set_workspace)");
  cudaError_t e = make_copy_streams(plan);
  if (e != cudaSuccess) return fail(DSNU_ECUDA, std::string("copy streams: ") + cudaGetErrorString(e));
  const size_t nbytes = size_t(plan->geom.nx) * plan->geom.ny * sizeof(double);
  const size_t slot = (nbytes + 255) & ~size_t(255);
  char* base = static_cast<char*>(staging_dev);
  double* rho_s[2] = {reinterpret_cast<double*>(base), reinterpret_cast<double*>(base + slot)};
  double* phi_s[2] = {reinterpret_cast<double*>(base + 2 * slot), reinterpret_cast<double*>(base + 3 * slot)};
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // the copy streams start after the caller's earlier work on `stream`
  e = cudaEventRecord(plan->ev_start, st);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->copy_in, plan->ev_start, 0);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->copy_out, plan->ev_start, 0);
  for (int i = 0; i < count && e == cudaSuccess; ++i) {
    const int k = i & 1;
    // slot k's density is free once solve i-2 has read it
    if (i >= 2) e = cudaStreamWaitEvent(plan->copy_in, plan->ev_solved[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(rho_s[k], rho_host[i], nbytes, cudaMemcpyHostToDevice, plan->copy_in);
    if (e == cudaSuccess) e = cudaEventRecord(plan->ev_in[k], plan->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(st, plan->ev_in[k], 0);
    // slot k's potential is free once download i-2 has finished
    if (e == cudaSuccess && i >= 2) e = cudaStreamWaitEvent(st, plan->ev_out[k], 0);
    if (e != cudaSuccess) break;
    const dsnu_status s = run(plan, rho_s[k], phi_s[k], stream, 0);
    if (s != DSNU_OK) return s;
    e = cudaEventRecord(plan->ev_solved[k], st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(plan->copy_out, plan->ev_solved[k], 0);
    if (e == cudaSuccess) e = cudaMemcpyAsync(phi_host[i], phi_s[k], nbytes, cudaMemcpyDeviceToHost, plan->copy_out);
    if (e == cudaSuccess) e = cudaEventRecord(plan->ev_out[k], plan->copy_out);
  }
  // `stream` is ordered after every download (the last one covers the others)
  if (e == cudaSuccess) e = cudaStreamWaitEvent(st, plan->ev_out[(count - 1) & 1], 0);
  if (e != cudaSuccess) return fail(DSNU_ECUDA, std::string("streamed solve: ") + cudaGetErrorString(e));
  return DSNU_OK;
}

dsnu_status dsnu_profile_begin(dsnu_plan plan, int max_solves) {
  if (!plan || max_solves < 1 || max_solves > (1 << 20)) return fail(DSNU_EINVAL, "bad plan or max_solves");
  if (plan->prof_events) return fail(DSNU_EINVAL, "profiling already active");
  const int n = max_solves * kProfEvents;
  cudaEvent_t* ev = new (std::nothrow) cudaEvent_t[n];
  if (!ev) return fail(DSNU_ENOMEM, "host allocation failed");
  for (int i = 0; i < n; ++i) {
    const cudaError_t e = cudaEventCreate(&ev[i]);
    if (e != cudaSuccess) {
      for (int k = 0; k < i; ++k) cudaEventDestroy(ev[k]);
      delete[] ev;
      return fail(DSNU_ECUDA, std::string("cudaEventCreate: ") + cudaGetErrorString(e));
    }
  }
  plan->prof_events = ev;
  plan->prof_max = max_solves;
  plan->prof_used = 0;
  return DSNU_OK;
}

dsnu_status dsnu_profile_end(dsnu_plan plan, double* stage_ms, int n_stages, int* n_solves) {
  if (!plan || !stage_ms || n_stages < kStages) return fail(DSNU_EINVAL, "bad arguments");
  if (!plan->prof_events) return fail(DSNU_EINVAL, "profiling not active");
  for (int k = 0; k < kStages; ++k) stage_ms[k] = 0.0;
  dsnu_status st = DSNU_OK;
  // stage k runs between events (from[k], to[k]) of a solve (see run_pipeline)
  // stage k runs between events k and k + 1 (launch order)
  for (int s = 0; s < plan->prof_used && st == DSNU_OK; ++s) {
    cudaEvent_t* ev = plan->prof_events + size_t(s) * kProfEvents;
    cudaError_t e = cudaEventSynchronize(ev[kProfEvents - 1]);
    for (int k = 0; k < kStages && e == cudaSuccess; ++k) {
      float ms = 0.f;
      e = cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
      stage_ms[k] += ms;
    }
    if (e != cudaSuccess) st = fail(DSNU_ECUDA, std::string("profile events: ") + cudaGetErrorString(e));
  }
  if (n_solves) *n_solves = plan->prof_used;
  free_profile(plan);
  return st;
}

dsnu_status dsnu_radial_nodes(int32_t n_r, int32_t rule, double cut_radius, double* r, double* w) {
  if (n_r < 1 || n_r > 4096 || !r || !w || !(cut_radius > 0.0) || !std::isfinite(cut_radius))
    return fail(DSNU_EINVAL, "n_r in [1, 4096], cut_radius > 0 and output arrays required");
  if (rule != DSNU_RADIAL_LEGENDRE && rule != DSNU_RADIAL_JACOBI) return fail(DSNU_EINVAL, "unknown radial rule");
  std::vector<double> rn, rw;
  radial_nodes(n_r, rule, cut_radius, rn, rw);
  for (int i = 0; i < n_r; ++i) {
    r[i] = rn[i];
    w[i] = rw[i];
  }
  return DSNU_OK;
}

dsnu_status dsnu_params_auto(int32_t nx, int32_t ny, double lx, double ly, double eps, int32_t precision,
                             dsnu_params* out) {
  if (!out) return fail(DSNU_EINVAL, "NULL out");
  if (!is_pow2(nx) || !is_pow2(ny) || nx < 16 || ny < 16 || nx > 4096 || ny > 4096)
    return fail(DSNU_EINVAL, "nx, ny must be powers of two in [16, 4096]");
  if (!(lx > 0.0) || !(ly > 0.0) || !std::isfinite(lx) || !std::isfinite(ly))
    return fail(DSNU_EINVAL, "lx, ly must be positive and finite");
  if (precision != DSNU_FP64 && precision != DSNU_MIXED) return fail(DSNU_EINVAL, "unknown precision");
  if (!(eps > 0.0) || !(eps < 1.0)) return fail(DSNU_EINVAL, "eps must be in (0, 1)");
  eps = std::min(std::max(eps, precision == DSNU_MIXED ? 1e-7 : 1e-15), 1e-2);
  const double sigma = 12.0 / std::min(lx, ly);             // sigma L = 12
  const double c = sigma * std::sqrt(std::log(1.0 / eps));  // p(c) = eps
  const double cR = c * std::sqrt(lx * lx + ly * ly);       // largest phase of e^{i k.x} on the disk
  const int n_theta = 4 * int(std::ceil((cR + 16.0) / 4.0));
  const int n_r = 8 * int(std::ceil((0.5 * cR + 4.0) / 8.0));
  const int w = (precision == DSNU_FP64) ? 15 : 8;
  const double hx = 2.0 * lx / nx, hy = 2.0 * ly / ny;
  if (c * hx + w * M_PI / (2.0 * nx) >= M_PI || c * hy + w * M_PI / (2.0 * ny) >= M_PI)
    return fail(DSNU_EINVAL, "grid too coarse for this domain: the disk radius 12 sqrt(ln 1/eps)/min(lx, ly) "
                             "plus the ES stencil exceeds the padded frequency grid");
  dsnu_params p{};
  p.nx = nx;
  p.ny = ny;
  p.lx = lx;
  p.ly = ly;
  p.cut_radius = c;
  p.sigma = sigma;
  p.n_r = n_r;
  p.n_theta = n_theta;
  p.kernel_width = 0;
  p.pad_factor = 2;
  p.precision = precision;
  p.partition = DSNU_PARTITION_GAUSS;
  p.radial_rule = DSNU_RADIAL_JACOBI;
  *out = p;
  return DSNU_OK;
}

int32_t dsnu_stage_count(void) { return kStages; }

const char* dsnu_stage_name(int32_t stage) {
  static const char* names[kStages] = {"row_fwd", "band_fwd", "interp", "spread",
                                       "spread_reduce", "band_inv", "col_main", "row_inv"};
  return (stage >= 0 && stage < kStages) ? names[stage] : "";
}

dsnu_status dsnu_plan_get_info(dsnu_plan plan, dsnu_plan_info* info) {
  if (!plan || !info) return fail(DSNU_EINVAL, "NULL plan or info");
  const PlanGeom& g = plan->geom;
  info->n_nodes = g.n_nodes;
  info->band_q = g.Q;
  info->kernel_width = g.w;
  info->precision = g.precision;
  info->sigma = g.sigma;
  info->es_beta = g.beta;
  info->n_tiles = g.n_tiles;
  info->max_tile_nodes = g.max_tile_nodes;
  info->n_items = g.n_items;
  info->spread_tile = g.spread_tile;
  info->spread_split = kSpreadCfgs[g.spread_cfg].split;
  info->spread_chunk = kSpreadCfgs[g.spread_cfg].chunk;
  info->row_prefetch = g.standard ? 0 : g.row_pf;
  info->reserved = 0;
  return DSNU_OK;
}

}  // extern "C"
