// measure.cu -- arithmetic throughput of this GPU, the denominator of the
// FP64 path's roofline (its column and row passes are bound by FP64
// arithmetic, not by HBM).  Not part of the solver: a plain FMA loop timed
// with CUDA events, which touches no device setting.
#include <cuda_runtime.h>

#include <string>

#include "dsnu_measure.h"
#include "internal.h"

namespace {

constexpr int kChains = 8;  // independent FMA chains per thread (latency hiding)

// Every thread runs `iters` rounds of kChains dependent-free FMAs
// a_c <- a_c * x + y; one value per thread is stored so that nothing is
// optimised away.
template <typename T>
__global__ void __launch_bounds__(256) k_fma_loop(T* out, int iters, T x, T y) {
  T a[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) a[c] = T(threadIdx.x + c);
#pragma unroll 1
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 16; ++k)
#pragma unroll
      for (int c = 0; c < kChains; ++c) a[c] = fma(a[c], x, y);
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < kChains; ++c) s += a[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename T>
dsnu_status run(double* flops_per_s, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int per_sm = 0;
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fma_loop<T>, 256, 0);
  if (e != cudaSuccess) {
    dsnu::set_last_error(std::string("measure: ") + cudaGetErrorString(e));
    return DSNU_ECUDA;
  }
  const int blocks = sms * (per_sm > 0 ? per_sm : 1);
  // FP64 runs at a small fraction of FP32 on this part: fewer rounds keep
  // the FP64 run near 0.1 s
  const int iters = sizeof(T) == 8 ? 256 : 8192;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  e = cudaMalloc(&out, size_t(blocks) * 256 * sizeof(T));
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float ms = 0.f, best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {  // first launch warms up
    cudaEventRecord(e0, st);
    k_fma_loop<T><<<blocks, 256, 0, st>>>(out, iters, T(0.999999), T(1e-7));
    cudaEventRecord(e1, st);
    e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (rep > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (out) cudaFree(out);
  if (e != cudaSuccess) {
    dsnu::set_last_error(std::string("measure: ") + cudaGetErrorString(e));
    return DSNU_ECUDA;
  }
  const double flops = 2.0 * double(blocks) * 256.0 * double(iters) * 16.0 * kChains;
  *flops_per_s = flops / (double(best) * 1e-3);
  return DSNU_OK;
}

}  // namespace

extern "C" dsnu_status dsnu_measure_fma_peak(int32_t precision, double* flops_per_s, void* stream) {
  if (!flops_per_s || (precision != DSNU_FP64 && precision != DSNU_MIXED)) {
    dsnu::set_last_error("dsnu_measure_fma_peak: precision must be DSNU_FP64 or DSNU_MIXED, output non-NULL");
    return DSNU_EINVAL;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return precision == DSNU_FP64 ? run<double>(flops_per_s, st) : run<float>(flops_per_s, st);
}
