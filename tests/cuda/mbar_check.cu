// Checks the bounded mbarrier wait and the asynchronous copies of common.cuh
// that the row passes use:
//   1. a wait on a phase that nothing completes gives up after its time limit
//      and returns false (the kernel's own status path; no fault, no hang);
//   2. one arrival completes the phase and the wait returns true;
//   3. a bulk copy global -> shared completes its expected bytes on the next
//      phase and the data arrive intact;
//   4. per-thread 16-byte cp.async copies land after cp_async_wait_all;
//   5. the way out of a prefetching loop (cta_timed_out): when every thread's
//      wait expired (a phase that no copy completes, so nothing is in flight),
//      the CTA records DSNU_ETIMEOUT in the status word and returns without
//      writing; when the phase completed, it carries on and writes.
// Prints "OK <elapsed ns of the expired wait>" or "FAIL ..."; exit status 0 on
// success.
#include <cstdio>
#include <vector>

#include "common.cuh"

constexpr int kThreads = 128;
constexpr int kWords = 1024;  // doubles copied in cases 3 and 4 (8 KB)

__global__ void k_mbar(const double* src, int* res, unsigned long long* elapsed, unsigned long long limit_ns) {
  __shared__ unsigned long long bar;
  __shared__ __align__(16) double buf[kWords];
  __shared__ __align__(16) double buf2[kWords];
  const int tid = threadIdx.x;
  if (tid == 0) dsnu::mbar_init(&bar, 1);
  __syncthreads();
  // 1: phase 0 never completes (no arrival)
  const unsigned long long t0 = dsnu::global_ns();
  const bool expired_ok = dsnu::mbar_wait(&bar, 0, limit_ns);
  const unsigned long long t1 = dsnu::global_ns();
  if (expired_ok) atomicOr(&res[0], 1);
  if (tid == 0) elapsed[0] = t1 - t0;
  __syncthreads();
  // 2: one arrival (no bytes expected) completes phase 0
  if (tid == 0) dsnu::mbar_expect_tx(&bar, 0);
  if (!dsnu::mbar_wait(&bar, 0, 1000000000ull)) atomicOr(&res[1], 1);
  __syncthreads();
  // 3: a bulk copy completes phase 1
  if (tid == 0) {
    const unsigned long long pol = dsnu::l2_evict_first();
    dsnu::mbar_expect_tx(&bar, kWords * sizeof(double));
    dsnu::bulk_load(buf, src, kWords * sizeof(double), &bar, pol);
  }
  if (!dsnu::mbar_wait(&bar, 1, 1000000000ull)) atomicOr(&res[2], 1);
  for (int i = tid; i < kWords; i += kThreads)
    if (buf[i] != src[i]) atomicOr(&res[3], 1);
  // 4: per-thread 16-byte asynchronous copies
  for (int i = tid; i < kWords / 2; i += kThreads) dsnu::cp_async16(buf2 + 2 * i, src + 2 * i);
  dsnu::cp_async_commit();
  dsnu::cp_async_wait_all();
  __syncthreads();
  for (int i = tid; i < kWords; i += kThreads)
    if (buf2[i] != src[i]) atomicOr(&res[4], 1);
}

__global__ void k_exit(int* status, int* wrote, int arrive, unsigned long long limit_ns) {
  __shared__ unsigned long long bar;
  if (threadIdx.x == 0) dsnu::mbar_init(&bar, 1);
  __syncthreads();
  if (arrive && threadIdx.x == 0) dsnu::mbar_expect_tx(&bar, 0);  // completes phase 0
  const bool landed = dsnu::mbar_wait(&bar, 0, limit_ns);
  if (dsnu::cta_timed_out(landed, &bar, 0, status, limit_ns)) return;
  if (threadIdx.x == 0) atomicAdd(wrote, 1);
}

int main() {
  std::vector<double> h(kWords);
  for (int i = 0; i < kWords; ++i) h[i] = 0.5 * i - 3.25;
  double* d = nullptr;
  int* res = nullptr;
  unsigned long long* el = nullptr;
  if (cudaMalloc(&d, kWords * sizeof(double)) != cudaSuccess || cudaMalloc(&res, 5 * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&el, sizeof(unsigned long long)) != cudaSuccess) {
    std::printf("FAIL cudaMalloc\n");
    return 1;
  }
  cudaMemcpy(d, h.data(), kWords * sizeof(double), cudaMemcpyHostToDevice);
  cudaMemset(res, 0, 5 * sizeof(int));
  const unsigned long long limit = 2000000ull;  // 2 ms
  k_mbar<<<2, kThreads>>>(d, res, el, limit);
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    std::printf("FAIL %s\n", cudaGetErrorString(e));
    return 1;
  }
  int r[5];
  unsigned long long ns = 0;
  cudaMemcpy(r, res, sizeof(r), cudaMemcpyDeviceToHost);
  cudaMemcpy(&ns, el, sizeof(ns), cudaMemcpyDeviceToHost);
  // 5: the exit path, with and without an expired wait (status word, writes)
  int* ex = nullptr;  // [status, wrote] for "expired", then for "arrived"
  if (cudaMalloc(&ex, 4 * sizeof(int)) != cudaSuccess) {
    std::printf("FAIL cudaMalloc\n");
    return 1;
  }
  cudaMemset(ex, 0, 4 * sizeof(int));
  k_exit<<<2, kThreads>>>(ex, ex + 1, 0, limit);
  k_exit<<<2, kThreads>>>(ex + 2, ex + 3, 1, limit);
  const cudaError_t e5 = cudaDeviceSynchronize();
  int x[4] = {-1, -1, -1, -1};
  cudaMemcpy(x, ex, sizeof(x), cudaMemcpyDeviceToHost);
  const bool exit_ok = e5 == cudaSuccess && x[0] == int(DSNU_ETIMEOUT) && x[1] == 0 && x[2] == 0 && x[3] == 2;
  const bool ok = r[0] == 0 && r[1] == 0 && r[2] == 0 && r[3] == 0 && r[4] == 0 && ns >= limit &&
                  ns < 100 * limit && exit_ok;
  std::printf("%s %llu expired=%d arrive=%d bulk=%d bulk_data=%d cp_async=%d exit=%d,%d,%d,%d\n", ok ? "OK" : "FAIL",
              ns, r[0], r[1], r[2], r[3], r[4], x[0], x[1], x[2], x[3]);
  return ok ? 0 : 1;
}
