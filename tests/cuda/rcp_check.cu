// Checks dsnu::rcp_nr (Newton-Raphson FP64 reciprocal) and the FP64 fdiv built
// on it against CUDA's IEEE division over wide, seeded ranges of normal
// inputs.  Prints "OK <max ulp of 1/b> <max ulp of a/b>" when the maxima are
// within 2 and 3 ulp, else "FAIL ..."; exit status 0 on success.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <cstring>
#include <vector>

#include "common.cuh"

__global__ void k_rcp(const double* a, const double* b, int n, double* r_nr, double* r_ref, double* q_nr,
                      double* q_ref) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  r_nr[i] = dsnu::rcp_nr(b[i]);
  r_ref[i] = 1.0 / b[i];
  q_nr[i] = dsnu::fdiv<double>(a[i], b[i]);
  q_ref[i] = a[i] / b[i];
}

static double ulp_diff(double x, double y) {
  int64_t ix, iy;
  std::memcpy(&ix, &x, 8);
  std::memcpy(&iy, &y, 8);
  return std::fabs(double(ix - iy));
}

int main() {
  const int n = 1 << 22;
  std::vector<double> a(n), b(n);
  uint64_t st = 0x9E3779B97F4A7C15ull;
  auto next = [&]() {  // splitmix64
    uint64_t z = (st += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  for (int i = 0; i < n; ++i) {
    const double u = double(next() >> 11) * 0x1.0p-53, v = double(next() >> 11) * 0x1.0p-53;
    b[i] = std::ldexp(1.0 + u, int(next() % 200) - 100);  // 2^-100 .. 2^100
    a[i] = std::ldexp(1.0 + v, int(next() % 60) - 30) * ((next() & 1) ? 1.0 : -1.0);
  }
  double *da, *db, *r1, *r2, *q1, *q2;
  cudaMalloc(&da, n * 8);
  cudaMalloc(&db, n * 8);
  cudaMalloc(&r1, n * 8);
  cudaMalloc(&r2, n * 8);
  cudaMalloc(&q1, n * 8);
  cudaMalloc(&q2, n * 8);
  cudaMemcpy(da, a.data(), n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(db, b.data(), n * 8, cudaMemcpyHostToDevice);
  k_rcp<<<(n + 255) / 256, 256>>>(da, db, n, r1, r2, q1, q2);
  if (cudaDeviceSynchronize() != cudaSuccess) {
    std::printf("FAIL cuda\n");
    return 1;
  }
  std::vector<double> h1(n), h2(n), h3(n), h4(n);
  cudaMemcpy(h1.data(), r1, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(h2.data(), r2, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(h3.data(), q1, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(h4.data(), q2, n * 8, cudaMemcpyDeviceToHost);
  double mr = 0, mq = 0;
  for (int i = 0; i < n; ++i) {
    mr = std::fmax(mr, ulp_diff(h1[i], h2[i]));
    mq = std::fmax(mq, ulp_diff(h3[i], h4[i]));
  }
  const bool ok = mr <= 2.0 && mq <= 3.0;
  std::printf("%s %.0f %.0f\n", ok ? "OK" : "FAIL", mr, mq);
  return ok ? 0 : 1;
}
