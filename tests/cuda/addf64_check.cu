// Checks dsnu::add_f32_f64(a, b) against the FP64 addition double(a) +
// double(b), bit for bit (NaNs compared as NaNs), on
//   * 2^26 pairs of seeded random 32-bit patterns (every class of float);
//   * 2^26 structured pairs: a random normal a and b of either sign whose
//     exponent is a's minus 0..63 (exact sums, sums that round, cancellation),
//     b = -a (1 + tiny), powers of two a with a small remainder of the other
//     sign, subnormals, zeros, infinities and NaNs.
// Prints "OK <pairs>" or "FAIL <a bits> <b bits>"; exit status 0 on success.
#include <cstdio>
#include <cstdint>

#include "common.cuh"

__device__ unsigned long long mix(unsigned long long z) {  // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ void pair(unsigned long long i, float* pa, float* pb) {
  const unsigned long long z = mix(i), w = mix(i ^ 0xD1B54A32D192ED03ull);
  if (i < (1ull << 26)) {  // random bit patterns
    *pa = __uint_as_float(unsigned(z));
    *pb = __uint_as_float(unsigned(w));
    return;
  }
  const unsigned sa = unsigned(z) & 0x80000000u, sb = unsigned(w) & 0x80000000u;
  const unsigned ea = 1u + unsigned((z >> 32) % 254u);   // normal exponent of a
  const unsigned ma = unsigned(z >> 8) & 0x7FFFFFu, mb = unsigned(w >> 8) & 0x7FFFFFu;
  const float a = __uint_as_float(sa | (ea << 23) | ((w & 7u) == 0 ? 0u : ma));  // 1 in 8: a power of two
  const int gap = int((w >> 40) % 64u);
  const int eb = int(ea) - gap;
  float b;
  switch (int((z >> 40) % 8u)) {
    case 0:  // -a (1 + tiny)
      b = -a * (1.0f + __uint_as_float(((unsigned(w >> 48) % 30u) + 97u) << 23));
      break;
    case 1:  // subnormal b
      b = __uint_as_float(sb | (mb ? mb : 1u));
      break;
    case 2:  // zero, infinity or NaN b
      b = __uint_as_float(sb | ((w >> 52) & 1u ? 0x7F800000u | ((w >> 53) & 1u ? 0x400000u : 0u) : 0u));
      break;
    default:  // b a given number of binades below a (flushed to 0 below the subnormals)
      b = (eb >= 1) ? __uint_as_float(sb | (unsigned(eb) << 23) | mb) : __uint_as_float(sb);
      break;
  }
  *pa = a;
  *pb = b;
}

__global__ void k_check(unsigned long long n, unsigned long long* bad, unsigned long long* count) {
  unsigned long long c = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    float a, b;
    pair(i, &a, &b);
    const double x = dsnu::add_f32_f64(a, b);
    const double y = static_cast<double>(a) + static_cast<double>(b);
    const bool same = (y != y) ? (x != x) : (__double_as_longlong(x) == __double_as_longlong(y));
    if (!same) atomicMin(bad, i);
    ++c;
  }
  atomicAdd(count, c);
}

int main() {
  const unsigned long long n = 1ull << 27;
  unsigned long long *d = nullptr, h[2] = {~0ull, 0ull};
  if (cudaMalloc(&d, 2 * sizeof(unsigned long long)) != cudaSuccess) return 2;
  cudaMemcpy(d, h, sizeof(h), cudaMemcpyHostToDevice);
  k_check<<<1216, 256>>>(n, d, d + 1);
  if (cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
  cudaFree(d);
  if (h[0] != ~0ull || h[1] != n) {
    std::printf("FAIL first bad pair %llu (checked %llu)\n", h[0], h[1]);
    return 1;
  }
  std::printf("OK %llu\n", h[1]);
  return 0;
}
