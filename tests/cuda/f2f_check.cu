// Checks dsnu::f32_of_f64_int(d) (with the hardware conversion for the values
// it flags) against __double2float_rn(d), bit for bit (NaNs compared as NaNs),
// on
//   * 2^26 seeded random 64-bit patterns (every class of double);
//   * 2^26 structured doubles: every exponent from just below FP32's
//     subnormals to just above its largest finite value, with fractions whose
//     29 dropped bits are exact ties (with an even or odd kept last bit), one
//     unit below or above a tie, all ones (a carry into the exponent, up to
//     the infinity pattern) or random; zeros of both signs, subnormal
//     doubles, infinities and NaNs.
// Prints "OK <values>" or "FAIL <index>"; exit status 0 on success.
#include <cstdio>
#include <cstdint>

#include "common.cuh"

__device__ unsigned long long mix(unsigned long long z) {  // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ double value(unsigned long long i) {
  const unsigned long long z = mix(i), w = mix(i ^ 0xD1B54A32D192ED03ull);
  if (i < (1ull << 26)) return __longlong_as_double((long long)z);  // random bit patterns
  const unsigned long long sign = z & 0x8000000000000000ull;
  // biased FP64 exponents 860 .. 1160: FP32's subnormal range up to past its largest value
  const unsigned long long e = 860ull + (z >> 20) % 301ull;
  const unsigned long long kept = (w & 0xFFFFFull) | (((w >> 20) & 7ull) << 20);  // 23 kept fraction bits
  unsigned long long drop;  // 29 dropped fraction bits
  switch (int((z >> 8) % 8u)) {
    case 0: drop = 1ull << 28; break;                          // exact tie
    case 1: drop = (1ull << 28) - 1ull; break;                  // just below a tie
    case 2: drop = (1ull << 28) + 1ull; break;                  // just above a tie
    case 3: drop = (1ull << 29) - 1ull; break;                  // all ones
    case 4: drop = 0ull; break;                                 // exact in FP32
    default: drop = (w >> 24) & ((1ull << 29) - 1ull); break;   // random
  }
  unsigned long long frac = (kept << 29) | drop;
  if (((z >> 12) & 15u) == 0) frac |= 0xFFFFFFFFFFFFFull;       // all-ones fraction: carries
  unsigned long long bits = sign | (e << 52) | frac;
  switch (int((z >> 16) % 64u)) {
    case 0: bits = sign; break;                                          // zero
    case 1: bits = sign | (w & 0xFFFFFFFFFFFFFull) | 1ull; break;        // subnormal double
    case 2: bits = sign | 0x7FF0000000000000ull; break;                  // infinity
    case 3: bits = sign | 0x7FF0000000000000ull | (w & 0xFFFFFFFFFFFFFull) | 1ull; break;  // NaN
    default: break;
  }
  return __longlong_as_double((long long)bits);
}

__global__ void k_check(unsigned long long n, unsigned long long* bad, unsigned long long* count) {
  unsigned long long c = 0;
  const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n; i += stride) {
    const double d = value(i);
    bool odd = false;
    float x = dsnu::f32_of_f64_int(d, odd);
    if (odd) x = dsnu::f32_of_f64_hw(d);
    const float y = __double2float_rn(d);
    const bool same = (y != y) ? (x != x) : (__float_as_uint(x) == __float_as_uint(y));
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
    std::printf("FAIL first bad value %llu (checked %llu)\n", h[0], h[1]);
    return 1;
  }
  std::printf("OK %llu\n", h[1]);
  return 0;
}
