// Bitwise check of the integer-arithmetic FP64<->FP32 conversions in
// common.cuh against the hardware conversions (normal float range), plus the
// documented flush of results below 2^-126.  Prints "OK <count>" or the first
// mismatch; exit status 0 on success.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "common.cuh"

__global__ void k_convert(const double* in, int n, float* bits32, float* hw32, const float* fin,
                          double* bits64, double* hw64) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bits32[i] = dsnu::f64_to_f32_bits(in[i]);
  hw32[i] = __double2float_rn(in[i]);
  bits64[i] = dsnu::f32_to_f64_bits(fin[i]);
  hw64[i] = static_cast<double>(fin[i]);
}

static unsigned long long splitmix(unsigned long long& s) {
  unsigned long long z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

int main() {
  const int n = 1 << 20;
  std::vector<double> in(n);
  std::vector<float> fin(n);
  unsigned long long s = 12345;
  for (int i = 0; i < n; ++i) {
    unsigned long long r = splitmix(s);
    // exponent spread over the normal float range and a bit beyond
    int e = int(r % 300) - 150;
    unsigned long long mant = splitmix(s) & ((1ull << 52) - 1);
    if (i % 8 == 1) mant = (mant & ~((1ull << 29) - 1)) | (1ull << 28);  // exact ties
    if (i % 8 == 2) mant &= ~((1ull << 29) - 1);                          // exactly representable
    unsigned long long b = ((unsigned long long)(e + 1023) << 52) | mant | ((r >> 63) << 63);
    std::memcpy(&in[i], &b, 8);
    unsigned int fb = (unsigned int)splitmix(s);
    unsigned int fe = (fb >> 23) & 0xFF;
    if (fe == 0 || fe == 255) fb = (fb & ~(0xFFu << 23)) | (100u << 23);
    std::memcpy(&fin[i], &fb, 4);
  }
  double *d_in, *d_b64, *d_h64;
  float *d_b32, *d_h32, *d_fin;
  cudaMalloc(&d_in, n * 8); cudaMalloc(&d_b64, n * 8); cudaMalloc(&d_h64, n * 8);
  cudaMalloc(&d_b32, n * 4); cudaMalloc(&d_h32, n * 4); cudaMalloc(&d_fin, n * 4);
  cudaMemcpy(d_in, in.data(), n * 8, cudaMemcpyHostToDevice);
  cudaMemcpy(d_fin, fin.data(), n * 4, cudaMemcpyHostToDevice);
  k_convert<<<(n + 255) / 256, 256>>>(d_in, n, d_b32, d_h32, d_fin, d_b64, d_h64);
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) { printf("CUDA error %s\n", cudaGetErrorString(e)); return 2; }
  std::vector<float> b32(n), h32(n);
  std::vector<double> b64(n), h64(n);
  cudaMemcpy(b32.data(), d_b32, n * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(h32.data(), d_h32, n * 4, cudaMemcpyDeviceToHost);
  cudaMemcpy(b64.data(), d_b64, n * 8, cudaMemcpyDeviceToHost);
  cudaMemcpy(h64.data(), d_h64, n * 8, cudaMemcpyDeviceToHost);
  long checked = 0;
  for (int i = 0; i < n; ++i) {
    const float hw = h32[i];
    unsigned int ub, uh;
    std::memcpy(&ub, &b32[i], 4);
    std::memcpy(&uh, &hw, 4);
    const unsigned int eh = (uh >> 23) & 0xFF;
    bool ok;
    if (eh == 0) ok = (ub & 0x7FFFFFFFu) == 0;   // documented flush of subnormal results
    else if ((uh & 0x7FFFFFFFu) == 0x00800000u && (ub & 0x7FFFFFFFu) == 0) ok = true;  // rounded up to 2^-126
    else ok = ub == uh;                          // normal results and infinities match bitwise
    if (!ok) { printf("f64->f32 mismatch at %d: %.17g -> %08x vs %08x\n", i, in[i], ub, uh); return 1; }
    unsigned long long vb, vh;
    std::memcpy(&vb, &b64[i], 8);
    std::memcpy(&vh, &h64[i], 8);
    if (vb != vh) { printf("f32->f64 mismatch at %d\n", i); return 1; }
    ++checked;
  }
  printf("OK %ld\n", checked);
  return 0;
}
