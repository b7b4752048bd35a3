// Accuracy of the library's FP64 reciprocal (glemur::recip, the 1/det G of
// the FP64 stages) against the IEEE quotient 1.0 / x, on n inputs given on
// the command line's seed: log-uniform over 2^-40 .. 2^40 with random
// mantissas.  Prints "n <n> max_ulp <u> differing <k>".
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "stage_kernels.cuh"

__global__ void k_recip(const double* x, double* y, double* ref, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  y[i] = glemur::recip(x[i]);
  ref[i] = 1.0 / x[i];
}

int main(int argc, char** argv) {
  const int n = argc > 1 ? atoi(argv[1]) : (1 << 22);
  const unsigned seed = argc > 2 ? (unsigned)atoi(argv[2]) : 1u;
  if (n <= 0) return 2;
  std::vector<double> h(3 * (size_t)n);
  uint64_t s = seed * 0x9E3779B97F4A7C15ull + 1;
  for (int i = 0; i < n; ++i) {  // xorshift64 mantissa bits and exponent
    s ^= s << 13;
    s ^= s >> 7;
    s ^= s << 17;
    const int ex = (int)((s >> 57) % 81) - 40;  // 2^-40 .. 2^40
    const uint64_t bits = (s & 0x000FFFFFFFFFFFFFull) | ((uint64_t)(1023 + ex) << 52);
    memcpy(&h[i], &bits, 8);
  }
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 3 * (size_t)n) != cudaSuccess) return 1;
  cudaMemcpy(d, h.data(), sizeof(double) * n, cudaMemcpyHostToDevice);
  k_recip<<<(n + 255) / 256, 256>>>(d, d + n, d + 2 * (size_t)n, n);
  if (cudaDeviceSynchronize() != cudaSuccess) return 1;
  cudaMemcpy(h.data() + n, d + n, sizeof(double) * 2 * (size_t)n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  int64_t umax = 0;
  long long differing = 0;
  for (int i = 0; i < n; ++i) {
    int64_t a, b;
    memcpy(&a, &h[(size_t)n + i], 8);
    memcpy(&b, &h[2 * (size_t)n + i], 8);
    const int64_t u = a > b ? a - b : b - a;
    umax = u > umax ? u : umax;
    differing += u != 0;
  }
  printf("n %d max_ulp %lld differing %lld\n", n, (long long)umax, differing);
  return 0;
}
