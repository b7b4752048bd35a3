// glemur_energy_static: the magnetic-energy reduction without any device
// allocation, for callers that cannot allocate device memory themselves --
// for example a host simulation framework that owns the whole device pool
// and forbids foreign allocations, or code that must not trigger the
// implicit device synchronisation cudaMalloc/cudaFree can cause.
//
// The per-CTA partial sums live in a file-scope static device array of
// fixed size (GLEMUR_STATIC_MAX_NODES / 256 doubles = 512 KiB), which every
// GPU that loads this library keeps until the process exits.  Every call
// shares that array: each CTA overwrites its own slot before the final sum
// reads it, so nothing has to be cleared, but calls that overlap on the GPU
// (other streams, other threads) race on it.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "glemur.h"

namespace glemur {
namespace {

constexpr int kThreads = 256;
constexpr long long kMaxBlocks = GLEMUR_STATIC_MAX_NODES / kThreads;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_energy_partials[kMaxBlocks];

// Address of g_energy_partials on each device, resolved once per device and
// context: a device address belongs to the context it was resolved in, so a
// call from another context (after cudaDeviceReset, or from a framework's
// own non-primary context) resolves it again.
std::mutex g_mutex;
double* g_scratch[kMaxDevices] = {nullptr};
CUcontext g_scratch_ctx[kMaxDevices] = {nullptr};

// cuCtxGetCurrent through the runtime's driver entry point (no link against
// the driver library); null if the driver does not provide it.
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn ctx_get_current() {
  static CtxGetCurrentFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (CtxGetCurrentFn)p;
  }
  return fn;
}

struct Geom {
  int nx, ny, nz;
  double h[3];
};

// x at node (i, j, k), component c.
__device__ __forceinline__ double xat(const double* x, long long N, const Geom& g, int c, int i,
                                      int j, int k) {
  return x[c * N + ((long long)k * g.ny + j) * g.nx + i];
}

// Column b of dx/dX at node (i, j, k): central differences inside,
// second-order one-sided on the boundary faces.
__device__ __forceinline__ void jac_col(const double* x, long long N, const Geom& g, int b, int i,
                                        int j, int k, double F[3]) {
  const int id[3] = {i, j, k};
  const int n[3] = {g.nx, g.ny, g.nz};
  int p0[3] = {i, j, k}, p1[3] = {i, j, k}, p2[3] = {i, j, k};
  double w0, w1, w2;
  if (id[b] > 0 && id[b] < n[b] - 1) {
    p0[b] -= 1; p1[b] += 1; w0 = -1.0; w1 = 1.0; w2 = 0.0;
  } else if (id[b] == 0) {
    p1[b] = 1; p2[b] = 2; w0 = -3.0; w1 = 4.0; w2 = -1.0;
  } else {
    p1[b] = n[b] - 2; p2[b] = n[b] - 3; w0 = 3.0; w1 = -4.0; w2 = 1.0;
  }
  for (int c = 0; c < 3; ++c)
    F[c] = (w0 * xat(x, N, g, c, p0[0], p0[1], p0[2]) + w1 * xat(x, N, g, c, p1[0], p1[1], p1[2]) +
            w2 * xat(x, N, g, c, p2[0], p2[1], p2[2])) /
           (2.0 * g.h[b]);
}

// zeta B^2 Delta at every node (eq. "magnetic energy", B from eq. "B
// transformation"), one node per thread; one partial sum per CTA.
__global__ void __launch_bounds__(kThreads) k_energy_partials(Geom g, const double* __restrict__ x,
                                                              const double* __restrict__ B0,
                                                              double* partials) {
  const long long N = (long long)g.nx * g.ny * g.nz;
  const long long n = (long long)blockIdx.x * kThreads + threadIdx.x;
  double w = 0.0;
  if (n < N) {
    const int i = (int)(n % g.nx), j = (int)((n / g.nx) % g.ny), k = (int)(n / ((long long)g.nx * g.ny));
    double F0[3], F1[3], F2[3];
    jac_col(x, N, g, 0, i, j, k, F0);
    jac_col(x, N, g, 1, i, j, k, F1);
    jac_col(x, N, g, 2, i, j, k, F2);
    const double D = F0[0] * (F1[1] * F2[2] - F1[2] * F2[1]) +
                     F0[1] * (F1[2] * F2[0] - F1[0] * F2[2]) +
                     F0[2] * (F1[0] * F2[1] - F1[1] * F2[0]);
    const double b0 = B0[n], b1 = B0[N + n], b2 = B0[2 * N + n];
    double B2 = 0.0;
    for (int c = 0; c < 3; ++c) {
      const double Bc = (F0[c] * b0 + F1[c] * b1 + F2[c] * b2) / D;
      B2 += Bc * Bc;
    }
    double zeta = 1.0;
    if (i == 0 || i == g.nx - 1) zeta *= 0.5;
    if (j == 0 || j == g.ny - 1) zeta *= 0.5;
    if (k == 0 || k == g.nz - 1) zeta *= 0.5;
    w = zeta * B2 * D;
  }
  __shared__ double sh[kThreads / 32];
  for (int o = 16; o > 0; o >>= 1) w += __shfl_xor_sync(0xffffffffu, w, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = w;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) s += sh[q];
    partials[blockIdx.x] = s;
  }
}

// Fixed-order sum of the partials into *E (deterministic).
__global__ void k_energy_finalize(const double* partials, long long nb, double scale, double* E) {
  __shared__ double sh[kThreads / 32];
  double s = 0.0;
  for (long long b = threadIdx.x; b < nb; b += kThreads) s += partials[b];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += sh[q];
    *E = scale * t;
  }
}

// Resolve the static scratch's device address for the current device and
// context (cudaGetSymbolAddress with that device current).
int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return GLEMUR_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return GLEMUR_ERR_BADARG;
  CtxGetCurrentFn get_ctx = ctx_get_current();
  if (!get_ctx) return GLEMUR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mutex);
  CUcontext ctx = nullptr;
  if (get_ctx(&ctx) != CUDA_SUCCESS) return GLEMUR_ERR_CUDA;
  if (!g_scratch[dev] || !ctx || ctx != g_scratch_ctx[dev]) {
    double* p = nullptr;
    if (cudaGetSymbolAddress((void**)&p, g_energy_partials) != cudaSuccess || !p)
      return GLEMUR_ERR_CUDA;
    // the runtime made its context current if there was none
    if (get_ctx(&ctx) != CUDA_SUCCESS) return GLEMUR_ERR_CUDA;
    g_scratch[dev] = p;
    g_scratch_ctx[dev] = ctx;
  }
  *out = g_scratch[dev];
  return GLEMUR_OK;
}

}  // namespace
}  // namespace glemur

extern "C" int glemur_energy_static(int nx, int ny, int nz, const double lo[3],
                                    const double hi[3], const double* x, const double* B0,
                                    double* E, void* stream) {
  using namespace glemur;
  if (!lo || !hi || !x || !B0 || !E || nx < 3 || ny < 3 || nz < 3) return GLEMUR_ERR_BADARG;
  const long long N = (long long)nx * ny * nz;
  if (N > GLEMUR_STATIC_MAX_NODES) return GLEMUR_ERR_TOO_LARGE;
  Geom g{nx, ny, nz, {0, 0, 0}};
  const int n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    if (!(hi[a] > lo[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a]))
      return GLEMUR_ERR_BADARG;
    g.h[a] = (hi[a] - lo[a]) / (n[a] - 1);
  }
  double* partials = nullptr;
  int rc = scratch_for_current_device(&partials);
  if (rc != GLEMUR_OK) return rc;
  const long long nb = (N + kThreads - 1) / kThreads;
  cudaStream_t s = (cudaStream_t)stream;
  k_energy_partials<<<(unsigned)nb, kThreads, 0, s>>>(g, x, B0, partials);
  k_energy_finalize<<<1, kThreads, 0, s>>>(partials, nb, 0.5 * g.h[0] * g.h[1] * g.h[2], E);
  return cudaGetLastError() == cudaSuccess ? GLEMUR_OK : GLEMUR_ERR_CUDA;
}
