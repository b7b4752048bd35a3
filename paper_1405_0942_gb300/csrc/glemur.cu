// Host side of the C ABI declared in include/glemur.h: context, workspace
// layout, the attempt loop with device-side step control, diagnostics and
// the layout conversions at the boundary.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include <cudaTypedefs.h>

#include "control.cuh"
#include "glemur.h"
#include "glemur_dev.cuh"
#include "tma.cuh"

namespace glemur {
cudaError_t launch_f64_mimetic(const StageArgs<double>& a, int stage, dim3 grid, cudaStream_t s);
cudaError_t launch_f64_direct(const StageArgs<double>& a, int stage, dim3 grid, cudaStream_t s);
cudaError_t launch_f32_mimetic(const StageArgs<float>& a, int stage, dim3 grid, cudaStream_t s);
cudaError_t launch_f32_direct(const StageArgs<float>& a, int stage, dim3 grid, cudaStream_t s);
cudaError_t prepare_f64_mimetic();
cudaError_t prepare_f64_direct();
cudaError_t prepare_f32_mimetic();
cudaError_t prepare_f32_direct();
int ctas_per_sm_f64_mimetic();
int ctas_per_sm_f64_direct();
int ctas_per_sm_f32_mimetic();
int ctas_per_sm_f32_direct();
cudaError_t launch_f32_mimetic_tma(const StageArgs<float>& a, const TmaMaps& maps, int stage,
                                   dim3 grid, cudaStream_t s);
cudaError_t prepare_f32_mimetic_tma();
int ctas_per_sm_f32_mimetic_tma();
int tile_rows_f32_mimetic_tma();

cudaError_t launch_f64_split(const SplitArgs& a, int stage, cudaStream_t s, int curl);
void split_ctas_per_sm(int b[6], int c[6], int curl);
int persist_ctas_per_sm(int curl);
cudaError_t launch_f64_persist(const SplitArgs& a, const PersistArgs& pa, int grid, int curl,
                               cudaStream_t s);

// dt-scaled coefficients of the pending attempt.
__device__ void set_coeffs(DevState* st) {
  const double dt = st->dt;
  for (int s = 0; s < 6; ++s) {
    for (int j = 0; j < 6; ++j) {
      st->dta[s][j] = dt * CK_A[s][j];
      st->dtaf[s][j] = (float)st->dta[s][j];
    }
    st->dtb[s] = dt * CK_B5[s];
    st->dte[s] = dt * (CK_B5[s] - CK_B4[s]);
    st->dtbf[s] = (float)st->dtb[s];
    st->dtef[s] = (float)st->dte[s];
  }
}

__global__ void k_reset_state(DevState* st, double dt0, double lambda0, double dt_min,
                              double grow_max, double shrink_min, int max_rejects,
                              double safety) {
  st->dt = dt0;
  st->dt_last = 0.0;
  st->t = 0.0;
  st->lambda = 0.0;
  st->lambda0 = lambda0;
  st->dt_min = dt_min;
  st->grow_max = grow_max;
  st->shrink_min = shrink_min;
  st->safety = safety;
  st->n_accept = 0;
  st->n_reject = 0;
  st->target = 0;
  st->consec = 0;
  st->cur = 0;
  st->status = ST_OK;
  st->flags = 0;
  st->max_rejects = max_rejects;
  st->replay = 0;
  st->E = st->xi = st->xi_sin = 0.0;
  set_coeffs(st);
}

__global__ void k_set_target(DevState* st, long long extra, int relative) {
  st->target = relative ? st->n_accept + extra : extra;
}

__global__ void k_set_dt(DevState* st, double dt, int replay) {
  st->dt = dt;
  st->replay = replay;
  st->target = st->n_accept + 1;
  set_coeffs(st);
}

__global__ void k_diag_finalize(DevState* st, const double* part, int nb) {
  __shared__ double sh[96];
  finalize_diag<LdPlain>(st, part, nb, sh);
  if (threadIdx.x == 0 && (st->flags & FLAG_TIMEOUT)) st->status = ST_TIMEOUT;
}

bool pdl_enabled() {
  static const bool on = [] {
    const char* e = getenv("GLEMUR_PDL");
    return !(e && e[0] == '0');
  }();
  return on;
}

// Eq. "time stepping" and the acceptance rule after each attempt (see
// control.cuh), as a kernel of one CTA.
__global__ void k_control(DevState* st, const double* part, int nb, int diag, double* dtlog) {
  pdl_trigger();
  pdl_wait();
  __shared__ double sh[96];
  control_block<LdPlain>(st, part, nb, diag, dtlog, sh);
}

// ---- layout conversions at the boundary (float64 SoA fields) ----------

struct GridGeom {
  int nx, ny, nz;
  double lo[3], h[3];
  int periodic;  // periodic in z (ghost planes 0 and nz-1)
};

__device__ __forceinline__ double label(const GridGeom& g, int a, int i) {
  return g.lo[a] + (double)i * g.h[a];
}

template <typename T>
// d = x - X into both displacement buffers and both stage-input buffers
// (whose boundary entries must hold the fixed boundary positions).  Grids
// hold fewer than 2^31 / 3 nodes, so 32-bit indices suffice.
__global__ void k_set_x(GridGeom g, const double* __restrict__ x, T* d0, T* d1, T* y0, T* y1) {
  const int N = g.nx * g.ny * g.nz;
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const int i = n % g.nx, r = n / g.nx, j = r % g.ny, k = r / g.ny;
    // periodic in z: a ghost plane takes its partner's displacement (the
    // ghost's position is the partner's shifted by the period)
    const int ks = g.periodic && k == 0 ? g.nz - 2 : (g.periodic && k == g.nz - 1 ? 1 : k);
    const int ns = (ks * g.ny + j) * g.nx + i;
    const double X[3] = {label(g, 0, i), label(g, 1, j), label(g, 2, ks)};
    for (int c = 0; c < 3; ++c) {
      const T v = (T)(x[c * N + ns] - X[c]);
      d0[c * N + n] = v;
      d1[c * N + n] = v;
      y0[c * N + n] = v;
      y1[c * N + n] = v;
    }
  }
}

template <typename T>
__global__ void k_get_x(GridGeom g, const T* const* dbuf, const DevState* st,
                        double* __restrict__ x) {
  const int N = g.nx * g.ny * g.nz;
  const T* d = dbuf[st->cur];
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x) {
    const int i = n % g.nx, r = n / g.nx, j = r % g.ny, k = r / g.ny;
    const double X[3] = {label(g, 0, i), label(g, 1, j), label(g, 2, k)};
    for (int c = 0; c < 3; ++c) x[c * N + n] = X[c] + (double)d[c * N + n];
  }
}

template <typename T>
__global__ void k_set_B0(GridGeom g, const double* __restrict__ B0, T* B0s) {
  const int N = g.nx * g.ny * g.nz;
  // B0s_a = B0_a * 4 h_{a+1} h_{a+2}
  const double s[3] = {4.0 * g.h[1] * g.h[2], 4.0 * g.h[2] * g.h[0], 4.0 * g.h[0] * g.h[1]};
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < N; n += gridDim.x * blockDim.x)
    for (int c = 0; c < 3; ++c) B0s[c * N + n] = (T)(B0[c * N + n] * s[c]);
}

template <typename T>
__global__ void k_to_f64(long long M, const T* __restrict__ src, double* __restrict__ dst) {
  for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < M;
       n += (long long)gridDim.x * blockDim.x)
    dst[n] = (double)src[n];
}

}  // namespace glemur

using namespace glemur;

struct glemur_ctx {
  int nx, ny, nz;
  long long N;
  double lo[3], hi[3], h[3];
  glemur_opts o;
  cudaStream_t s;
  unsigned char* ws;
  size_t ws_bytes;
  size_t esize;     // bytes per stored scalar (8 or 4)
  void* dbuf[2];
  void** dbuf_dev;  // device copy of {dbuf[0], dbuf[1]}
  void* B0s;
  void* k[5];
  double* stage;    // 3N doubles for host transfers
  double* part;     // NPART * max_blocks
  DevState* st;
  double* dtlog;    // ring of GLEMUR_DT_LOG accepted step sizes
  int split;                             // FP64 mimetic stages in two passes
  int tma;                               // mixed mimetic stages with TMA tiles
  int tma_test;                          // test hook: unsatisfiable tile wait
  TmaMaps maps;                          // their tensor maps
  void* ys[2];                           // mimetic stages: stage inputs y_1..y_5
  double* Bb;                            // split path: B
  double* Gb;                            // split path: g_0, g_1, g_2
  int max_blocks, nblocks, kz;          // mimetic-current launches
  int split_grid_b[6] = {}, split_grid_c[6] = {};  // FP64 two-pass grids (CTAs)
  int persist;                           // whole attempts in one persistent launch
  int persist_grid;                      // its CTAs (all resident)
  PersistArgs pa;                        // its plan and counters (workspace)
  int* persist_base;                     // counters to zero before each launch
  size_t persist_zero_bytes;
  int nblocks_direct, kz_direct;         // direct-current launches
  dim3 grid, grid_direct;
  int nsm;
  int target_unbounded;                  // the device's step target is LLONG_MAX
};

namespace {

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

constexpr int PERSIST_MAX_CTAS = 16384;

struct Layout {
  size_t field, stage, part, state, ptrs, dtlog, persist, split, total;
  int max_blocks;
};

// Kernels index the three components of a field with 32-bit ints.
bool valid_dims(int nx, int ny, int nz) {
  return nx >= 3 && ny >= 3 && nz >= 3 && 3LL * nx * ny * nz < (1LL << 31);
}

Layout layout(int nx, int ny, int nz, int precision) {
  Layout L{};
  const long long N = (long long)nx * ny * nz;
  const size_t es = precision == GLEMUR_MIXED ? 4 : 8;
  L.field = align256((size_t)(3 * N) * es);
  L.stage = align256((size_t)(3 * N) * sizeof(double));
  const long long gx = (nx + TX - 1) / TX, gy = (ny + TY - 1) / TY;
  L.max_blocks = (int)(gx * gy * nz);
  L.part = align256((size_t)NPART * L.max_blocks * sizeof(double));
  L.state = align256(sizeof(DevState));
  L.ptrs = 256;
  L.dtlog = align256((size_t)GLEMUR_DT_LOG * sizeof(double));
  // persistent FP64 attempts: counters and touches per plane (4 nz ints),
  // the barrier, and the plan of up to PERSIST_MAX_CTAS CTAs
  L.persist = precision == GLEMUR_FP64
                  ? align256(sizeof(int) * (4 * (size_t)nz + 64 +
                                            (size_t)PERSIST_MAX_CTAS * (2 * PERSIST_BI + 2)))
                  : 0;
  // two stage inputs (mimetic stages); FP64 also B and the node records
  // (differences and 1/det G) of the two-pass stages
  L.split = 2 * L.field + (precision == GLEMUR_FP64 ? align256((size_t)(3 * N) * 8) +
                                                          align256((size_t)(10 * N) * 8)
                                                    : 0);
  L.total = 8 * L.field + L.stage + L.part + L.state + L.ptrs + L.dtlog + L.persist + L.split;
  return L;
}

int cuda_rc(cudaError_t e) { return e == cudaSuccess ? GLEMUR_OK : GLEMUR_ERR_CUDA; }

// Node range [begin, end) of CTA b of G over n items in whole warps, as the
// two-pass kernels' cta_range computes it on the device.
void host_cta_range(long long n, int b, int G, long long& begin, long long& end) {
  const long long W = (n + 31) / 32;
  const long long w0 = W * b / G, w1 = W * (b + 1) / G;
  begin = w0 * 32;
  end = w1 * 32 < n ? w1 * 32 : n;
}

// Plane of boundary item t, in the order of the kernels' boundary_node:
// the inner parts of the z, y and x faces, the edges along x, y and z, the
// corners.
int host_boundary_plane(int nx, int ny, int nz, long long t) {
  const long long xi = nx - 2, yi = ny - 2, zi = nz - 2;
  const long long fz = xi * yi, fy = xi * zi, fx = yi * zi;
  if (t < 2 * fz) return t < fz ? 0 : nz - 1;
  t -= 2 * fz;
  if (t < 2 * fy) return 1 + (int)((t < fy ? t : t - fy) / xi);
  t -= 2 * fy;
  if (t < 2 * fx) return 1 + (int)((t < fx ? t : t - fx) / yi);
  t -= 2 * fx;
  if (t < 4 * xi) return ((t / xi) & 2) ? nz - 1 : 0;
  t -= 4 * xi;
  if (t < 4 * yi) return ((t / yi) & 2) ? nz - 1 : 0;
  t -= 4 * yi;
  if (t < 4 * zi) return 1 + (int)(t % zi);
  t -= 4 * zi;
  return (t & 4) ? nz - 1 : 0;
}

// The persistent kernel's plan: per CTA the plane intervals of its pass-B
// work (the interior range, then the planes of its boundary range as runs
// of adjacent planes, at most PERSIST_BI - 1 of them: the last run absorbs
// any further planes, a superset that only widens the waits) and of its
// pass-C work (the interior range); per plane how many CTAs' intervals
// contain it.  False if the plan does not fit.
bool persist_plan(glemur_ctx* c, int G) {
  const int nx = c->nx, ny = c->ny, nz = c->nz;
  if (G < 1 || G > PERSIST_MAX_CTAS) return false;
  const long long N = c->N, NI = (long long)(nx - 2) * (ny - 2) * (nz - 2);
  const long long A = (long long)(nx - 2) * (ny - 2);
  int* h = new (std::nothrow) int[4 * (size_t)nz + 64 + (size_t)G * (2 * PERSIST_BI + 2)];
  if (!h) return false;
  // h[0, 2 nz): the completion counters, zeroed per launch
  int* touchB = h + 2 * nz;
  int* touchC = h + 3 * nz;
  int* ivB = h + 4 * nz + 64;
  int* ivC = ivB + (size_t)G * 2 * PERSIST_BI;
  for (int i = 0; i < 4 * nz + 64; ++i) h[i] = 0;
  for (int b = 0; b < G; ++b) {
    int* vb = ivB + (size_t)b * 2 * PERSIST_BI;
    for (int q = 0; q < PERSIST_BI; ++q) {
      vb[2 * q] = 1;
      vb[2 * q + 1] = 0;  // empty
    }
    long long t0, t1;
    host_cta_range(NI, b, G, t0, t1);
    int* vc = ivC + 2 * b;
    vc[0] = 1;
    vc[1] = 0;
    if (t1 > t0) {
      vc[0] = vb[0] = 1 + (int)(t0 / A);
      vc[1] = vb[1] = 1 + (int)((t1 - 1) / A);
    }
    host_cta_range(N - NI, b, G, t0, t1);
    int q = 1;
    for (long long t = t0; t < t1; ++t) {
      const int pl = host_boundary_plane(nx, ny, nz, t);
      if (q > 1) {
        int& lo = vb[2 * (q - 1)];
        int& hi = vb[2 * (q - 1) + 1];
        if ((pl >= lo - 1 && pl <= hi + 1) || q == PERSIST_BI) {
          lo = pl < lo ? pl : lo;
          hi = pl > hi ? pl : hi;
          continue;
        }
      }
      vb[2 * q] = vb[2 * q + 1] = pl;
      ++q;
    }
    for (int qq = 0; qq < PERSIST_BI; ++qq)
      for (int pl = vb[2 * qq]; pl <= vb[2 * qq + 1]; ++pl) ++touchB[pl];
    for (int pl = vc[0]; pl <= vc[1]; ++pl) ++touchC[pl];
  }
  const size_t bytes = sizeof(int) * (4 * (size_t)nz + 64 + (size_t)G * (2 * PERSIST_BI + 2));
  cudaError_t e = cudaMemcpyAsync(c->persist_base, h, bytes, cudaMemcpyHostToDevice, c->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  delete[] h;
  if (e != cudaSuccess) return false;
  int* d = c->persist_base;
  c->pa.cntB = d;
  c->pa.cntC = d + nz;
  c->pa.touchB = d + 2 * nz;
  c->pa.touchC = d + 3 * nz;
  c->pa.bar = (unsigned*)(d + 4 * nz);
  c->pa.ivB = d + 4 * nz + 64;
  c->pa.ivC = c->pa.ivB + (size_t)G * 2 * PERSIST_BI;
  c->pa.dtlog = c->dtlog;
  c->pa.n_attempts = 0;
  // GLEMUR_TEST_PERSIST_TIMEOUT=1: one CTA withholds a pass's completion so
  // that the bounded waits give up (the attempt ends with TIMEOUT, no fault)
  const char* tp = getenv("GLEMUR_TEST_PERSIST_TIMEOUT");
  c->pa.test_withhold = tp && atoi(tp) == 1 ? G / 2 : -1;
  c->persist_grid = G;
  c->persist_zero_bytes = sizeof(int) * (4 * (size_t)nz + 64);
  return true;
}

GridGeom geom(const glemur_ctx* c) {
  GridGeom g;
  g.nx = c->nx;
  g.ny = c->ny;
  g.nz = c->nz;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = c->lo[a];
    g.h[a] = c->h[a];
  }
  g.periodic = c->o.periodic_z;
  return g;
}

int elementwise_blocks(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

// Planes per CTA along z.  Cost model: the time of the busiest SM, in units
// of one B plane (a CTA of kz planes computes kz + 2 B planes).  FP64 stages
// are bound by the SM's FP64 pipe, which co-resident CTAs share, so an SM's
// time is its CTA count x (kz + 2); the FP32 stages are latency-bound, so
// up to `per_sm` co-resident CTAs overlap and the time is waves x (kz + 2).
int choose_kz(int nz, int gxy, int nsm, int per_sm, bool shared_pipe) {
  const char* env = getenv("GLEMUR_KZ");
  if (env && atoi(env) > 0) return atoi(env) < nz ? atoi(env) : nz;
  if (nsm < 1) nsm = 1;
  if (per_sm < 1) per_sm = 1;
  int best = nz;
  double best_cost = 1e300;
  for (int kz = 1; kz <= nz; ++kz) {
    const long long ctas = (long long)gxy * ((nz + kz - 1) / kz);
    const long long slots = shared_pipe ? nsm : (long long)nsm * per_sm;
    const double waves = (double)((ctas + slots - 1) / slots);
    const double cost = waves * (kz + 2);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = kz;
    }
  }
  return best;
}

template <typename T>
StageArgs<T> make_args(const glemur_ctx* c, int stage, int diag, int force) {
  StageArgs<T> a;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  a.kz = c->kz;
  for (int i = 0; i < 3; ++i) {
    a.h2[i] = 2.0 * c->h[i];
    a.h2f[i] = (float)a.h2[i];
  }
  a.d[0] = (const T*)c->dbuf[0];
  a.d[1] = (const T*)c->dbuf[1];
  a.B0s = (const T*)c->B0s;
  for (int j = 0; j < 5; ++j) a.k[j] = (T*)c->k[j];
  a.k6 = nullptr;
  a.ys[0] = (T*)c->ys[0];
  a.ys[1] = (T*)c->ys[1];
  a.stage = stage;
  a.diag = diag;
  a.force = force;
  a.st = c->st;
  a.part = c->part;
  a.nblocks = c->nblocks;
  a.tma_test = c->tma_test;
  return a;
}

int nblocks_of(const glemur_ctx* c, int curl) {
  return curl == GLEMUR_CURL_DIRECT ? c->nblocks_direct : c->nblocks;
}

cudaError_t launch_split(const glemur_ctx* c, int stage, int diag, int force, void* k6,
                         int curl) {
  SplitArgs a;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  for (int i = 0; i < 3; ++i) a.h2[i] = 2.0 * c->h[i];
  a.d[0] = (const double*)c->dbuf[0];
  a.d[1] = (const double*)c->dbuf[1];
  a.B0s = (const double*)c->B0s;
  for (int j = 0; j < 5; ++j) a.k[j] = (double*)c->k[j];
  a.k[5] = (double*)k6;
  a.ys[0] = (double*)c->ys[0];
  a.ys[1] = (double*)c->ys[1];
  a.Bb = c->Bb;
  a.rb = nullptr;  // pass C reads 1/det G with the differences in Gb
  a.Gb = c->Gb;
  a.diag = diag;
  a.force = force;
  a.periodic = c->o.periodic_z;
  a.st = c->st;
  a.part = c->part;
  a.nblocks = c->nblocks;
  for (int j = 0; j < 6; ++j) {
    a.grid_b[j] = c->split_grid_b[j];
    a.grid_c[j] = c->split_grid_c[j];
  }
  return launch_f64_split(a, stage, c->s, curl == GLEMUR_CURL_NNN ? 2 : 0);
}

cudaError_t launch_stage(const glemur_ctx* c, int curl, int stage, int diag, int force,
                         void* k6 = nullptr) {
  if (c->split && curl != GLEMUR_CURL_DIRECT)
    return launch_split(c, stage, diag, force, k6, curl);
  if (curl == GLEMUR_CURL_NNN) return cudaErrorInvalidValue;  // FP64 two-pass only
  const dim3 g = curl == GLEMUR_CURL_DIRECT ? c->grid_direct : c->grid;
  if (c->o.precision == GLEMUR_MIXED) {
    StageArgs<float> a = make_args<float>(c, stage, diag, force);
    a.k6 = (float*)k6;
    if (curl == GLEMUR_CURL_DIRECT) {
      a.kz = c->kz_direct;
      a.nblocks = c->nblocks_direct;
      return launch_f32_direct(a, stage, g, c->s);
    }
    if (c->tma) return launch_f32_mimetic_tma(a, c->maps, stage, g, c->s);
    return launch_f32_mimetic(a, stage, g, c->s);
  }
  StageArgs<double> a = make_args<double>(c, stage, diag, force);
  a.k6 = (double*)k6;
  if (curl == GLEMUR_CURL_DIRECT) {
    a.kz = c->kz_direct;
    a.nblocks = c->nblocks_direct;
    return launch_f64_direct(a, stage, g, c->s);
  }
  return launch_f64_mimetic(a, stage, g, c->s);
}

// n attempts in one persistent launch: the plane counters and the barrier
// start from zero (the per-plane touch counts after them are kept).
cudaError_t launch_attempts_persist(const glemur_ctx* c, int n) {
  SplitArgs a;
  a.nx = c->nx;
  a.ny = c->ny;
  a.nz = c->nz;
  for (int i = 0; i < 3; ++i) a.h2[i] = 2.0 * c->h[i];
  a.d[0] = (const double*)c->dbuf[0];
  a.d[1] = (const double*)c->dbuf[1];
  a.B0s = (const double*)c->B0s;
  for (int j = 0; j < 5; ++j) a.k[j] = (double*)c->k[j];
  a.k[5] = nullptr;
  a.ys[0] = (double*)c->ys[0];
  a.ys[1] = (double*)c->ys[1];
  a.Bb = c->Bb;
  a.rb = nullptr;
  a.Gb = c->Gb;
  a.diag = c->o.diag_each_attempt ? 1 : 0;
  a.force = 0;
  a.periodic = 0;
  a.st = c->st;
  a.part = c->part;
  a.nblocks = c->nblocks;
  for (int j = 0; j < 6; ++j) a.grid_b[j] = a.grid_c[j] = c->persist_grid;
  PersistArgs pa = c->pa;
  pa.n_attempts = n;
  // counters (2 nz ints) and the barrier (at 4 nz ints) start at zero
  cudaError_t e = cudaMemsetAsync(c->persist_base, 0, sizeof(int) * 2 * c->nz, c->s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(c->persist_base + 4 * c->nz, 0, sizeof(int) * 64, c->s);
  if (e == cudaSuccess)
    e = launch_f64_persist(a, pa, c->persist_grid, c->o.curl == GLEMUR_CURL_NNN ? 2 : 0, c->s);
  return e;
}

cudaError_t launch_attempt(const glemur_ctx* c) {
  const int diag = c->o.diag_each_attempt ? 1 : 0;
  for (int s = 0; s < 6; ++s) {
    cudaError_t e = launch_stage(c, c->o.curl, s, s == 0 ? diag : 0, 0);
    if (e != cudaSuccess) return e;
  }
  return launch_pdl(k_control, dim3(1), dim3(256), 0, c->s, c->st, (const double*)c->part,
                    nblocks_of(c, c->o.curl), diag, c->dtlog);
}

// n attempts: one persistent launch where the context uses it, else the
// per-pass kernels attempt by attempt.
cudaError_t launch_attempts(const glemur_ctx* c, long long n) {
  if (n <= 0) return cudaSuccess;
  if (c->persist) {
    // counters reach touch x 6 x attempts (touch <= PERSIST_MAX_CTAS): at
    // most 16384 attempts per launch keep them within 32 bits
    while (n > 0) {
      const int m = n > 16384 ? 16384 : (int)n;
      cudaError_t e = launch_attempts_persist(c, m);
      if (e != cudaSuccess) return e;
      n -= m;
    }
    return cudaSuccess;
  }
  for (long long i = 0; i < n; ++i) {
    cudaError_t e = launch_attempt(c);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int read_state(glemur_ctx* c, DevState* hs) {
  cudaError_t e = cudaMemcpyAsync(hs, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, c->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  return cuda_rc(e);
}

void fill_stats(const DevState& hs, int curl, glemur_stats* out) {
  if (!out) return;
  out->accepted = hs.n_accept;
  out->rejected = hs.n_reject;
  out->t = hs.t;
  out->dt = hs.dt;
  out->lambda = hs.lambda;
  // the direct-current kernel visits interior nodes only: no per-attempt E_M
  out->energy = curl == GLEMUR_CURL_DIRECT ? NAN : hs.E;
  out->xi = hs.xi;
  out->xi_sin = hs.xi_sin;
  out->status = hs.status;
  out->dt_last = hs.dt_last;
}

// The mimetic stages write stage inputs at interior nodes only; the
// boundary entries must hold the (fixed) boundary positions.
int seed_stage_inputs(glemur_ctx* c) {
  if (!c->ys[0]) return GLEMUR_OK;
  const size_t n = c->esize * 3 * c->N;
  cudaError_t e = cudaMemcpyAsync(c->ys[0], c->dbuf[0], n, cudaMemcpyDeviceToDevice, c->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->ys[1], c->dbuf[0], n, cudaMemcpyDeviceToDevice, c->s);
  return cuda_rc(e);
}

int reset_state(glemur_ctx* c) {
  c->target_unbounded = 0;
  k_reset_state<<<1, 1, 0, c->s>>>(c->st, c->o.dt0, c->o.lambda0, c->o.dt_min, c->o.grow_max,
                                   c->o.shrink_min, c->o.max_rejects, c->o.safety);
  return cuda_rc(cudaGetLastError());
}

// Source pointer of an input field: the caller's device pointer, or the
// staging buffer after an H2D copy.
// The device's address of a page-locked host buffer (mapped into the
// device address space), else null: the conversion kernels then read and
// write it in place over the host link instead of through a staging copy.
double* mapped_host(const void* p) {
  if (getenv("GLEMUR_HOST_STAGING")) return nullptr;
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();  // not a pointer the runtime knows: pageable memory
    return nullptr;
  }
  return at.type == cudaMemoryTypeHost ? (double*)at.devicePointer : nullptr;
}

int stage_in(glemur_ctx* c, const double* src, int mem, const double** dev) {
  if (!src) return GLEMUR_ERR_BADARG;
  if (mem == GLEMUR_MEM_DEVICE) {
    *dev = src;
    return GLEMUR_OK;
  }
  if (mem != GLEMUR_MEM_HOST) return GLEMUR_ERR_BADARG;
  if (const double* m = mapped_host(src)) {
    *dev = m;
    return GLEMUR_OK;
  }
  cudaError_t e = cudaMemcpyAsync(c->stage, src, sizeof(double) * 3 * c->N,
                                  cudaMemcpyHostToDevice, c->s);
  *dev = c->stage;
  return cuda_rc(e);
}

// Where a conversion kernel writes a host-bound result: the caller's buffer
// (device memory, or page-locked host memory mapped into the device), else
// the staging buffer that stage_out copies from.
double* out_target(glemur_ctx* c, double* dst, int mem) {
  if (mem == GLEMUR_MEM_DEVICE) return dst;
  double* m = mapped_host(dst);
  return m ? m : c->stage;
}

int stage_out(glemur_ctx* c, double* dst, double* written, int mem) {
  if (mem == GLEMUR_MEM_DEVICE) return GLEMUR_OK;
  cudaError_t e = cudaSuccess;
  if (written == c->stage)
    e = cudaMemcpyAsync(dst, c->stage, sizeof(double) * 3 * c->N, cudaMemcpyDeviceToHost, c->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  return cuda_rc(e);
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link
// against the driver library); null if the driver does not provide it.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

// 4-D map (x, y, z, component) of an FP32 SoA field with boxes of
// YW x box_h x 1 x 3; out-of-range elements read as zero.
bool encode_field_map(PFN_cuTensorMapEncodeTiled_v12000 enc, CUtensorMap* m, void* base,
                      int nx, int ny, int nz, int box_h) {
  const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, 3};
  const cuuint64_t strides[3] = {(cuuint64_t)nx * 4, (cuuint64_t)nx * ny * 4,
                                 (cuuint64_t)nx * ny * nz * 4};
  const cuuint32_t box[4] = {(cuuint32_t)YW, (cuuint32_t)box_h, 1, 3};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
             CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// TMA tiles for the mixed mimetic stages: rows 16-byte aligned (nx a
// multiple of 4) and a grid at least one box wide and high (box heights:
// tile height + 4 for the stage input, + 2 for B0).
bool setup_tma(glemur_ctx* c) {
  const int th = tile_rows_f32_mimetic_tma();
  if (c->o.precision != GLEMUR_MIXED || c->nx % 4 || c->nx < YW || c->ny < th + 4) return false;
  const char* env = getenv("GLEMUR_TMA");
  if (env && atoi(env) == 0) return false;
  PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
  if (!enc) return false;
  bool ok = true;
  for (int i = 0; i < 2 && ok; ++i)
    ok = encode_field_map(enc, &c->maps.d[i], c->dbuf[i], c->nx, c->ny, c->nz, th + 4) &&
         encode_field_map(enc, &c->maps.ys[i], c->ys[i], c->nx, c->ny, c->nz, th + 4);
  return ok && encode_field_map(enc, &c->maps.b0, c->B0s, c->nx, c->ny, c->nz, th + 2);
}

}  // namespace

namespace glemur {

// Stage derivatives k1..k6 of one attempt of size dt at the current state,
// without advancing it (k6 into `k6`); used by the adjoint's recompute.
// Leaves dt as the pending step size.
int ctx_recompute_stages(glemur_ctx* c, double dt, void* k6) {
  if (c->o.curl != GLEMUR_CURL_MIMETIC) return GLEMUR_ERR_BADARG;
  c->target_unbounded = 0;
  k_set_dt<<<1, 1, 0, c->s>>>(c->st, dt, 0);
  cudaError_t e = cudaGetLastError();
  for (int s = 0; s < 6 && e == cudaSuccess; ++s)
    e = launch_stage(c, GLEMUR_CURL_MIMETIC, s, 0, 1, s == 5 ? k6 : nullptr);
  return cuda_rc(e);
}

// The same recompute for FP64 two-pass contexts, keeping every stage's
// data for the adjoint: stage s writes B and 1/det G into BS[s], RS[s]
// (3N and N doubles) and its next input y_{s+1} into yS[s+1] (3N doubles;
// the caller has put the boundary positions in yS[1..5]); y_0 is the state
// itself.  BADARG for other contexts (the caller then recomputes stage data
// itself).
int ctx_recompute_stages_saved(glemur_ctx* c, double dt, void* k6, double* const* yS,
                               double* const* BS, double* const* RS) {
  if (c->o.curl != GLEMUR_CURL_MIMETIC || !c->split) return GLEMUR_ERR_BADARG;
  c->target_unbounded = 0;
  k_set_dt<<<1, 1, 0, c->s>>>(c->st, dt, 0);
  cudaError_t e = cudaGetLastError();
  for (int s = 0; s < 6 && e == cudaSuccess; ++s) {
    SplitArgs a;
    a.nx = c->nx;
    a.ny = c->ny;
    a.nz = c->nz;
    for (int i = 0; i < 3; ++i) a.h2[i] = 2.0 * c->h[i];
    a.d[0] = (const double*)c->dbuf[0];
    a.d[1] = (const double*)c->dbuf[1];
    a.B0s = (const double*)c->B0s;
    for (int j = 0; j < 5; ++j) a.k[j] = (double*)c->k[j];
    a.k[5] = s == 5 ? (double*)k6 : nullptr;
    a.ys[0] = a.ys[1] = nullptr;
    if (s >= 1) a.ys[s & 1] = yS[s];
    if (s < 5) a.ys[(s + 1) & 1] = yS[s + 1];
    a.Bb = BS[s];
    a.rb = RS[s];
    a.Gb = c->Gb;
    a.diag = 0;
    a.force = 1;
    a.periodic = 0;  // the adjoint refuses periodic contexts (ctx_info)
    a.st = c->st;
    a.part = c->part;
    a.nblocks = c->nblocks;
    for (int j = 0; j < 6; ++j) {
      a.grid_b[j] = c->split_grid_b[j];
      a.grid_c[j] = c->split_grid_c[j];
    }
    e = launch_f64_split(a, s, c->s, 0);
  }
  return cuda_rc(e);
}

// Geometry, storage and the current accepted displacement (synchronises).
int ctx_info(glemur_ctx* c, int* nx, int* ny, int* nz, double h[3], int* precision,
             void** d_cur, void** B0s, void** k, void** stream) {
  if (c->o.periodic_z) return GLEMUR_ERR_BADARG;  // no adjoint of the periodic step
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  if (hs.status != ST_OK) return hs.status;
  *nx = c->nx;
  *ny = c->ny;
  *nz = c->nz;
  for (int a = 0; a < 3; ++a) h[a] = c->h[a];
  *precision = c->o.precision;
  *d_cur = c->dbuf[hs.cur];
  *B0s = c->B0s;
  for (int j = 0; j < 5; ++j) k[j] = c->k[j];
  *stream = (void*)c->s;
  return GLEMUR_OK;
}

int ctx_diag(glemur_ctx* c, DiagCtx* o) {
  o->nx = c->nx;
  o->ny = c->ny;
  o->nz = c->nz;
  for (int a = 0; a < 3; ++a) {
    o->lo[a] = c->lo[a];
    o->h[a] = c->h[a];
  }
  o->precision = c->o.precision;
  o->curl = c->o.curl;
  o->periodic = c->o.periodic_z;
  o->dbuf_dev = (const void* const*)c->dbuf_dev;
  o->B0s = c->B0s;
  o->st = c->st;
  o->part = c->part;
  o->max_blocks = c->max_blocks;
  o->stage = c->stage;
  o->s = c->s;
  return GLEMUR_OK;
}

}  // namespace glemur

extern "C" {

void glemur_default_opts(glemur_opts* o) {
  if (!o) return;
  o->precision = GLEMUR_FP64;
  o->curl = GLEMUR_CURL_MIMETIC;
  o->lambda0 = 1e-7;
  o->dt0 = 1e-3;
  o->dt_min = 1e-14;
  o->grow_max = 5.0;
  o->shrink_min = 0.1;
  o->max_rejects = 64;
  o->diag_each_attempt = 1;
  o->safety = 1.0;
  o->periodic_z = 0;
}

size_t glemur_workspace_bytes(int nx, int ny, int nz, int precision) {
  if (!valid_dims(nx, ny, nz)) return 0;
  if (precision != GLEMUR_FP64 && precision != GLEMUR_MIXED) return 0;
  return layout(nx, ny, nz, precision).total;
}

int glemur_init_grid(glemur_ctx** out, int nx, int ny, int nz, const double lo[3],
                     const double hi[3], const glemur_opts* opts, void* stream,
                     void* workspace, size_t ws_bytes) {
  if (!out || !lo || !hi || !valid_dims(nx, ny, nz)) return GLEMUR_ERR_BADARG;
  *out = nullptr;
  glemur_opts o;
  glemur_default_opts(&o);
  if (opts) o = *opts;
  if ((o.precision != GLEMUR_FP64 && o.precision != GLEMUR_MIXED) ||
      (o.curl != GLEMUR_CURL_MIMETIC && o.curl != GLEMUR_CURL_DIRECT &&
       o.curl != GLEMUR_CURL_NNN) ||
      (o.curl == GLEMUR_CURL_NNN && o.precision != GLEMUR_FP64) ||
      (o.periodic_z != 0 && o.periodic_z != 1) ||
      (o.periodic_z && (o.precision != GLEMUR_FP64 || o.curl == GLEMUR_CURL_DIRECT)) ||
      !(o.lambda0 > 0) || !(o.dt0 > 0) || !(o.dt_min >= 0) || !(o.grow_max >= 1) ||
      !(o.shrink_min > 0 && o.shrink_min <= 1) || o.max_rejects < 0 ||
      !(o.safety > 0 && o.safety <= 1))
    return GLEMUR_ERR_BADARG;
  for (int a = 0; a < 3; ++a)
    if (!(hi[a] > lo[a]) || !std::isfinite(lo[a]) || !std::isfinite(hi[a]))
      return GLEMUR_ERR_BADARG;
  const Layout L = layout(nx, ny, nz, o.precision);
  if (!workspace || ws_bytes < L.total || ((uintptr_t)workspace & 255))
    return GLEMUR_ERR_WORKSPACE;
  glemur_ctx* c = new (std::nothrow) glemur_ctx();
  if (!c) return GLEMUR_ERR_BADARG;
  c->nx = nx;
  c->ny = ny;
  c->nz = nz;
  c->N = (long long)nx * ny * nz;
  const int n[3] = {nx, ny, nz};
  for (int a = 0; a < 3; ++a) {
    c->lo[a] = lo[a];
    c->hi[a] = hi[a];
    c->h[a] = (hi[a] - lo[a]) / (n[a] - 1);
  }
  c->o = o;
  c->s = (cudaStream_t)stream;
  c->ws = (unsigned char*)workspace;
  c->ws_bytes = ws_bytes;
  c->esize = o.precision == GLEMUR_MIXED ? 4 : 8;
  unsigned char* p = c->ws;
  c->dbuf[0] = p; p += L.field;
  c->dbuf[1] = p; p += L.field;
  c->B0s = p; p += L.field;
  for (int j = 0; j < 5; ++j) { c->k[j] = p; p += L.field; }
  c->stage = (double*)p; p += L.stage;
  c->part = (double*)p; p += L.part;
  c->st = (DevState*)p; p += L.state;
  c->dbuf_dev = (void**)p; p += L.ptrs;
  c->dtlog = (double*)p; p += L.dtlog;
  c->persist_base = (int*)p; p += L.persist;
  c->max_blocks = L.max_blocks;
  c->split = 0;
  c->ys[0] = c->ys[1] = c->Bb = c->Gb = nullptr;
  c->ys[0] = p; p += L.field;
  c->ys[1] = p; p += L.field;
  if (o.precision == GLEMUR_FP64) {
    c->Bb = (double*)p; p += align256((size_t)(3 * c->N) * 8);
    c->Gb = (double*)p;
    const char* fused = getenv("GLEMUR_F64_FUSED");
    // the next-nearest-neighbour current exists in the two-pass form only
    c->split = o.curl == GLEMUR_CURL_NNN || o.periodic_z || !(fused && atoi(fused) > 0);
  }

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev);
  const bool mixed = o.precision == GLEMUR_MIXED;
  if (e == cudaSuccess) e = mixed ? prepare_f32_mimetic() : prepare_f64_mimetic();
  c->tma = 0;
  // GLEMUR_TEST_TMA_TIMEOUT=1 (2) makes the TMA prologue wait (the first
  // wait inside the plane loop) also wait on a barrier that never completes,
  // so that tests can exercise the bounded wait and the GLEMUR_ERR_TIMEOUT
  // status without any fault
  const char* tt = getenv("GLEMUR_TEST_TMA_TIMEOUT");
  c->tma_test = tt && (atoi(tt) == 1 || atoi(tt) == 2) ? atoi(tt) : 0;
  if (e == cudaSuccess && setup_tma(c)) {
    e = prepare_f32_mimetic_tma();
    c->tma = 1;
  }
  if (e == cudaSuccess) e = mixed ? prepare_f32_direct() : prepare_f64_direct();
  if (e != cudaSuccess) {
    delete c;
    return GLEMUR_ERR_CUDA;
  }
  const int gx = (nx + TX - 1) / TX, gy = (ny + TY - 1) / TY;
  // the TMA mimetic tile's height depends on its geometry
  const int thm = c->tma ? tile_rows_f32_mimetic_tma() : TY;
  const int gym = (ny + thm - 1) / thm;
  const int pm = mixed ? (c->tma ? ctas_per_sm_f32_mimetic_tma()
                                 : ctas_per_sm_f32_mimetic())
                       : ctas_per_sm_f64_mimetic();
  const int pd = mixed ? ctas_per_sm_f32_direct() : ctas_per_sm_f64_direct();
  c->kz = choose_kz(nz, gx * gym, c->nsm, pm, !mixed);
  c->grid = dim3(gx, gym, (nz + c->kz - 1) / c->kz);
  c->nblocks = gx * gym * (int)c->grid.z;
  if (c->split) {
    // per pass one wave of CTAs of 256 threads, each over an equal range of
    // node warps; the partials' stride is the larger grid
    int ob[6], oc[6];
    split_ctas_per_sm(ob, oc, o.curl == GLEMUR_CURL_NNN ? 2 : 0);
    const long long need = (c->N + 255) / 256;
    c->nblocks = 1;
    for (int s = 0; s < 6; ++s) {
      const long long cb = (long long)ob[s] * c->nsm, cc = (long long)oc[s] * c->nsm;
      c->split_grid_b[s] = (int)(need < cb ? need : cb);
      c->split_grid_c[s] = (int)(need < cc ? need : cc);
      c->nblocks = c->split_grid_b[s] > c->nblocks ? c->split_grid_b[s] : c->nblocks;
      c->nblocks = c->split_grid_c[s] > c->nblocks ? c->split_grid_c[s] : c->nblocks;
    }
  }
  // whole attempts in one persistent launch (FP64 two-pass stages of the
  // loop currents, line-tied), on request: measured slower than the
  // per-pass kernels chained by programmatic dependent launch
  c->persist = 0;
  if (c->split && o.curl != GLEMUR_CURL_DIRECT && !o.periodic_z) {
    const char* pe = getenv("GLEMUR_PERSIST");
    if (pe && atoi(pe) == 1) {
      const int per = persist_ctas_per_sm(o.curl == GLEMUR_CURL_NNN ? 2 : 0);
      long long G = (long long)per * c->nsm;
      const long long need = (c->N + 255) / 256;
      if (G > need) G = need;
      if (per >= 1 && persist_plan(c, (int)G)) {
        c->persist = 1;
        if (c->nblocks < (int)G) c->nblocks = (int)G;
      }
    }
  }
  c->kz_direct = choose_kz(nz, gx * gy, c->nsm, pd, !mixed);
  c->grid_direct = dim3(gx, gy, (nz + c->kz_direct - 1) / c->kz_direct);
  c->nblocks_direct = gx * gy * (int)c->grid_direct.z;

  // zero displacement (x = X), B0 and stage fields; boundary entries of the
  // stage fields stay zero for ever (line-tied nodes do not move)
  e = cudaMemsetAsync(c->ws, 0, 8 * L.field + L.stage + L.part, c->s);
  void* ptrs[2] = {c->dbuf[0], c->dbuf[1]};
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->dbuf_dev, ptrs, sizeof(ptrs), cudaMemcpyHostToDevice, c->s);
  if (e == cudaSuccess) e = seed_stage_inputs(c) == GLEMUR_OK ? cudaSuccess : cudaErrorUnknown;
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  if (e != cudaSuccess || reset_state(c) != GLEMUR_OK) {
    delete c;
    return GLEMUR_ERR_CUDA;
  }
  *out = c;
  return GLEMUR_OK;
}

int glemur_set_x(glemur_ctx* c, const double* x, int mem) {
  if (!c) return GLEMUR_ERR_BADARG;
  const double* src = nullptr;
  int rc = stage_in(c, x, mem, &src);
  if (rc) return rc;
  const int nb = elementwise_blocks(c->N);
  if (c->o.precision == GLEMUR_MIXED)
    k_set_x<float><<<nb, 256, 0, c->s>>>(geom(c), src, (float*)c->dbuf[0], (float*)c->dbuf[1],
                                         (float*)c->ys[0], (float*)c->ys[1]);
  else
    k_set_x<double><<<nb, 256, 0, c->s>>>(geom(c), src, (double*)c->dbuf[0],
                                          (double*)c->dbuf[1], (double*)c->ys[0],
                                          (double*)c->ys[1]);
  rc = cuda_rc(cudaGetLastError());
  if (rc) return rc;
  return reset_state(c);  // k_set_x also seeded the stage inputs
}

size_t glemur_state_bytes(const glemur_ctx* c) {
  return c ? (size_t)(3 * c->N) * c->esize : 0;
}

int glemur_get_state(glemur_ctx* c, void* buf) {
  if (!c || !buf) return GLEMUR_ERR_BADARG;
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  return cuda_rc(cudaMemcpyAsync(buf, c->dbuf[hs.cur], glemur_state_bytes(c),
                                 cudaMemcpyDeviceToDevice, c->s));
}

int glemur_set_state(glemur_ctx* c, const void* buf) {
  if (!c || !buf) return GLEMUR_ERR_BADARG;
  const size_t n = glemur_state_bytes(c);
  cudaError_t e = cudaMemcpyAsync(c->dbuf[0], buf, n, cudaMemcpyDeviceToDevice, c->s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->dbuf[1], buf, n, cudaMemcpyDeviceToDevice, c->s);
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  int rc = seed_stage_inputs(c);
  if (rc) return rc;
  return reset_state(c);
}

int glemur_set_B0(glemur_ctx* c, const double* B0, int mem) {
  if (!c) return GLEMUR_ERR_BADARG;
  const double* src = nullptr;
  int rc = stage_in(c, B0, mem, &src);
  if (rc) return rc;
  const int nb = elementwise_blocks(c->N);
  if (c->o.precision == GLEMUR_MIXED)
    k_set_B0<float><<<nb, 256, 0, c->s>>>(geom(c), src, (float*)c->B0s);
  else
    k_set_B0<double><<<nb, 256, 0, c->s>>>(geom(c), src, (double*)c->B0s);
  return cuda_rc(cudaGetLastError());
}

int glemur_get_x(glemur_ctx* c, double* x, int mem) {
  if (!c || !x || (mem != GLEMUR_MEM_DEVICE && mem != GLEMUR_MEM_HOST)) return GLEMUR_ERR_BADARG;
  double* dst = out_target(c, x, mem);
  const int nb = elementwise_blocks(c->N);
  if (c->o.precision == GLEMUR_MIXED)
    k_get_x<float><<<nb, 256, 0, c->s>>>(geom(c), (const float* const*)c->dbuf_dev, c->st, dst);
  else
    k_get_x<double><<<nb, 256, 0, c->s>>>(geom(c), (const double* const*)c->dbuf_dev, c->st,
                                          dst);
  int rc = cuda_rc(cudaGetLastError());
  if (rc) return rc;
  return stage_out(c, x, dst, mem);
}

int glemur_velocity(glemur_ctx* c, double* u, int mem) {
  if (!c || !u || (mem != GLEMUR_MEM_DEVICE && mem != GLEMUR_MEM_HOST)) return GLEMUR_ERR_BADARG;
  cudaError_t e = launch_stage(c, c->o.curl, 0, 0, 1);
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  double* dst = out_target(c, u, mem);
  const long long M = 3 * c->N;
  if (c->o.precision == GLEMUR_MIXED)
    k_to_f64<float><<<elementwise_blocks(M), 256, 0, c->s>>>(M, (const float*)c->k[0], dst);
  else
    k_to_f64<double><<<elementwise_blocks(M), 256, 0, c->s>>>(M, (const double*)c->k[0], dst);
  int rc = cuda_rc(cudaGetLastError());
  if (rc) return rc;
  return stage_out(c, u, dst, mem);
}

int glemur_attempts(glemur_ctx* c, int n_attempts) {
  if (!c || n_attempts < 0) return GLEMUR_ERR_BADARG;
  cudaError_t e = cudaSuccess;
  if (!c->target_unbounded) {
    k_set_target<<<1, 1, 0, c->s>>>(c->st, LLONG_MAX, 0);
    e = cudaGetLastError();
    c->target_unbounded = e == cudaSuccess;
  }
  if (e == cudaSuccess) e = launch_attempts(c, n_attempts);
  return cuda_rc(e);
}

int glemur_step(glemur_ctx* c, int n_accept, glemur_stats* stats) {
  if (!c || n_accept < 0) return GLEMUR_ERR_BADARG;
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  if (hs.status != ST_OK) {
    fill_stats(hs, c->o.curl, stats);
    return hs.status;
  }
  const long long target = hs.n_accept + n_accept;
  c->target_unbounded = 0;
  k_set_target<<<1, 1, 0, c->s>>>(c->st, target, 0);
  if ((rc = cuda_rc(cudaGetLastError()))) return rc;
  while (hs.n_accept < target) {
    const long long remaining = target - hs.n_accept;
    if ((rc = cuda_rc(launch_attempts(c, remaining)))) return rc;
    if ((rc = read_state(c, &hs))) return rc;
    if (hs.status != ST_OK) break;
  }
  fill_stats(hs, c->o.curl, stats);
  return hs.status;
}

int glemur_step_fixed(glemur_ctx* c, double dt, glemur_stats* stats) {
  if (!c || !(dt > 0) || !std::isfinite(dt)) return GLEMUR_ERR_BADARG;
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  if (hs.status != ST_OK) {
    fill_stats(hs, c->o.curl, stats);
    return hs.status;
  }
  c->target_unbounded = 0;
  k_set_dt<<<1, 1, 0, c->s>>>(c->st, dt, 1);
  if ((rc = cuda_rc(cudaGetLastError()))) return rc;
  if ((rc = cuda_rc(launch_attempts(c, 1)))) return rc;
  if ((rc = read_state(c, &hs))) return rc;
  fill_stats(hs, c->o.curl, stats);
  return hs.status;
}

int glemur_energy(glemur_ctx* c, double* E) {
  if (!c || !E) return GLEMUR_ERR_BADARG;
  cudaError_t e = launch_stage(c, GLEMUR_CURL_MIMETIC, 0, 1, 1);
  if (e == cudaSuccess) {
    k_diag_finalize<<<1, 256, 0, c->s>>>(c->st, c->part, nblocks_of(c, GLEMUR_CURL_MIMETIC));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  if (hs.status == ST_TIMEOUT) return GLEMUR_ERR_TIMEOUT;
  *E = hs.E;
  return GLEMUR_OK;
}

int glemur_forcefree_err(glemur_ctx* c, double* xi, double* xi_sin) {
  if (!c || !xi || !xi_sin) return GLEMUR_ERR_BADARG;
  cudaError_t e = launch_stage(c, c->o.curl, 0, 1, 1);
  if (e == cudaSuccess) {
    k_diag_finalize<<<1, 256, 0, c->s>>>(c->st, c->part, nblocks_of(c, c->o.curl));
    e = cudaGetLastError();
  }
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  if (hs.status == ST_TIMEOUT) return GLEMUR_ERR_TIMEOUT;
  *xi = hs.xi;
  *xi_sin = hs.xi_sin;
  return GLEMUR_OK;
}

int glemur_get_dt_schedule(glemur_ctx* c, long long first, int count, double* dts) {
  if (!c || !dts || first < 0 || count < 0 || count > GLEMUR_DT_LOG) return GLEMUR_ERR_BADARG;
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  // the range must have been accepted and still be held by the ring
  if (first + count > hs.n_accept || first < hs.n_accept - GLEMUR_DT_LOG) return GLEMUR_ERR_BADARG;
  if (count == 0) return GLEMUR_OK;
  // at most two contiguous pieces of the ring
  const int s0 = (int)(first % GLEMUR_DT_LOG);
  const int n0 = count < GLEMUR_DT_LOG - s0 ? count : GLEMUR_DT_LOG - s0;
  cudaError_t e = cudaMemcpyAsync(dts, c->dtlog + s0, sizeof(double) * n0,
                                  cudaMemcpyDeviceToHost, c->s);
  if (e == cudaSuccess && n0 < count)
    e = cudaMemcpyAsync(dts + n0, c->dtlog, sizeof(double) * (count - n0),
                        cudaMemcpyDeviceToHost, c->s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->s);
  return cuda_rc(e);
}

int glemur_get_stats(glemur_ctx* c, glemur_stats* stats) {
  if (!c || !stats) return GLEMUR_ERR_BADARG;
  DevState hs;
  int rc = read_state(c, &hs);
  if (rc) return rc;
  fill_stats(hs, c->o.curl, stats);
  return GLEMUR_OK;
}

int glemur_kernels_per_attempt(const glemur_ctx* c) {
  if (!c) return 0;
  if (c->persist) return 1;
  return c->split && c->o.curl != GLEMUR_CURL_DIRECT ? 13 : 7;
}

int glemur_profile_attempt(glemur_ctx* c, float* ms, int cap) {
  if (!c || !ms || cap < 7) return GLEMUR_ERR_BADARG;
  cudaEvent_t ev[8];
  int made = 0;
  cudaError_t e = cudaSuccess;
  for (; made < 8 && e == cudaSuccess; ++made) e = cudaEventCreate(&ev[made]);
  if (e != cudaSuccess) {
    for (int i = 0; i < made - 1; ++i) cudaEventDestroy(ev[i]);
    return GLEMUR_ERR_CUDA;
  }
  k_set_target<<<1, 1, 0, c->s>>>(c->st, LLONG_MAX, 0);
  e = cudaGetLastError();
  c->target_unbounded = e == cudaSuccess;
  const int diag = c->o.diag_each_attempt ? 1 : 0;
  for (int s = 0; s < 6 && e == cudaSuccess; ++s) {
    e = cudaEventRecord(ev[s], c->s);
    if (e == cudaSuccess) e = launch_stage(c, c->o.curl, s, s == 0 ? diag : 0, 0);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[6], c->s);
  if (e == cudaSuccess) {
    e = launch_pdl(k_control, dim3(1), dim3(256), 0, c->s, c->st, (const double*)c->part,
                   nblocks_of(c, c->o.curl), diag, c->dtlog);
  }
  if (e == cudaSuccess) e = cudaEventRecord(ev[7], c->s);
  if (e == cudaSuccess) e = cudaEventSynchronize(ev[7]);
  for (int i = 0; i < 7 && e == cudaSuccess; ++i) e = cudaEventElapsedTime(&ms[i], ev[i], ev[i + 1]);
  for (int i = 0; i < 8; ++i) cudaEventDestroy(ev[i]);
  return e == cudaSuccess ? 7 : GLEMUR_ERR_CUDA;
}

void glemur_destroy(glemur_ctx* c) { delete c; }

const char* glemur_strerror(int status) {
  switch (status) {
    case GLEMUR_OK: return "ok";
    case GLEMUR_ERR_BADARG: return "invalid argument";
    case GLEMUR_ERR_CUDA: return "CUDA runtime error";
    case GLEMUR_ERR_COLLAPSED: return "grid collapsed (det dx/dX <= 0)";
    case GLEMUR_ERR_NONFINITE: return "non-finite error estimate";
    case GLEMUR_ERR_DT_UNDERFLOW: return "step size underflow / too many rejections";
    case GLEMUR_ERR_WORKSPACE: return "workspace missing, misaligned or too small";
    case GLEMUR_ERR_TOO_LARGE: return "grid larger than the fixed scratch supports";
    case GLEMUR_ERR_TIMEOUT: return "a device-side wait for a tile load timed out";
    default: return "unknown status";
  }
}

}  // extern "C"
