// FP64 stage evaluation in two passes, without halo recomputation.
//
// On GB300 the FP64 pipe (2 lanes per SM per cycle, 1/64 of FP32) bounds
// the FP64 step, not HBM.  The fused stage kernel recomputes B on the tile
// halo (about 1.7 B evaluations per node) and the stage input on the
// halo-2 tile (about 2.5 combines per node); for FP64 those FP64
// instructions cost more than the extra HBM traffic of writing B once.  So
// the FP64 path evaluates each stage as
//   pass B:  B = G B0s / det G and 1/det G at every node, from the stage
//            input y_s (index-space differences: central inside,
//            second-order one-sided on boundary faces; eq. "B
//            transformation"); at interior nodes also the differences g_a
//            themselves (the current needs them again);
//   pass C:  the mimetic current J = (c_0 g_0 + c_1 g_1 + c_2 g_2)/det G
//            and u = J x B at interior nodes (eqs. "current discrete" to
//            "current matrix equation", eq. "magneto friction"), writing
//            k_s and, pointwise, the next stage input
//            y_{s+1} = d + sum_{j<=s} dt a_{s+1,j} k_j; the last stage
//            writes the fifth-order update and the embedded error instead.
// Pass C reads g_a as pass B stored it rather than forming it again from
// the stage input's neighbours: 12 fewer FP64 additions per interior node
// and stage for 72 more bytes written and read, which HBM (used at well
// under a fifth of its bandwidth by these passes) absorbs.
// Each pass runs one wave of CTAs (as many as fit on the SMs: each pass
// sizes its own grid), each over a contiguous range of whole warps of
// nodes: the FP64 pipe is per SM, so every SM gets the same number of
// node-warps (to within one per CTA) and no SM idles while another finishes
// a second round.  Each pass is launched as a programmatic dependent of the
// one before it (launch_pdl), so its CTAs take the SMs the previous pass
// leaves and start as soon as it ends; a grid of exactly the CTAs the SMs
// hold cannot crowd one SM when it is placed that way.  The per-CTA
// partials (Lambda, E_M, xi) keep the fused kernel's layout.
#include "stage_kernels.cuh"

namespace glemur {

// This CTA's node range: warps [W b / G, W (b+1) / G) of the W = N/32 node
// warps (rounded up), as node indices [begin, end).
__device__ __forceinline__ void cta_range(int N, int& begin, int& end) {
  const long long W = (N + 31) / 32;
  const long long w0 = W * blockIdx.x / gridDim.x, w1 = W * (blockIdx.x + 1) / gridDim.x;
  begin = (int)(w0 * 32);
  end = (int)(w1 * 32 < N ? w1 * 32 : N);
}

// Interior nodes enumerated densely: t in [0, (nx-2)(ny-2)(nz-2)) -> node.
// A warp then holds 32 interior nodes, so the interior code (central
// differences only) runs with no boundary lanes in it.
__device__ __forceinline__ int interior_node(const SplitArgs& a, int t, int& i, int& j, int& k) {
  const int nxi = a.nx - 2, nyi = a.ny - 2;
  i = 1 + t % nxi;
  const int r = t / nxi;
  j = 1 + r % nyi;
  k = 1 + r / nyi;
  return (k * a.ny + j) * a.nx + i;
}

// Boundary nodes enumerated densely, face by face: the two z faces (whole
// planes), the two y faces without their z edges, the two x faces without
// their y and z edges; b in [0, N - interior).
__device__ __forceinline__ int boundary_node(const SplitArgs& a, int b, int& i, int& j, int& k) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int fz = nx * ny, fy = nx * (nz - 2);
  if (b < 2 * fz) {
    k = b < fz ? 0 : nz - 1;
    const int r = b < fz ? b : b - fz;
    j = r / nx;
    i = r - j * nx;
  } else if (b < 2 * fz + 2 * fy) {
    int r = b - 2 * fz;
    j = r < fy ? 0 : ny - 1;
    r = r < fy ? r : r - fy;
    k = 1 + r / nx;
    i = r % nx;
  } else {
    const int fx = (ny - 2) * (nz - 2);
    int r = b - 2 * fz - 2 * fy;
    i = r < fx ? 0 : nx - 1;
    r = r < fx ? r : r - fx;
    k = 1 + r / (ny - 2);
    j = 1 + r % (ny - 2);
  }
  return (k * ny + j) * nx + i;
}

// Column a of G at node (i, j, k) from the stage input y.
__device__ __forceinline__ void split_gcol(const SplitArgs& a, const double* __restrict__ y, int N,
                                           int n, int ax, int idx, int ext, int stride,
                                           double out[3]) {
  const int kind = idx == 0 ? 1 : (idx == ext - 1 ? 2 : 0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double* v = y + c * N;
    double d;
    if (kind == 0)
      d = __ldg(&v[n + stride]) - __ldg(&v[n - stride]);
    else if (kind == 1)
      d = (4.0 * __ldg(&v[n + stride]) - 3.0 * __ldg(&v[n])) - __ldg(&v[n + 2 * stride]);
    else
      d = (3.0 * __ldg(&v[n]) - 4.0 * __ldg(&v[n - stride])) + __ldg(&v[n - 2 * stride]);
    out[c] = d;
  }
  out[ax] += a.h2[ax];
}

// B and 1/det G at node n = (i, j, k) from the stage input y (eq. "B
// transformation"); returns the node's energy term zeta |B|^2 det G if
// `energy`.  FACE: the general stencil (one-sided differences on the
// boundary faces the node touches), else central differences only.
template <bool FACE>
__device__ __forceinline__ double split_B_node(const SplitArgs& a, const double* __restrict__ y,
                                               int N, int n, int i, int j, int k, bool state,
                                               bool energy) {
  double g0[3], g1[3], g2[3];
  if (FACE) {
    split_gcol(a, y, N, n, 0, i, a.nx, 1, g0);
    split_gcol(a, y, N, n, 1, j, a.ny, a.nx, g1);
    split_gcol(a, y, N, n, 2, k, a.nz, a.nx * a.ny, g2);
  } else {
    const int sy = a.nx, sz = a.nx * a.ny;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double* v = y + c * N;
      g0[c] = __ldg(&v[n + 1]) - __ldg(&v[n - 1]);
      g1[c] = __ldg(&v[n + sy]) - __ldg(&v[n - sy]);
      g2[c] = __ldg(&v[n + sz]) - __ldg(&v[n - sz]);
    }
    g0[0] += a.h2[0];
    g1[1] += a.h2[1];
    g2[2] += a.h2[2];
    // 9N may exceed the 32-bit range the 3N fields stay within
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      a.Gb[(size_t)c * N + n] = g0[c];
      a.Gb[(size_t)(3 + c) * N + n] = g1[c];
      a.Gb[(size_t)(6 + c) * N + n] = g2[c];
    }
  }
  const double det = det3(g0, g1, g2);
  if (le_zero(det))  // NaN: reported by the error norm
    atomicOr(&a.st->flags, state ? FLAG_COLLAPSED : FLAG_FOLDED_TRIAL);
  const double r = recip(det);
  const double b0 = __ldg(&a.B0s[n]), b1 = __ldg(&a.B0s[N + n]), b2 = __ldg(&a.B0s[2 * N + n]);
  double B[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    B[c] = (g0[c] * b0 + g1[c] * b1 + g2[c] * b2) * r;
    a.Bb[c * N + n] = B[c];
  }
  a.rb[n] = r;
  if (!energy) return 0.0;
  // eq. "magnetic energy": zeta halves per boundary index coordinate
  const int nb = (i == 0 || i == a.nx - 1) + (j == 0 || j == a.ny - 1) + (k == 0 || k == a.nz - 1);
  const double zeta = nb == 0 ? 1.0 : nb == 1 ? 0.5 : nb == 2 ? 0.25 : 0.125;
  return zeta * dot3(B, B) * det;
}

// This CTA's partial of kind `kind`; the slots of the partial stride beyond
// this launch's grid are zeroed (neutral for the sums and for the maxima of
// non-negative values), so a pass with fewer CTAs than the stride leaves no
// stale slot behind.
__device__ __forceinline__ void put_partial(const SplitArgs& a, int kind, double v) {
  double* p = a.part + kind * a.nblocks;
  p[blockIdx.x] = v;
  for (int b = gridDim.x + blockIdx.x; b < a.nblocks; b += gridDim.x) p[b] = 0.0;
}

// a.b - c.d as one multiply and five FMAs (one FP64 instruction fewer than
// two dot products and a subtraction)
__device__ __forceinline__ double dot3_sub(const double a[3], const double b[3],
                                           const double c[3], const double d[3]) {
  double t = a[0] * b[0];
  t = fma(a[1], b[1], t);
  t = fma(a[2], b[2], t);
  t = fma(-c[0], d[0], t);
  t = fma(-c[1], d[1], t);
  return fma(-c[2], d[2], t);
}

// Pass B (stage s): B and 1/det G at every node, interior nodes (central
// differences) and boundary nodes (one-sided on their faces) in separate
// dense loops -- in one loop the compiler evaluates the one-sided variants
// under predicates for every node, and predicated-off FP64 instructions
// still take FP64-pipe slots; in the diagnostic launch also the energy
// partials (eq. "magnetic energy").
template <int S>
__global__ void __launch_bounds__(256) k_split_B(const SplitArgs a) {
  pdl_wait();
  const DevState* st = a.st;
  if (!a.force && (st->status != ST_OK || st->n_accept >= st->target)) return;
  __shared__ double red[8];
  const int N = a.nx * a.ny * a.nz;
  const int NI = (a.nx - 2) * (a.ny - 2) * (a.nz - 2);
  const double* y = S == 0 ? a.d[st->cur] : a.ys[S & 1];
  const bool energy = S == 0 && a.diag;
  double eacc = 0.0;
  int tb, te;
  cta_range(NI, tb, te);
#pragma unroll 2  // two nodes' loads in flight (48 -> 64 registers, +1 % at 64^3)
  for (int t = tb + threadIdx.x; t < te; t += blockDim.x) {
    int i, j, k;
    const int n = interior_node(a, t, i, j, k);
    eacc += split_B_node<false>(a, y, N, n, i, j, k, S == 0, energy);
  }
  cta_range(N - NI, tb, te);
  for (int b = tb + threadIdx.x; b < te; b += blockDim.x) {
    int i, j, k;
    const int n = boundary_node(a, b, i, j, k);
    eacc += split_B_node<true>(a, y, N, n, i, j, k, S == 0, energy);
  }
  pdl_trigger();
  if (energy) {
    const double v = block_reduce<false>(eacc, red);
    if (threadIdx.x == 0) put_partial(a, PART_E, v);
  }
}

// Pass C (stage s): current and velocity at interior nodes; k_s and the
// next stage input, or (s = 5) the update, the error and k6.  Held to 64
// registers (a few spilled values in two of the stages): four CTAs (32
// warps) per SM instead of three, at no measured cost.
template <int S>
__global__ void __launch_bounds__(256, 4) k_split_C(const SplitArgs a) {
  constexpr bool FINAL = S == 5;
  pdl_wait();
  const DevState* st = a.st;
  if (!a.force && (st->status != ST_OK || st->n_accept >= st->target)) return;
  __shared__ double red[8];
  const int N = a.nx * a.ny * a.nz;
  const int cur = st->cur;
  const double* d = a.d[cur];
  double* dout = const_cast<double*>(a.d[cur ^ 1]);
  double* ynext = a.ys[(S + 1) & 1];
  double an[5];  // dt a_{S+1, j}: next stage input (non-final stages)
#pragma unroll
  for (int j = 0; j < 5; ++j) an[j] = (!FINAL && j <= S) ? st->dta[S + 1][j] : 0.0;
  Acc<double> acc;
  const int sy = a.nx, sz = a.nx * a.ny;
  const int NI = (a.nx - 2) * (a.ny - 2) * (a.nz - 2);
  int tb, te;
  cta_range(NI, tb, te);
  for (int t = tb + threadIdx.x; t < te; t += blockDim.x) {
    int i, j, k;
    const int n = interior_node(a, t, i, j, k);
    double g0[3], g1[3], g2[3], P0[3], P1[3], P2[3], B[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double* b = a.Bb + c * N;
      g0[c] = __ldg(&a.Gb[(size_t)c * N + n]);
      g1[c] = __ldg(&a.Gb[(size_t)(3 + c) * N + n]);
      g2[c] = __ldg(&a.Gb[(size_t)(6 + c) * N + n]);
      P0[c] = __ldg(&b[n + 1]) - __ldg(&b[n - 1]);
      P1[c] = __ldg(&b[n + sy]) - __ldg(&b[n - sy]);
      P2[c] = __ldg(&b[n + sz]) - __ldg(&b[n - sz]);
      B[c] = __ldg(&b[n]);
    }
    const double c0 = dot3_sub(P1, g2, P2, g1);
    const double c1 = dot3_sub(P2, g0, P0, g2);
    const double c2 = dot3_sub(P0, g1, P1, g0);
    const double r = __ldg(&a.rb[n]);
    double J[3], u[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) J[c] = (c0 * g0[c] + c1 * g1[c] + c2 * g2[c]) * r;
    u[0] = J[1] * B[2] - J[2] * B[1];
    u[1] = J[2] * B[0] - J[0] * B[2];
    u[2] = J[0] * B[1] - J[1] * B[0];
    if (S == 0 && a.diag) acc.max_xi(dot3(u, u), dot3(B, B), dot3(J, J));
    if (!FINAL) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a.k[S][c * N + n] = u[c];
        // next stage input y_{S+1} = d + sum_{j<=S} dt a_{S+1,j} k_j
        double v = __ldg(&d[c * N + n]);
#pragma unroll
        for (int jj = 0; jj < S; ++jj) v = fma(an[jj], __ldg(&a.k[jj][c * N + n]), v);
        v = fma(an[S], u[c], v);
        ynext[c * N + n] = v;
      }
    } else {
      const double b0 = st->dtb[0], b2 = st->dtb[2], b3 = st->dtb[3], b5 = st->dtb[5];
      const double e0 = st->dte[0], e2 = st->dte[2], e3 = st->dte[3], e4 = st->dte[4],
                   e5 = st->dte[5];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double k1 = __ldg(&a.k[0][c * N + n]), k3 = __ldg(&a.k[2][c * N + n]),
                     k4 = __ldg(&a.k[3][c * N + n]), k5 = __ldg(&a.k[4][c * N + n]);
        double up = b0 * k1;
        up = fma(b2, k3, up);
        up = fma(b3, k4, up);
        up = fma(b5, u[c], up);
        double er = e0 * k1;
        er = fma(e2, k3, er);
        er = fma(e3, k4, er);
        er = fma(e4, k5, er);
        er = fma(e5, u[c], er);
        dout[c * N + n] = __ldg(&d[c * N + n]) + up;
        acc.max_lam(fabs(er));
        if (a.k[5]) a.k[5][c * N + n] = u[c];
      }
    }
  }
  pdl_trigger();
  if (FINAL) {
    const double v = block_reduce<true>(acc.lam, red);
    if (threadIdx.x == 0) put_partial(a, PART_LAMBDA, v);
  }
  if (S == 0 && a.diag) {
    double v = block_reduce<true>(acc.xi2(), red);
    if (threadIdx.x == 0) put_partial(a, PART_XI2, v);
    v = block_reduce<true>(acc.xis2(), red);
    if (threadIdx.x == 0) put_partial(a, PART_XIS2, v);
  }
}

// CTAs of 256 threads per SM that pass B and pass C of each stage can hold.
void split_ctas_per_sm(int b[6], int c[6]) {
  void (*kb[6])(const SplitArgs) = {k_split_B<0>, k_split_B<1>, k_split_B<2>,
                                    k_split_B<3>, k_split_B<4>, k_split_B<5>};
  void (*kc[6])(const SplitArgs) = {k_split_C<0>, k_split_C<1>, k_split_C<2>,
                                    k_split_C<3>, k_split_C<4>, k_split_C<5>};
  for (int s = 0; s < 6; ++s) {
    b[s] = c[s] = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[s], kb[s], 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c[s], kc[s], 256, 0);
    if (b[s] < 1) b[s] = 1;
    if (c[s] < 1) c[s] = 1;
  }
}

// Launch both passes of stage s (grid_b[s], grid_c[s] CTAs of 256 threads).
cudaError_t launch_f64_split(const SplitArgs& a, int stage, cudaStream_t s) {
  if (stage < 0 || stage > 5) return cudaErrorInvalidValue;
  const dim3 gb(a.grid_b[stage]), gc(a.grid_c[stage]);
  cudaError_t e = cudaSuccess;
#define GLEMUR_SPLIT_CASE(SS)                                                      \
  case SS:                                                                         \
    e = launch_pdl(k_split_B<SS>, gb, dim3(256), 0, s, a);                         \
    if (e == cudaSuccess) e = launch_pdl(k_split_C<SS>, gc, dim3(256), 0, s, a);   \
    break;
  switch (stage) {
    GLEMUR_SPLIT_CASE(0)
    GLEMUR_SPLIT_CASE(1)
    GLEMUR_SPLIT_CASE(2)
    GLEMUR_SPLIT_CASE(3)
    GLEMUR_SPLIT_CASE(4)
    GLEMUR_SPLIT_CASE(5)
    default:
      return cudaErrorInvalidValue;
  }
#undef GLEMUR_SPLIT_CASE
  return e;
}

}  // namespace glemur
