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
// Pass C reads g_a (and 1/det G) as pass B stored them, interleaved per
// node, rather than forming g_a again from the stage input's neighbours:
// 12 fewer FP64 additions per interior node and stage for 80 bytes written
// and read (five 16-byte accesses each way), which HBM (used at well under
// a fifth of its bandwidth by these passes) absorbs.
// Each pass runs one wave of CTAs (as many as fit on the SMs: each pass
// sizes its own grid), each over a contiguous range of whole warps of
// nodes: the FP64 pipe is per SM, so every SM gets the same number of
// node-warps (to within one per CTA) and no SM idles while another finishes
// a second round.  Each pass is launched as a programmatic dependent of the
// one before it (launch_pdl), so its CTAs take the SMs the previous pass
// leaves and start as soon as it ends; a grid of exactly the CTAs the SMs
// hold cannot crowd one SM when it is placed that way.  The per-CTA
// partials (Lambda, E_M, xi) keep the fused kernel's layout.
#include "control.cuh"
#include "stage_kernels.cuh"
#include "tma.cuh"

namespace glemur {

// How the passes load data that another CTA of the same launch may have
// written: the per-pass kernels use the read-only path (__ldg) -- each pass
// only reads what earlier launches wrote -- while the persistent attempt
// kernel, whose CTAs read each other's results within one launch, uses
// ordinary (weak) global loads: the read-only path may keep lines from an
// earlier pass, whereas weak loads that follow, in causality order, an
// acquire that observed the writer's release must return the released
// values (the PTX memory model; the waits below are exactly that pattern).
// The loads are volatile asm so that the compiler neither merges loads of
// one address from different passes nor moves them across the waits.
struct LdRO {
  __device__ static __forceinline__ double ld(const double* p) { return __ldg(p); }
  __device__ static __forceinline__ double2 ld2(const double2* p) { return __ldg(p); }
  __device__ static __forceinline__ int ldi(const int* p) { return *p; }
};
struct LdL2 {
  __device__ static __forceinline__ double ld(const double* p) {
    double v;
    asm volatile("ld.global.f64 %0, [%1];" : "=d"(v) : "l"(p));
    return v;
  }
  __device__ static __forceinline__ double2 ld2(const double2* p) {
    double2 v;
    asm volatile("ld.global.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p));
    return v;
  }
  __device__ static __forceinline__ int ldi(const int* p) {
    int v;
    asm volatile("ld.global.b32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
  }
};

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

// Boundary nodes enumerated densely, grouped so that the lanes of a warp
// share one stencil variant per axis: the inner parts of the two z faces,
// the two y faces and the two x faces (one boundary index coordinate), the
// edges along x, y and z (two), then the eight corners; b in
// [0, N - interior).  (A warp mixes variants only where it straddles two
// groups.)  The host's persistent-kernel plan mirrors this order.
__device__ __forceinline__ int boundary_node(const SplitArgs& a, int b, int& i, int& j, int& k) {
  const int nx = a.nx, ny = a.ny, nz = a.nz;
  const int xi = nx - 2, yi = ny - 2, zi = nz - 2;
  const int fz = xi * yi, fy = xi * zi, fx = yi * zi;
  if (b < 2 * fz) {
    k = b < fz ? 0 : nz - 1;
    const int r = b < fz ? b : b - fz;
    i = 1 + r % xi;
    j = 1 + r / xi;
  } else if ((b -= 2 * fz) < 2 * fy) {
    j = b < fy ? 0 : ny - 1;
    const int r = b < fy ? b : b - fy;
    i = 1 + r % xi;
    k = 1 + r / xi;
  } else if ((b -= 2 * fy) < 2 * fx) {
    i = b < fx ? 0 : nx - 1;
    const int r = b < fx ? b : b - fx;
    j = 1 + r % yi;
    k = 1 + r / yi;
  } else if ((b -= 2 * fx) < 4 * xi) {
    const int e = b / xi;
    i = 1 + b % xi;
    j = (e & 1) ? ny - 1 : 0;
    k = (e & 2) ? nz - 1 : 0;
  } else if ((b -= 4 * xi) < 4 * yi) {
    const int e = b / yi;
    j = 1 + b % yi;
    i = (e & 1) ? nx - 1 : 0;
    k = (e & 2) ? nz - 1 : 0;
  } else if ((b -= 4 * yi) < 4 * zi) {
    const int e = b / zi;
    k = 1 + b % zi;
    i = (e & 1) ? nx - 1 : 0;
    j = (e & 2) ? ny - 1 : 0;
  } else {
    b -= 4 * zi;
    i = (b & 1) ? nx - 1 : 0;
    j = (b & 2) ? ny - 1 : 0;
    k = (b & 4) ? nz - 1 : 0;
  }
  return (k * ny + j) * nx + i;
}

// One column of G from the stage input y along an axis of node stride
// `stride`, without the 2 h_a e_a term.  ONE = false: the central
// difference v(n+s) - v(n-s).  ONE = true: the second-order one-sided
// difference into the domain, (4 v(n+s) - 3 v(n)) - v(n+2s) at the low face
// (sg = +1) and (3 v(n) - 4 v(n-s)) + v(n-2s) at the high face (sg = -1),
// both as sg times the first form with s -> sg s: the signs ride on
// constants chosen by a select (multiplying by -1 is exact), so both faces
// run the same three FP64 instructions per component.
template <bool ONE, class LD>
__device__ __forceinline__ void gcol(const double* __restrict__ y, int N, int n, int stride,
                                     int sg, double out[3]) {
  const int s = sg * stride;
  const double c4 = sg > 0 ? 4.0 : -4.0, m3 = sg > 0 ? -3.0 : 3.0, m1 = sg > 0 ? -1.0 : 1.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double* v = y + c * N;
    if (!ONE)
      out[c] = LD::ld(&v[n + stride]) - LD::ld(&v[n - stride]);
    else
      out[c] = fma(m1, LD::ld(&v[n + 2 * s]), fma(c4, LD::ld(&v[n + s]), m3 * LD::ld(&v[n])));
  }
}

// det G, 1/det G and B = G B0s / det G at node n from its columns (eq. "B
// transformation"); B (and 1/det G if rb is set) stored at node nw (n
// itself, or a periodic ghost node that carries n's B), with G: the
// differences and 1/det G interleaved for pass C (interior nodes).  Returns
// the node's energy term zeta |B|^2 det G if `energy`.
template <bool WITH_G>
__device__ __forceinline__ double split_B_finish(const SplitArgs& a, int N, int n, int i, int j,
                                                 int k, bool state, bool energy, int nw,
                                                 double g0[3], double g1[3], double g2[3]) {
  g0[0] += a.h2[0];
  g1[1] += a.h2[1];
  g2[2] += a.h2[2];
  const double det = det3(g0, g1, g2);
  if (le_zero(det))  // NaN: reported by the error norm
    atomicOr(&a.st->flags, state ? FLAG_COLLAPSED : FLAG_FOLDED_TRIAL);
  const double r = recip(det);
  if (WITH_G) {
    // the node's differences and 1/det G for pass C, as five 16-byte
    // stores (10 N doubles: size_t offsets)
    double2* q = reinterpret_cast<double2*>(a.Gb + (size_t)n * 10);
    q[0] = make_double2(g0[0], g0[1]);
    q[1] = make_double2(g0[2], g1[0]);
    q[2] = make_double2(g1[1], g1[2]);
    q[3] = make_double2(g2[0], g2[1]);
    q[4] = make_double2(g2[2], r);
  }
  const double b0 = __ldg(&a.B0s[n]), b1 = __ldg(&a.B0s[N + n]), b2 = __ldg(&a.B0s[2 * N + n]);
  double B[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    B[c] = (g0[c] * b0 + g1[c] * b1 + g2[c] * b2) * r;
    a.Bb[c * N + nw] = B[c];
  }
  if (a.rb) a.rb[nw] = r;
  if (!energy) return 0.0;
  // eq. "magnetic energy": zeta halves per boundary index coordinate
  const int nb = (i == 0 || i == a.nx - 1) + (j == 0 || j == a.ny - 1) + (k == 0 || k == a.nz - 1);
  const double zeta = nb == 0 ? 1.0 : nb == 1 ? 0.5 : nb == 2 ? 0.25 : 0.125;
  return zeta * dot3(B, B) * det;
}

// B at an interior node (central differences), storing G for pass C.
template <class LD>
__device__ __forceinline__ double split_B_interior(const SplitArgs& a,
                                                   const double* __restrict__ y, int N, int n,
                                                   int i, int j, int k, bool state,
                                                   bool energy) {
  double g0[3], g1[3], g2[3];
  gcol<false, LD>(y, N, n, 1, 1, g0);
  gcol<false, LD>(y, N, n, a.nx, 1, g1);
  gcol<false, LD>(y, N, n, a.nx * a.ny, 1, g2);
  return split_B_finish<true>(a, N, n, i, j, k, state, energy, n, g0, g1, g2);
}

// B at a boundary node (or, with periodic z, at the partner of a ghost
// node): one-sided along the axes with sx, sy, sz != 0 (+1 low face, -1
// high face), central along the others; the variant is a template
// argument, so each runs its own FP64 instructions only.
template <bool OX, bool OY, bool OZ, class LD>
__device__ __forceinline__ double split_B_bvar(const SplitArgs& a, const double* __restrict__ y,
                                               int N, int n, int i, int j, int k, int sx,
                                               int sy, int sz, bool state, bool energy,
                                               int nw) {
  double g0[3], g1[3], g2[3];
  gcol<OX, LD>(y, N, n, 1, sx, g0);
  gcol<OY, LD>(y, N, n, a.nx, sy, g1);
  gcol<OZ, LD>(y, N, n, a.nx * a.ny, sz, g2);
  return split_B_finish<false>(a, N, n, i, j, k, state, energy, nw, g0, g1, g2);
}

template <class LD>
__device__ __forceinline__ double split_B_boundary(const SplitArgs& a,
                                                   const double* __restrict__ y, int N, int n,
                                                   int i, int j, int k, int sx, int sy, int sz,
                                                   bool state, bool energy, int nw) {
#define GLEMUR_BVAR(X, Y, Z) \
  return split_B_bvar<X, Y, Z, LD>(a, y, N, n, i, j, k, sx, sy, sz, state, energy, nw)
  switch ((sx != 0) * 4 + (sy != 0) * 2 + (sz != 0)) {
    case 0: GLEMUR_BVAR(false, false, false);
    case 1: GLEMUR_BVAR(false, false, true);
    case 2: GLEMUR_BVAR(false, true, false);
    case 3: GLEMUR_BVAR(false, true, true);
    case 4: GLEMUR_BVAR(true, false, false);
    case 5: GLEMUR_BVAR(true, false, true);
    case 6: GLEMUR_BVAR(true, true, false);
    default: GLEMUR_BVAR(true, true, true);
  }
#undef GLEMUR_BVAR
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
template <int S, class LD>
__device__ __forceinline__ void pass_B(const SplitArgs& a, int cur, double* red) {
  const int N = a.nx * a.ny * a.nz;
  const int NI = (a.nx - 2) * (a.ny - 2) * (a.nz - 2);
  const double* y = S == 0 ? a.d[cur] : a.ys[S & 1];
  const bool energy = S == 0 && a.diag;
  double eacc = 0.0;
  int tb, te;
  cta_range(NI, tb, te);
#pragma unroll 2  // two nodes' loads in flight (48 -> 64 registers, +1 % at 64^3)
  for (int t = tb + threadIdx.x; t < te; t += blockDim.x) {
    int i, j, k;
    const int n = interior_node(a, t, i, j, k);
    eacc += split_B_interior<LD>(a, y, N, n, i, j, k, S == 0, energy);
  }
  cta_range(N - NI, tb, te);
  for (int b = tb + threadIdx.x; b < te; b += blockDim.x) {
    int i, j, k;
    const int n = boundary_node(a, b, i, j, k);
    const int sx = i == 0 ? 1 : (i == a.nx - 1 ? -1 : 0);
    const int sy = j == 0 ? 1 : (j == a.ny - 1 ? -1 : 0);
    const int sz = k == 0 ? 1 : (k == a.nz - 1 ? -1 : 0);
    if (a.periodic && sz != 0) {
      // a ghost plane carries its partner's B (section "Boundary
      // Conditions"); it is not part of the period's energy
      const int kk = sz > 0 ? a.nz - 2 : 1;
      const int np = (kk * a.ny + j) * a.nx + i;
      split_B_boundary<LD>(a, y, N, np, i, j, kk, sx, sy, 0, S == 0, false, n);
    } else {
      eacc += split_B_boundary<LD>(a, y, N, n, i, j, k, sx, sy, sz, S == 0, energy, n);
    }
  }
  pdl_trigger();
  if (energy) {
    const double v = block_reduce<false>(eacc, red);
    if (threadIdx.x == 0) put_partial(a, PART_E, v);
  }
}

// No minimum-CTA bound: the later stages' pass B fits 64 registers (four
// CTAs per SM) by itself, the first (with the energy sum) takes 76 (three
// CTAs, its grid sized to match); forcing four CTAs on every stage made each
// of them spill.
template <int S>
__global__ void __launch_bounds__(256) k_split_B(const SplitArgs a) {
  pdl_wait();
  const DevState* st = a.st;
  if (!a.force && (st->status != ST_OK || st->n_accept >= st->target)) return;
  __shared__ double red[8];
  pass_B<S, LdRO>(a, st->cur, red);
}

// One octilateral loop of the next-nearest-neighbour current (section
// "Next Nearest Neighbor Mimetic Approach") in the index surface spanned by
// P and Q: the eight in-plane neighbours V_1..V_8 at (along P, along Q) =
// (1,-1), (1,0), (1,1), (0,1), (-1,1), (-1,0), (-1,-1), (0,-1), positions
// r_m taken relative to the node (displacement differences plus the label
// offsets).  Returns twice the circulation and twice the vector area (the
// common factor 1/2 cancels in M J = c):
//   circulation with edge-mean B (eq. "current discrete", eight edges):
//     sum_m (B_m + B_m+1)/2 . (r_m+1 - r_m) = sum_m B_m . (r_m+1 - r_m-1) / 2
//   vector area (eq. "sum of eight triangles": four corner triangles plus the
//   inner quadrilateral through V_2, V_4, V_6, V_8): a surface spanning the
//   loop, so its vector area is the loop's, sum_m r_m x r_m+1 / 2.
// The vertices stream through registers (three positions and one B live).
template <int P, int Q, class LD>
__device__ __forceinline__ void nnn_loop(const SplitArgs& a, const double* __restrict__ y,
                                         int N, int n, const double yc[3], double& circ2,
                                         double area2[3]) {
  constexpr int OP[8] = {1, 1, 1, 0, -1, -1, -1, 0};
  constexpr int OQ[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
  const int sp = P == 0 ? 1 : (P == 1 ? a.nx : a.nx * a.ny);
  const int sq = Q == 0 ? 1 : (Q == 1 ? a.nx : a.nx * a.ny);
  const double hp = 0.5 * a.h2[P], hq = 0.5 * a.h2[Q];
  double r0[3], b0[3], r1[3], rp[3], rc[3], bc[3];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int nn = n + OP[m] * sp + OQ[m] * sq;
    double rv[3], bv[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      rv[c] = LD::ld(&y[c * N + nn]) - yc[c];
      bv[c] = LD::ld(&a.Bb[c * N + nn]);
    }
    if (OP[m] != 0) rv[P] += OP[m] > 0 ? hp : -hp;
    if (OQ[m] != 0) rv[Q] += OQ[m] > 0 ? hq : -hq;
    if (m == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c) { r0[c] = rv[c]; b0[c] = bv[c]; }
    } else {
      // r_m-1 x r_m
      const double* u = m == 1 ? r0 : rc;
      if (m == 1) {
        area2[0] = u[1] * rv[2] - u[2] * rv[1];
        area2[1] = u[2] * rv[0] - u[0] * rv[2];
        area2[2] = u[0] * rv[1] - u[1] * rv[0];
      } else {
        area2[0] = fma(u[1], rv[2], fma(-u[2], rv[1], area2[0]));
        area2[1] = fma(u[2], rv[0], fma(-u[0], rv[2], area2[1]));
        area2[2] = fma(u[0], rv[1], fma(-u[1], rv[0], area2[2]));
      }
      if (m >= 2) {  // the term of vertex m-1: B_m-1 . (r_m - r_m-2)
        const double* w = m == 2 ? r0 : rp;
        double t = bc[0] * (rv[0] - w[0]);
        t = fma(bc[1], rv[1] - w[1], t);
        t = fma(bc[2], rv[2] - w[2], t);
        circ2 = m == 2 ? t : circ2 + t;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        if (m == 1) r1[c] = rv[c];
        rp[c] = m == 1 ? r0[c] : rc[c];
        rc[c] = rv[c];
        bc[c] = bv[c];
      }
    }
  }
  // close the loop: r_8 x r_1, and the terms of V_8 and V_1
  area2[0] = fma(rc[1], r0[2], fma(-rc[2], r0[1], area2[0]));
  area2[1] = fma(rc[2], r0[0], fma(-rc[0], r0[2], area2[1]));
  area2[2] = fma(rc[0], r0[1], fma(-rc[1], r0[0], area2[2]));
#pragma unroll
  for (int c = 0; c < 3; ++c) circ2 = fma(bc[c], r0[c] - rp[c], circ2);
#pragma unroll
  for (int c = 0; c < 3; ++c) circ2 = fma(b0[c], r1[c] - rc[c], circ2);
}

// The next-nearest-neighbour current at interior node n and B there: the
// three loops (surfaces r = 0, 1, 2 spanned by p = r+1, q = r+2 mod 3,
// counter-clockwise about +r) give the rows of M and the entries of c in
// eq. "current matrix equation", solved by the adjugate,
// J = (c_0 a_1 x a_2 + c_1 a_2 x a_0 + c_2 a_0 x a_1) / det M.
template <class LD>
__device__ __forceinline__ void nnn_current(const SplitArgs& a, const double* __restrict__ y,
                                            int N, int n, double J[3], double B[3]) {
  double yc[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) yc[c] = LD::ld(&y[c * N + n]);
  double M[3][3], cr[3];
  nnn_loop<1, 2, LD>(a, y, N, n, yc, cr[0], M[0]);
  nnn_loop<2, 0, LD>(a, y, N, n, yc, cr[1], M[1]);
  nnn_loop<0, 1, LD>(a, y, N, n, yc, cr[2], M[2]);
  double adj[3][3];  // adj[r] = a_{r+1} x a_{r+2}
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    const double* u = M[(r + 1) % 3];
    const double* v = M[(r + 2) % 3];
    adj[r][0] = u[1] * v[2] - u[2] * v[1];
    adj[r][1] = u[2] * v[0] - u[0] * v[2];
    adj[r][2] = u[0] * v[1] - u[1] * v[0];
  }
  const double detM = dot3(M[0], adj[0]);
#pragma unroll
  for (int c = 0; c < 3; ++c)
    J[c] = (cr[0] * adj[0][c] + cr[1] * adj[1][c] + cr[2] * adj[2][c]) / detM;
#pragma unroll
  for (int c = 0; c < 3; ++c) B[c] = LD::ld(&a.Bb[c * N + n]);
}

// Pass C (stage s): current and velocity at interior nodes; k_s and the
// next stage input, or (s = 5) the update, the error and k6.  CURL 0: the
// nearest-neighbour current, held to 64 registers (four CTAs, 32 warps, per
// SM); CURL 2: the next-nearest-neighbour current (a comparison option,
// two CTAs per SM).
template <int S, int CURL, class LD>
__device__ __forceinline__ void pass_C(const SplitArgs& a, int cur, double* red) {
  constexpr bool FINAL = S == 5;
  const DevState* st = a.st;
  const int N = a.nx * a.ny * a.nz;
  const double* d = a.d[cur];
  double* dout = const_cast<double*>(a.d[cur ^ 1]);
  double* ynext = a.ys[(S + 1) & 1];
  double an[5];  // dt a_{S+1, j}: next stage input (non-final stages)
#pragma unroll
  for (int j = 0; j < 5; ++j) an[j] = (!FINAL && j <= S) ? LD::ld(&st->dta[S + 1][j]) : 0.0;
  Acc<double> acc;
  const int sy = a.nx, sz = a.nx * a.ny;
  const int NI = (a.nx - 2) * (a.ny - 2) * (a.nz - 2);
  int tb, te;
  cta_range(NI, tb, te);
  for (int t = tb + threadIdx.x; t < te; t += blockDim.x) {
    int i, j, k;
    const int n = interior_node(a, t, i, j, k);
    double J[3], B[3], u[3];
    if constexpr (CURL == 2) {
      nnn_current<LD>(a, S == 0 ? d : a.ys[S & 1], N, n, J, B);
    } else {
      double g0[3], g1[3], g2[3], P0[3], P1[3], P2[3];
      const double2* q = reinterpret_cast<const double2*>(a.Gb + (size_t)n * 10);
      const double2 q0 = LD::ld2(q), q1 = LD::ld2(q + 1), q2 = LD::ld2(q + 2),
                    q3 = LD::ld2(q + 3), q4 = LD::ld2(q + 4);
      g0[0] = q0.x; g0[1] = q0.y; g0[2] = q1.x;
      g1[0] = q1.y; g1[1] = q2.x; g1[2] = q2.y;
      g2[0] = q3.x; g2[1] = q3.y; g2[2] = q4.x;
      const double r = q4.y;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double* b = a.Bb + c * N;
        P0[c] = LD::ld(&b[n + 1]) - LD::ld(&b[n - 1]);
        P1[c] = LD::ld(&b[n + sy]) - LD::ld(&b[n - sy]);
        P2[c] = LD::ld(&b[n + sz]) - LD::ld(&b[n - sz]);
        B[c] = LD::ld(&b[n]);
      }
      const double c0 = dot3_sub(P1, g2, P2, g1);
      const double c1 = dot3_sub(P2, g0, P0, g2);
      const double c2 = dot3_sub(P0, g1, P1, g0);
#pragma unroll
      for (int c = 0; c < 3; ++c) J[c] = (c0 * g0[c] + c1 * g1[c] + c2 * g2[c]) * r;
    }
    u[0] = J[1] * B[2] - J[2] * B[1];
    u[1] = J[2] * B[0] - J[0] * B[2];
    u[2] = J[0] * B[1] - J[1] * B[0];
    if (S == 0 && a.diag) acc.max_xi(dot3(u, u), dot3(B, B), dot3(J, J));
    if (!FINAL) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        a.k[S][c * N + n] = u[c];
        // next stage input y_{S+1} = d + sum_{j<=S} dt a_{S+1,j} k_j
        double v = LD::ld(&d[c * N + n]);
#pragma unroll
        for (int jj = 0; jj < S; ++jj) v = fma(an[jj], LD::ld(&a.k[jj][c * N + n]), v);
        v = fma(an[S], u[c], v);
        ynext[c * N + n] = v;
        // periodic in z: the ghost of an end plane holds the same
        // displacement (its position differs by the period)
        if (a.periodic && (k == 1 || k == a.nz - 2))
          ynext[c * N + n + (k == 1 ? 1 : -1) * (a.nz - 2) * sz] = v;
      }
    } else {
      const double b0 = LD::ld(&st->dtb[0]), b2 = LD::ld(&st->dtb[2]),
                   b3 = LD::ld(&st->dtb[3]), b5 = LD::ld(&st->dtb[5]);
      const double e0 = LD::ld(&st->dte[0]), e2 = LD::ld(&st->dte[2]),
                   e3 = LD::ld(&st->dte[3]), e4 = LD::ld(&st->dte[4]),
                   e5 = LD::ld(&st->dte[5]);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double k1 = LD::ld(&a.k[0][c * N + n]), k3 = LD::ld(&a.k[2][c * N + n]),
                     k4 = LD::ld(&a.k[3][c * N + n]), k5 = LD::ld(&a.k[4][c * N + n]);
        double up = b0 * k1;
        up = fma(b2, k3, up);
        up = fma(b3, k4, up);
        up = fma(b5, u[c], up);
        double er = e0 * k1;
        er = fma(e2, k3, er);
        er = fma(e3, k4, er);
        er = fma(e4, k5, er);
        er = fma(e5, u[c], er);
        const double dn = LD::ld(&d[c * N + n]) + up;
        dout[c * N + n] = dn;
        if (a.periodic && (k == 1 || k == a.nz - 2))
          dout[c * N + n + (k == 1 ? 1 : -1) * (a.nz - 2) * sz] = dn;
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

template <int S, int CURL>
__global__ void __launch_bounds__(256, CURL == 2 ? 2 : 4) k_split_C(const SplitArgs a) {
  pdl_wait();
  const DevState* st = a.st;
  if (!a.force && (st->status != ST_OK || st->n_accept >= st->target)) return;
  __shared__ double red[8];
  pass_C<S, CURL, LdRO>(a, st->cur, red);
}

// ---- persistent attempts ------------------------------------------------
//
// One cooperative launch runs whole attempts: the twelve passes and the
// step control, with no kernel boundary between them.  Each CTA keeps the
// node ranges it has in the per-pass kernels (the grid is the CTAs the SMs
// hold, all resident), and instead of a grid-wide boundary after each pass
// it waits only for the node planes its next pass reads:
//   pass B of stage s at plane p reads the stage input at planes p-2..p+2,
//     written by pass C of stage s-1 (the one-sided boundary stencil reaches
//     two planes; the same wait orders pass C's earlier reads of the B, G
//     and stage-input buffers that pass B now overwrites);
//   pass C of stage s at plane p reads B at planes p-1..p+1 from pass B.
// A CTA publishes a finished pass by adding one to the completion counter
// of every plane its work touched (after a fence that makes its writes
// visible at device scope); a wait reads the counters through L2 until they
// reach (CTAs touching the plane) x (passes done).  The last CTA to finish
// an attempt runs the step control and releases the others; the next
// attempt's first pass reads the state the control selected.  All data
// another CTA may have written is loaded through L2 (LdL2).  Every wait is
// bounded: after 2 s it raises FLAG_TIMEOUT and status TIMEOUT and the CTA
// leaves; the others see the flag in their own waits and leave too.
// Results are bit-identical to the per-pass kernels: each node's
// arithmetic is the same.  Measured on GB300 it is about 5 % slower than
// the per-pass kernels chained by programmatic dependent launch (64^3 and
// 96^3 braids), so it runs only on request (GLEMUR_PERSIST=1).

constexpr unsigned long long PERSIST_WAIT_NS = 2000000000ull;

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Spin until *p >= want (bounded); false on timeout or abort.
__device__ __forceinline__ bool persist_wait(const int* p, int want, DevState* st,
                                             unsigned long long t0) {
  for (;;) {
    if (ld_acquire(p) >= want) return true;
    if (ld_acquire(&st->flags) & FLAG_TIMEOUT) return false;
    if (globaltimer_ns() - t0 > PERSIST_WAIT_NS) return false;
  }
}

// The t-th plane of the intervals [lo - r, hi + r] (clipped to [kmin,
// kmax]) taken in turn, or -1 past their end.
__device__ __forceinline__ int persist_plane_at(const int* iv, int nint, int r, int kmin,
                                                int kmax, int t) {
  for (int q = 0; q < nint; ++q) {
    const int lo = iv[2 * q], hi = iv[2 * q + 1];
    if (lo > hi) continue;
    const int a = max(lo - r, kmin), b = min(hi + r, kmax);
    if (a > b) continue;
    if (t <= b - a) return a + t;
    t -= b - a + 1;
  }
  return -1;
}

__device__ __forceinline__ void persist_abort(DevState* st) {
  atomicOr(&st->flags, FLAG_TIMEOUT);
  atomicExch(&st->status, ST_TIMEOUT);
}

// The whole CTA: wait for the counters of planes [lo - r, hi + r] (clipped
// to [kmin, kmax]) of every interval to reach touch x phases, one thread
// per plane (a second round of planes per thread where there are more
// planes than threads); true for every thread when all are reached.
__device__ __forceinline__ bool persist_wait_planes(const int* iv, int nint, int r, int kmin,
                                                    int kmax, const int* cnt, const int* touch,
                                                    int phases, DevState* st) {
  const unsigned long long t0 = globaltimer_ns();
  bool ok = true;
  for (int t = threadIdx.x;; t += blockDim.x) {
    const int p = persist_plane_at(iv, nint, r, kmin, kmax, t);
    if (p < 0) break;
    ok = ok && persist_wait(&cnt[p], touch[p] * phases, st, t0);
  }
  return __syncthreads_and(ok);
}

// The whole CTA, after its pass: one completion for every plane of every
// interval, one thread per plane, each after a device-scope fence (the
// barrier before it makes the CTA's writes part of what the fence orders).
__device__ __forceinline__ void persist_publish(const int* iv, int nint, int* cnt) {
  __syncthreads();
  for (int t = threadIdx.x;; t += blockDim.x) {
    const int p = persist_plane_at(iv, nint, 0, 0, 1 << 30, t);
    if (p < 0) break;
    __threadfence();
    atomicAdd(&cnt[p], 1);
  }
}

template <int CURL>
__global__ void __launch_bounds__(256, CURL == 2 ? 2 : 4)
    k_attempts_persist(const SplitArgs a, const PersistArgs pa) {
  __shared__ double red[8];
  __shared__ double sh[96];
  __shared__ int ok, last;
  DevState* st = a.st;
  const int G = gridDim.x;
  const int* ivB = pa.ivB + blockIdx.x * 2 * PERSIST_BI;
  const int* ivC = pa.ivC + blockIdx.x * 2;
  for (int att = 0; att < pa.n_attempts; ++att) {
    if (LdL2::ldi(&st->status) != ST_OK ||
        __ldcg(&st->n_accept) >= __ldcg(&st->target))
      return;
    const int cur = LdL2::ldi(&st->cur);
#define GLEMUR_PERSIST_STAGE(SS)                                                          \
    if (SS > 0 && !persist_wait_planes(ivB, PERSIST_BI, 2, 1, a.nz - 2, pa.cntC,          \
                                       pa.touchC, att * 6 + SS, st)) {                    \
      if (threadIdx.x == 0) persist_abort(st);                                            \
      return;                                                                             \
    }                                                                                     \
    pass_B<SS, LdL2>(a, cur, red);                                                        \
    if (!(SS == 2 && (int)blockIdx.x == pa.test_withhold))                                \
      persist_publish(ivB, PERSIST_BI, pa.cntB);                                          \
    if (!persist_wait_planes(ivC, 1, 1, 0, a.nz - 1, pa.cntB, pa.touchB,                  \
                             att * 6 + SS + 1, st)) {                                     \
      if (threadIdx.x == 0) persist_abort(st);                                            \
      return;                                                                             \
    }                                                                                     \
    pass_C<SS, CURL, LdL2>(a, cur, red);                                                  \
    persist_publish(ivC, 1, pa.cntC);
    GLEMUR_PERSIST_STAGE(0)
    GLEMUR_PERSIST_STAGE(1)
    GLEMUR_PERSIST_STAGE(2)
    GLEMUR_PERSIST_STAGE(3)
    GLEMUR_PERSIST_STAGE(4)
    GLEMUR_PERSIST_STAGE(5)
#undef GLEMUR_PERSIST_STAGE
    // end of the attempt: the last CTA to arrive runs the step control
    if (threadIdx.x == 0) {
      __threadfence();
      const unsigned old = atomicAdd(&pa.bar[0], 1u);
      last = old == (unsigned)(G * (att + 1) - 1);
    }
    __syncthreads();
    if (last) {
      __threadfence();
      control_block<LdCoherent>(st, a.part, a.nblocks, a.diag, pa.dtlog, sh);
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        atomicExch(&pa.bar[1], (unsigned)(att + 1));
      }
    } else {
      if (threadIdx.x == 0) {
        const unsigned long long t0 = globaltimer_ns();
        ok = 1;
        while (ld_acquire(&pa.bar[1]) < (unsigned)(att + 1)) {
          if ((ld_acquire(&st->flags) & FLAG_TIMEOUT) ||
              globaltimer_ns() - t0 > PERSIST_WAIT_NS) {
            ok = 0;
            break;
          }
        }
        __threadfence();
      }
      __syncthreads();
      if (!ok) {
        if (threadIdx.x == 0) persist_abort(st);
        return;
      }
    }
    __syncthreads();
  }
}

// CTAs of 256 threads per SM the persistent kernel can hold, and its launch
// (cooperative: every CTA resident, or the launch fails).
int persist_ctas_per_sm(int curl) {
  int n = 0;
  if (curl == 2)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_attempts_persist<2>, 256, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_attempts_persist<0>, 256, 0);
  return n;
}

cudaError_t launch_f64_persist(const SplitArgs& a, const PersistArgs& pa, int grid, int curl,
                               cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  if (curl == 2) return cudaLaunchKernelEx(&cfg, k_attempts_persist<2>, a, pa);
  return cudaLaunchKernelEx(&cfg, k_attempts_persist<0>, a, pa);
}

// CTAs of 256 threads per SM that pass B and pass C of each stage can hold
// (pass C with the current `curl`: 0 nearest, 2 next-nearest neighbours).
void split_ctas_per_sm(int b[6], int c[6], int curl) {
  void (*kb[6])(const SplitArgs) = {k_split_B<0>, k_split_B<1>, k_split_B<2>,
                                    k_split_B<3>, k_split_B<4>, k_split_B<5>};
  void (*kc0[6])(const SplitArgs) = {k_split_C<0, 0>, k_split_C<1, 0>, k_split_C<2, 0>,
                                     k_split_C<3, 0>, k_split_C<4, 0>, k_split_C<5, 0>};
  void (*kc2[6])(const SplitArgs) = {k_split_C<0, 2>, k_split_C<1, 2>, k_split_C<2, 2>,
                                     k_split_C<3, 2>, k_split_C<4, 2>, k_split_C<5, 2>};
  void (**kc)(const SplitArgs) = curl == 2 ? kc2 : kc0;
  for (int s = 0; s < 6; ++s) {
    b[s] = c[s] = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b[s], kb[s], 256, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c[s], kc[s], 256, 0);
    if (b[s] < 1) b[s] = 1;
    if (c[s] < 1) c[s] = 1;
  }
}

// Launch both passes of stage s (grid_b[s], grid_c[s] CTAs of 256 threads)
// with the current `curl` (0 nearest, 2 next-nearest neighbours).
cudaError_t launch_f64_split(const SplitArgs& a, int stage, cudaStream_t s, int curl) {
  if (stage < 0 || stage > 5 || (curl != 0 && curl != 2)) return cudaErrorInvalidValue;
  const dim3 gb(a.grid_b[stage]), gc(a.grid_c[stage]);
  cudaError_t e = cudaSuccess;
#define GLEMUR_SPLIT_CASE(SS)                                                          \
  case SS:                                                                             \
    e = launch_pdl(k_split_B<SS>, gb, dim3(256), 0, s, a);                             \
    if (e == cudaSuccess)                                                              \
      e = curl == 2 ? launch_pdl(k_split_C<SS, 2>, gc, dim3(256), 0, s, a)             \
                    : launch_pdl(k_split_C<SS, 0>, gc, dim3(256), 0, s, a);            \
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
