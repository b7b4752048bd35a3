// Fused Cash-Karp stage kernels for the Lagrangian magneto-frictional step.
//
// One launch evaluates one Runge-Kutta stage k_s = u(x_s) at every interior
// node (section "Time Stepping"; eq. "x integration" with u = J x B of eq.
// "magneto friction").  Per CTA: a TX x TY column tile that marches along z.
// Each z-plane of the stage input x_s = x + dt sum_{j<s} a_sj k_j is formed
// once in shared memory (tile + halo), B = G B0s / det G (eq. "B
// transformation", index-space form, see glemur_dev.cuh) is formed once per
// node of the tile + halo 1, and the current and velocity are evaluated at
// the tile's own nodes.  The last stage also forms the fifth-order update
// and the embedded error, and reduces the CTA's max error (the Lambda of eq.
// "time stepping").
//
// Mimetic current (section "Mimetic Operators").  With the index-space
// differences g_a = x(m + e_a) - x(m - e_a) and P_a = B(m + e_a) - B(m - e_a)
// the loop of eq. "current discrete" through the neighbours +e_p, +e_q, -e_p,
// -e_q has circulation (P_p . g_q - P_q . g_p) / 2 and the vector area of
// eq. "sum of triangles" is (g_p x g_q) / 2.  The three loop equations of
// eq. "current matrix equation", J . (g_p x g_q) = P_p . g_q - P_q . g_p for
// (p, q) = (1, 2), (2, 0), (0, 1), have the matrix of rows g_p x g_q =
// det(G) G^-1, so their solution is J = (c_0 g_0 + c_1 g_1 + c_2 g_2) / det G
// with c_r the right-hand sides: the same J as the paper's loop form, with
// no 3x3 solve and det G the one the pull-back already needs.
//
// Pipeline (mimetic kernel).  Stage s reads its input y_s (written pointwise
// by stage s-1; y_0 = x) with halos, and writes k_s and, at its own nodes,
// the next input y_{s+1} = d + sum_{j<=s} dt a_{s+1,j} k_j -- so the halo
// tiles carry one field, and the combine runs once per node.  Shared memory
// holds a ring of 6 planes of y_s and a ring of 4 planes of B.  Iteration m
// computes B at plane m+2, the current at plane m and loads plane m+4 of
// y_s: the three touch disjoint ring slots, so one barrier per plane
// suffices.  The global loads of y (plane m+4), of B0 (plane m+3) and of the
// centre values for y_{s+1} (plane m) are issued ahead of the arithmetic
// that hides their latency.
//
// Direct current (the classic method).  dB/dX follows from B = G B0s / det G
// by the product rule with second differences of x, differences of B0s and
// Jacobi's formula for d det G; dB/dx = dB/dX G^-1 (index-space scaling
// cancels) and J = curl_x B.
#pragma once

#include "glemur_dev.cuh"
#include "tma.cuh"

namespace glemur {

// ------------------------------------------------------------ arithmetic

// Determinant of G = [g0 g1 g2] (columns).
__device__ __forceinline__ double det3(const double g0[3], const double g1[3],
                                       const double g2[3]) {
  double m0 = g1[1] * g2[2] - g1[2] * g2[1];
  double m1 = g1[2] * g2[0] - g1[0] * g2[2];
  double m2 = g1[0] * g2[1] - g1[1] * g2[0];
  return g0[0] * m0 + g0[1] * m1 + g0[2] * m2;
}

// Error-free transformations on float (Dekker / Knuth): a*b = p + e and
// a + b = s + e exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Determinant of float columns carried in float-float (about 44 significant
// bits) and rounded once: each product of two entries is exact as a float
// pair, each 2x2 minor and the final sum are compensated.  This keeps the
// determinant at better than FP32 accuracy on the FP32 pipes; GB300's FP64
// rate is 1/62 of its FP32 rate, so an FP64 determinant would bound the
// mixed-precision stage.
__device__ __forceinline__ float det3(const float g0[3], const float g1[3],
                                      const float g2[3]) {
  float th[3], tl[3];
  const int ia[3] = {1, 2, 0}, ib[3] = {2, 0, 1};
#pragma unroll
  for (int r = 0; r < 3; ++r) {
    float p, pe, q, qe, s, se;
    two_prod(g1[ia[r]], g2[ib[r]], p, pe);
    two_prod(g1[ib[r]], g2[ia[r]], q, qe);
    two_sum(p, -q, s, se);
    float lo = se + (pe - qe);
    float t, te;
    two_prod(g0[r], s, t, te);
    te = fmaf(g0[r], lo, te);
    th[r] = t;
    tl[r] = te;
  }
  float s01, e01, s, e2;
  two_sum(th[0], th[1], s01, e01);
  two_sum(s01, th[2], s, e2);
  float lo = ((tl[0] + tl[1]) + tl[2]) + (e01 + e2);
  return s + lo;
}

template <typename C>
__device__ __forceinline__ C dot3(const C a[3], const C b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// 1/det.  FP64: Newton-Raphson refinement of the hardware approximation
// rcp.approx.ftz.f64, y <- y + y (1 - v y): each step squares the relative
// error (the classical iteration for reciprocals, e.g. Muller et al.,
// Handbook of Floating-Point Arithmetic, ch. on Newton-Raphson division),
// so two steps take the approximation to within an ulp or two of the
// correctly rounded 1/v in 4 FMAs, where the IEEE division costs about 12
// FP64-pipe instructions -- a quarter of the FP64 work of forming B.  NaN
// propagates; 0 and subnormal v give NaN or inf, and every caller has
// already flagged det <= 0.  In mixed precision the determinant is already
// carried beyond FP32 and the reciprocal only scales FP32 data, so the fast
// FP32 reciprocal (about 2 ulp) is used.
__device__ __forceinline__ double recip(double v) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(v));
  double e = fma(-v, y, 1.0);
  y = fma(y, e, y);
  e = fma(-v, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ float recip(float v) { return __fdividef(1.0f, v); }

__device__ __forceinline__ float nanmaxf_(float a, float b) {
  return (a > b || a != a) ? a : b;
}

template <typename C>
__device__ __forceinline__ C coef_a(const DevState* st, int s, int j);
template <>
__device__ __forceinline__ double coef_a<double>(const DevState* st, int s, int j) {
  return st->dta[s][j];
}
template <>
__device__ __forceinline__ float coef_a<float>(const DevState* st, int s, int j) {
  return st->dtaf[s][j];
}
template <typename C>
__device__ __forceinline__ C coef_b(const DevState* st, int j);
template <>
__device__ __forceinline__ double coef_b<double>(const DevState* st, int j) {
  return st->dtb[j];
}
template <>
__device__ __forceinline__ float coef_b<float>(const DevState* st, int j) {
  return st->dtbf[j];
}
template <typename C>
__device__ __forceinline__ C coef_e(const DevState* st, int j);
template <>
__device__ __forceinline__ double coef_e<double>(const DevState* st, int j) {
  return st->dte[j];
}
template <>
__device__ __forceinline__ float coef_e<float>(const DevState* st, int j) {
  return st->dtef[j];
}

template <typename T, typename C>
__device__ __forceinline__ C h2of(const StageArgs<T>& a, int i);
template <>
__device__ __forceinline__ double h2of<double, double>(const StageArgs<double>& a, int i) {
  return a.h2[i];
}
template <>
__device__ __forceinline__ float h2of<float, float>(const StageArgs<float>& a, int i) {
  return a.h2f[i];
}

// ------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = nanmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Deterministic block reduction (fixed tree); result valid in thread 0.
template <bool MAX>
__device__ __forceinline__ double block_reduce(double v, double* sh) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = MAX ? warp_max(v) : warp_sum(v);
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (w == 0) {
    v = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0.0;
    v = MAX ? warp_max(v) : warp_sum(v);
  }
  return v;
}

// Per-thread accumulators of the diagnostic and error reductions, reduced
// per CTA in FP64.  FP64 mode accumulates in double; mixed precision keeps
// the energy sum as a compensated float pair (error-free additions) and the
// maxima in float, so no per-node work lands on the FP64 pipe.
template <typename C>
struct Acc;
//
// The force-free maxima xi^2 = max |J x B|^2 / |B|^4 and xi'^2 = max
// |J x B|^2 / (|J|^2 |B|^2): FP64 keeps the largest ratio as its numerator
// and denominator and compares by cross-multiplication (a > n/d as
// a d > n b), dividing once per thread at the end -- an FP64 division per
// node, taken whenever a thread's maximum grows, cost a fifth of the first
// stage's FP64 work.  (The products overflow only for |B| beyond ~1e50.)
// FP32 keeps the ratio.
template <>
struct Acc<double> {
  double e = 0.0, lam = 0.0;
  double xn = 0.0, xd = 1.0, sn = 0.0, sd = 1.0;  // xi^2 = xn / xd, xi'^2 = sn / sd
  int bad = 0;
  __device__ __forceinline__ void add_e(double w) { e += w; }
  __device__ __forceinline__ void max_lam(double v) { lam = nanmax(lam, v); }
  __device__ __forceinline__ double e_total() const { return e; }
  // one node: u2 = |J x B|^2, b2 = |B|^2, j2 = |J|^2 (NaN u2 propagates)
  __device__ __forceinline__ void max_xi(double u2, double b2, double j2) {
    const double b4 = b2 * b2;
    if (gt_nonneg(u2 * xd, xn * b4)) {
      xn = u2;
      xd = b4;
    }
    const double jb = j2 * b2;
    if (gt_nonneg(jb, 0.0) && gt_nonneg(u2 * sd, sn * jb) && not_nan(u2)) {
      sn = u2;
      sd = jb;
    }
  }
  __device__ __forceinline__ double xi2() const { return xn / xd; }
  __device__ __forceinline__ double xis2() const { return sn / sd; }
};
template <>
struct Acc<float> {
  float eh = 0.0f, el = 0.0f, lam = 0.0f, x2 = 0.0f, s2 = 0.0f;
  int bad = 0;
  __device__ __forceinline__ void add_e(float w) {
    float s, err;
    two_sum(eh, w, s, err);
    eh = s;
    el += err;
  }
  __device__ __forceinline__ void max_lam(float v) { lam = nanmaxf_(lam, v); }
  __device__ __forceinline__ double e_total() const { return (double)eh + (double)el; }
  __device__ __forceinline__ void max_xi(float u2, float b2, float j2) {
    if (gt_nonneg(u2, x2 * b2 * b2)) x2 = u2 / (b2 * b2);
    const float jb = j2 * b2;
    if (gt_nonneg(jb, 0.0f) && gt_nonneg(u2, s2 * jb) && not_nan(u2)) s2 = u2 / jb;
  }
  __device__ __forceinline__ double xi2() const { return x2; }
  __device__ __forceinline__ double xis2() const { return s2; }
};

// ------------------------------------------------------------ x_s planes

// One shared-memory point of the mimetic kernel's tiles: (x, y, z, pad) of
// the stage input, or (B_x, B_y, B_z, 1/det G); a single 16-byte (float) or
// two 16-byte (double) shared loads fetch a stencil neighbour.
template <typename C>
struct alignas(4 * sizeof(C)) V4 {
  C x, y, z, w;
};

// The shared-memory points of a W x H tile (+halo) that this thread loads:
// LP slots, each the in-plane offset gj*nx + gi of the node, or -1.
template <int W, int H, int HALO>
struct LoadPts {
  static constexpr int LP = (W * H + NT - 1) / NT;
  int off[LP];
  __device__ __forceinline__ void init(int i0, int j0, int nx, int ny) {
#pragma unroll
    for (int t = 0; t < LP; ++t) {
      const int p = threadIdx.x + t * NT;
      off[t] = -1;
      if (p < W * H) {
        const int gi = i0 - HALO + p % W, gj = j0 - HALO + p / W;
        if (gi >= 0 && gi < nx && gj >= 0 && gj < ny) off[t] = gj * nx + gi;
      }
    }
  }
};

// One plane of the stage input y at the thread's points of a halo-1 tile,
// held in registers between issue and commit, stored as three scalar planes
// (component-major, pitch PITCH) for the direct current.
template <typename T, typename C, int LP>
struct PlaneSoA {
  C v[LP][3];
  __device__ __forceinline__ void issue(const T* __restrict__ y, int N, int nxy, const int* off,
                                        int q) {
    const int base = q * nxy;
#pragma unroll
    for (int t = 0; t < LP; ++t) {
      if (off[t] < 0) continue;
      const int n = base + off[t];
#pragma unroll
      for (int c = 0; c < 3; ++c) v[t][c] = (C)__ldg(&y[c * N + n]);
    }
  }
  template <int PITCH>
  __device__ __forceinline__ void commit(const int* off, C* __restrict__ dst) const {
#pragma unroll
    for (int t = 0; t < LP; ++t) {
      if (off[t] < 0) continue;
      const int p = threadIdx.x + t * NT;
#pragma unroll
      for (int c = 0; c < 3; ++c) dst[c * PITCH + p] = v[t][c];
    }
  }
};

// One plane of a single displacement-like field (the stage input y) at the
// thread's tile points, held in registers between issue and commit.
template <typename T, typename C, int LP>
struct YPlane {
  C v[LP][3];
  __device__ __forceinline__ void issue(const T* __restrict__ y, int N, int nxy, const int* off,
                                        int q) {
    const int base = q * nxy;
#pragma unroll
    for (int t = 0; t < LP; ++t) {
      if (off[t] < 0) continue;
      const int n = base + off[t];
#pragma unroll
      for (int c = 0; c < 3; ++c) v[t][c] = (C)__ldg(&y[c * N + n]);
    }
  }
  __device__ __forceinline__ void commit(const int* off, V4<C>* __restrict__ dst) const {
#pragma unroll
    for (int t = 0; t < LP; ++t)
      if (off[t] >= 0) dst[threadIdx.x + t * NT] = V4<C>{v[t][0], v[t][1], v[t][2], (C)0};
  }
};

// Centre values a stage output needs at its node: d and the k_j of the next
// stage input (stage S < 5: k_0..k_{S-1}), or of the update and error
// (S = 5: k1, k3, k4, k5).
template <typename T, typename C, int S>
struct Centre {
  static constexpr int NK = S == 5 ? 4 : S;
  C d[3];
  C k[NK > 0 ? NK : 1][3];
  __device__ __forceinline__ static int kidx(int j) { return S == 5 ? (j == 0 ? 0 : j + 1) : j; }
  __device__ __forceinline__ void issue(const StageArgs<T>& a, const T* __restrict__ dsrc, int N,
                                        int n) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      d[c] = (C)__ldg(&dsrc[c * N + n]);
#pragma unroll
      for (int j = 0; j < NK; ++j) k[j][c] = (C)__ldg(&a.k[kidx(j)][c * N + n]);
    }
  }
};

// ------------------------------------------------------------ mimetic

// The B-tile points this thread computes (tile + halo 1, at most BPT), with
// everything about them that does not change from plane to plane: the x
// tile index, the in-plane node offset, the x/y stencil (0 central, 1 lower
// face, 2 upper face), whether the node is the tile's own (energy sum), and
// how many of its x/y index coordinates lie on the boundary (zeta).
struct BPts {
  static constexpr int BPT = (BP + NT - 1) / NT;
  int x0[BPT], nxy[BPT], code[BPT];
  __device__ __forceinline__ void init(int i0, int j0, int nx, int ny) {
#pragma unroll
    for (int t = 0; t < BPT; ++t) {
      const int p = threadIdx.x + t * NT;
      x0[t] = -1;
      nxy[t] = 0;
      code[t] = 0;
      if (p >= BP) continue;
      const int bx = p % BW, by = p / BW;
      const int gi = i0 - 1 + bx, gj = j0 - 1 + by;
      if (gi < 0 || gi >= nx || gj < 0 || gj >= ny) continue;
      x0[t] = (by + 1) * XW + (bx + 1);
      nxy[t] = gj * nx + gi;
      const int sx = gi == 0 ? 1 : (gi == nx - 1 ? 2 : 0);
      const int sy = gj == 0 ? 1 : (gj == ny - 1 ? 2 : 0);
      const int own = bx >= 1 && bx <= TX && by >= 1 && by <= TY;
      code[t] = sx | (sy << 2) | (own << 4) | (((sx != 0) + (sy != 0)) << 5);
    }
  }
};

constexpr int XRING = 6;  // planes of x_s in shared memory
constexpr int BRING = 4;  // planes of B (+ 1/det G) in shared memory

__device__ __forceinline__ int xslot(int q) { return (q + XRING) % XRING; }
__device__ __forceinline__ int bslot(int q) { return (q + BRING) % BRING; }

// B (and 1/det G) at every node of plane q in the tile + halo 1.  Index-space
// differences: central inside, second-order one-sided on boundary faces.
template <typename C>
__device__ __forceinline__ void vsub(const V4<C>& a, const V4<C>& b, C o[3]) {
  o[0] = a.x - b.x;
  o[1] = a.y - b.y;
  o[2] = a.z - b.z;
}
// one-sided second-order difference 4 p1 - 3 p0 - p2 (lower face; the upper
// face is its negative with p1, p2 the inner neighbours)
template <typename C>
__device__ __forceinline__ void vside(const V4<C>& p0, const V4<C>& p1, const V4<C>& p2, C sgn,
                                      C o[3]) {
  o[0] = sgn * (((C)4 * p1.x - (C)3 * p0.x) - p2.x);
  o[1] = sgn * (((C)4 * p1.y - (C)3 * p0.y) - p2.y);
  o[2] = sgn * (((C)4 * p1.z - (C)3 * p0.z) - p2.z);
}

template <typename C>
struct B0Pts {
  C v[BPts::BPT][3];
};

// B0s at the thread's B points of plane q.
template <typename T, typename C>
__device__ __forceinline__ void load_B0(const StageArgs<T>& a, int q, const BPts& bp,
                                        B0Pts<C>& out) {
  const int N = a.nx * a.ny * a.nz;
  const int nq = q * a.nx * a.ny;
#pragma unroll
  for (int t = 0; t < BPts::BPT; ++t) {
    if (bp.x0[t] < 0) continue;
    const int n = nq + bp.nxy[t];
#pragma unroll
    for (int c = 0; c < 3; ++c) out.v[t][c] = (C)__ldg(&a.B0s[c * N + n]);
  }
}

template <typename T, typename C>
__device__ __forceinline__ void compute_B(const StageArgs<T>& a, int q, int k0, int k1,
                                          const BPts& bp, const B0Pts<C>& b0v,
                                          const V4<C>* __restrict__ xs,
                                          V4<C>* __restrict__ bs, bool diag, bool state,
                                          Acc<C>& acc) {
  const V4<C>* xq = xs + xslot(q) * XP;
  const V4<C>* xm = xs + xslot(q - 1) * XP;
  const V4<C>* xp = xs + xslot(q + 1) * XP;
  const V4<C>* xm2 = xs + xslot(q - 2) * XP;
  const V4<C>* xp2 = xs + xslot(q + 2) * XP;
  V4<C>* bq = bs + bslot(q) * BP;
  const C h20 = h2of<T, C>(a, 0), h21 = h2of<T, C>(a, 1), h22 = h2of<T, C>(a, 2);
  const int sz = q == 0 ? 1 : (q == a.nz - 1 ? 2 : 0);
  const bool own_plane = diag && q >= k0 && q < k1;
#pragma unroll
  for (int t = 0; t < BPts::BPT; ++t) {
    const int x0 = bp.x0[t];
    if (x0 < 0) continue;
    const int p = threadIdx.x + t * NT;
    const int code = bp.code[t];
    const int sx = code & 3, sy = (code >> 2) & 3;
    C g[3][3];
    if (sx == 0)
      vsub(xq[x0 + 1], xq[x0 - 1], g[0]);
    else if (sx == 1)
      vside(xq[x0], xq[x0 + 1], xq[x0 + 2], (C)1, g[0]);
    else
      vside(xq[x0], xq[x0 - 1], xq[x0 - 2], (C)-1, g[0]);
    if (sy == 0)
      vsub(xq[x0 + XW], xq[x0 - XW], g[1]);
    else if (sy == 1)
      vside(xq[x0], xq[x0 + XW], xq[x0 + 2 * XW], (C)1, g[1]);
    else
      vside(xq[x0], xq[x0 - XW], xq[x0 - 2 * XW], (C)-1, g[1]);
    if (sz == 0)
      vsub(xp[x0], xm[x0], g[2]);
    else if (sz == 1)
      vside(xq[x0], xp[x0], xp2[x0], (C)1, g[2]);
    else
      vside(xq[x0], xm[x0], xm2[x0], (C)-1, g[2]);
    g[0][0] += h20;
    g[1][1] += h21;
    g[2][2] += h22;
    const C det = det3(g[0], g[1], g[2]);
    if (le_zero(det))  // NaN: reported by the error norm
      atomicOr(&a.st->flags, state ? FLAG_COLLAPSED : FLAG_FOLDED_TRIAL);
    const C r = recip(det);
    const C b0 = b0v.v[t][0], b1 = b0v.v[t][1], b2 = b0v.v[t][2];
    C B[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) B[c] = (g[0][c] * b0 + g[1][c] * b1 + g[2][c] * b2) * r;
    bq[p] = V4<C>{B[0], B[1], B[2], r};
    if (own_plane && (code & 16)) {
      // eq. "magnetic energy": zeta halves per boundary index coordinate
      const int nb = ((code >> 5) & 3) + (sz != 0);
      const C zeta = nb == 0 ? (C)1 : nb == 1 ? (C)0.5 : nb == 2 ? (C)0.25 : (C)0.125;
      acc.add_e(zeta * dot3(B, B) * det);
    }
  }
}

// Stage-S output at node n from its centre values: k_S and the next stage
// input, or (S = 5) the update, the error and (optionally) k6.
template <typename T, typename C, int S>
__device__ __forceinline__ void emit_centre(const StageArgs<T>& a, int n, const C u[3],
                                            const C J[3], const C B[3],
                                            const Centre<T, C, S>& ce, T* __restrict__ dout,
                                            const C* an, const DevState* st, bool diag,
                                            Acc<C>& acc) {
  const int N = a.nx * a.ny * a.nz;
  if (diag) {
    // xi^2 = |J x B|^2 / |B|^4 and the sine form |J x B|^2 / (|J|^2 |B|^2)
    acc.max_xi(dot3(u, u), dot3(B, B), dot3(J, J));
  }
  if constexpr (S < 5) {
    T* ko = a.k[S];
    T* ynext = a.ys[(S + 1) & 1];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      ko[c * N + n] = (T)u[c];
      C v = ce.d[c];
#pragma unroll
      for (int j = 0; j < S; ++j) v = fma(an[j], ce.k[j][c], v);
      ynext[c * N + n] = (T)fma(an[S], u[c], v);
    }
  } else {
    // fifth-order update (b_2 = b_5 = 0) and embedded error (b_2 - b*_2 = 0)
    const C b0 = coef_b<C>(st, 0), b2 = coef_b<C>(st, 2), b3 = coef_b<C>(st, 3),
            b5 = coef_b<C>(st, 5);
    const C e0 = coef_e<C>(st, 0), e2 = coef_e<C>(st, 2), e3 = coef_e<C>(st, 3),
            e4 = coef_e<C>(st, 4), e5 = coef_e<C>(st, 5);
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const C k1 = ce.k[0][c], k3 = ce.k[1][c], k4 = ce.k[2][c], k5 = ce.k[3][c];
      C up = b0 * k1;
      up = fma(b2, k3, up);
      up = fma(b3, k4, up);
      up = fma(b5, u[c], up);
      C er = e0 * k1;
      er = fma(e2, k3, er);
      er = fma(e3, k4, er);
      er = fma(e4, k5, er);
      er = fma(e5, u[c], er);
      dout[c * N + n] = (T)(ce.d[c] + up);
      acc.max_lam(fabs(er));
      if (a.k6) a.k6[c * N + n] = (T)u[c];
    }
  }
}

// Mimetic current and velocity at the thread's node (gi, gj) of plane m.
template <typename T, typename C, int S>
__device__ __forceinline__ void mimetic_out(const StageArgs<T>& a, int m, int n,
                                            const V4<C>* __restrict__ xs,
                                            const V4<C>* __restrict__ bs,
                                            const Centre<T, C, S>& ce, T* dout, const C* an,
                                            const DevState* st, bool diag, Acc<C>& acc) {
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int x0 = (ty + 2) * XW + (tx + 2);
  const int b0i = (ty + 1) * BW + (tx + 1);
  const V4<C>* xq = xs + xslot(m) * XP;
  const V4<C>* xm = xs + xslot(m - 1) * XP;
  const V4<C>* xp = xs + xslot(m + 1) * XP;
  const V4<C>* bq = bs + bslot(m) * BP;
  const V4<C>* bm = bs + bslot(m - 1) * BP;
  const V4<C>* bp = bs + bslot(m + 1) * BP;
  C g0[3], g1[3], g2[3], P0[3], P1[3], P2[3];
  vsub(xq[x0 + 1], xq[x0 - 1], g0);
  vsub(xq[x0 + XW], xq[x0 - XW], g1);
  vsub(xp[x0], xm[x0], g2);
  vsub(bq[b0i + 1], bq[b0i - 1], P0);
  vsub(bq[b0i + BW], bq[b0i - BW], P1);
  vsub(bp[b0i], bm[b0i], P2);
  const V4<C> bc = bq[b0i];
  const C B[3] = {bc.x, bc.y, bc.z};
  g0[0] += h2of<T, C>(a, 0);
  g1[1] += h2of<T, C>(a, 1);
  g2[2] += h2of<T, C>(a, 2);
  const C c0 = dot3(P1, g2) - dot3(P2, g1);
  const C c1 = dot3(P2, g0) - dot3(P0, g2);
  const C c2 = dot3(P0, g1) - dot3(P1, g0);
  const C r = bc.w;
  C J[3], u[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) J[c] = (c0 * g0[c] + c1 * g1[c] + c2 * g2[c]) * r;
  u[0] = J[1] * B[2] - J[2] * B[1];
  u[1] = J[2] * B[0] - J[0] * B[2];
  u[2] = J[0] * B[1] - J[1] * B[0];
  emit_centre<T, C, S>(a, n, u, J, B, ce, dout, an, st, diag, acc);
}

template <typename T, typename C>
__device__ __forceinline__ void write_partials(const StageArgs<T>& a, bool final_stage,
                                               bool diag, Acc<C>& acc, double* red) {
  const int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
  if (final_stage) {
    const double v = block_reduce<true>((double)acc.lam, red);
    if (threadIdx.x == 0) a.part[PART_LAMBDA * a.nblocks + bid] = v;
  }
  if (diag) {
    double v = block_reduce<false>(acc.e_total(), red);
    if (threadIdx.x == 0) a.part[PART_E * a.nblocks + bid] = v;
    v = block_reduce<true>(acc.xi2(), red);
    if (threadIdx.x == 0) a.part[PART_XI2 * a.nblocks + bid] = v;
    v = block_reduce<true>(acc.xis2(), red);
    if (threadIdx.x == 0) a.part[PART_XIS2 * a.nblocks + bid] = v;
  }
}

// Stage S (0..5) of Cash-Karp with the mimetic current.
template <typename T, typename C, int S, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_stage_mimetic(const StageArgs<T> a) {
  constexpr bool FINAL = S == 5;
  pdl_wait();
  const DevState* st = a.st;
  if (!a.force && (st->status != ST_OK || st->n_accept >= st->target)) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[NT / 32];
  V4<C>* xs = reinterpret_cast<V4<C>*>(smem_raw);  // [XRING][XP] (y_s, -)
  V4<C>* bs = xs + XRING * XP;                      // [BRING][BP] (B, 1/det G)
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * a.kz, k1 = min(a.nz, k0 + a.kz);
  const int N = a.nx * a.ny * a.nz, nxy = a.nx * a.ny;
  const int cur = st->cur;
  const T* d = a.d[cur];
  T* dout = const_cast<T*>(a.d[cur ^ 1]);
  const T* y = S == 0 ? d : a.ys[S & 1];
  C an[S < 5 ? S + 1 : 1];  // dt a_{S+1, j}: the next stage input
#pragma unroll
  for (int j = 0; j < (S < 5 ? S + 1 : 0); ++j) an[j] = coef_a<C>(st, S + 1, j);
  const bool diag = a.diag != 0;
  Acc<C> acc;
  LoadPts<XW, XH, 2> pts;
  pts.init(i0, j0, a.nx, a.ny);
  BPts bp;
  bp.init(i0, j0, a.nx, a.ny);
  using Y = YPlane<T, C, LoadPts<XW, XH, 2>::LP>;
  // the thread's own output column
  const int gi = i0 + threadIdx.x % TX, gj = j0 + threadIdx.x / TX;
  const bool out_xy = gi >= 1 && gi <= a.nx - 2 && gj >= 1 && gj <= a.ny - 2;
  const int nxy_out = gj * a.nx + gi;
  // prologue: input planes k0-2 .. k0+3, then B at k0-1 .. k0+1
  for (int q = k0 - 2; q <= k0 + 3; ++q) {
    if (q < 0 || q >= a.nz || q > k1 + 1) continue;
    Y yp;
    yp.issue(y, N, nxy, pts.off, q);
    yp.commit(pts.off, xs + xslot(q) * XP);
  }
  __syncthreads();
  for (int q = k0 - 1; q <= k0 + 1; ++q)
    if (q >= 0 && q < a.nz && q <= k1) {
      B0Pts<C> b0v;
      load_B0(a, q, bp, b0v);
      compute_B<T, C>(a, q, k0, k1, bp, b0v, xs, bs, diag, S == 0, acc);
    }
  B0Pts<C> b0cur;
  if (k0 + 2 < a.nz && k0 + 2 <= k1) load_B0(a, k0 + 2, bp, b0cur);
  __syncthreads();
  for (int m = k0; m < k1; ++m) {
    const int qn = m + 4;  // input plane loaded in this iteration
    const bool load = qn < a.nz && qn <= k1 + 1;
    const bool out = out_xy && m >= 1 && m <= a.nz - 2;
    const int n = m * nxy + nxy_out;
    Y yp;
    if (load) yp.issue(y, N, nxy, pts.off, qn);
    Centre<T, C, S> ce;
    if (out) ce.issue(a, d, N, n);
    const int qb = m + 2;  // B plane computed in this iteration
    if (qb < a.nz && qb <= k1)
      compute_B<T, C>(a, qb, k0, k1, bp, b0cur, xs, bs, diag, S == 0, acc);
    if (qb + 1 < a.nz && qb + 1 <= k1) load_B0(a, qb + 1, bp, b0cur);
    if (out) mimetic_out<T, C, S>(a, m, n, xs, bs, ce, dout, an, st, diag, acc);
    if (load) yp.commit(pts.off, xs + xslot(qn) * XP);
    __syncthreads();
  }
  pdl_trigger();
  write_partials<T, C>(a, FINAL, diag, acc, red);
}

// ------------------------------------------------------------ direct

// Direct current and velocity at the thread's node n (interior) of a plane:
// stage-input planes below, at and above it (xm, xq, xp; [3][DP] each).
template <typename T, typename C, int S>
__device__ __forceinline__ void direct_out(const StageArgs<T>& a, int n,
                                           const C* __restrict__ xm, const C* __restrict__ xq,
                                           const C* __restrict__ xp,
                                           const Centre<T, C, S>& ce, T* dout, const C* an,
                                           const DevState* st, bool diag, Acc<C>& acc) {
  const int tx = threadIdx.x % TX, ty = threadIdx.x / TX;
  const int N = a.nx * a.ny * a.nz;
  const int p0 = (ty + 1) * DW + (tx + 1);
  // columns g_a of G and the second differences S_ac = S_ca (index space)
  C g[3][3], Sd[3][3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const C* s = xq + c * DP;
    const C* sm = xm + c * DP;
    const C* sp = xp + c * DP;
    const C xc = s[p0];
    g[0][c] = s[p0 + 1] - s[p0 - 1];
    g[1][c] = s[p0 + DW] - s[p0 - DW];
    g[2][c] = sp[p0] - sm[p0];
    Sd[0][0][c] = (C)4 * ((s[p0 + 1] + s[p0 - 1]) - (C)2 * xc);
    Sd[1][1][c] = (C)4 * ((s[p0 + DW] + s[p0 - DW]) - (C)2 * xc);
    Sd[2][2][c] = (C)4 * ((sp[p0] + sm[p0]) - (C)2 * xc);
    Sd[0][1][c] = (s[p0 + 1 + DW] - s[p0 + 1 - DW]) - (s[p0 - 1 + DW] - s[p0 - 1 - DW]);
    Sd[0][2][c] = (sp[p0 + 1] - sm[p0 + 1]) - (sp[p0 - 1] - sm[p0 - 1]);
    Sd[1][2][c] = (sp[p0 + DW] - sm[p0 + DW]) - (sp[p0 - DW] - sm[p0 - DW]);
    Sd[1][0][c] = Sd[0][1][c];
    Sd[2][0][c] = Sd[0][2][c];
    Sd[2][1][c] = Sd[1][2][c];
  }
  g[0][0] += h2of<T, C>(a, 0);
  g[1][1] += h2of<T, C>(a, 1);
  g[2][2] += h2of<T, C>(a, 2);
  // B0s at the node and its differences D_c B0s = B0s(+e_c) - B0s(-e_c)
  const int sx = 1, sy = a.nx, sz = a.nx * a.ny;
  C b[3], Db[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* B0 = a.B0s + c * N;
    b[c] = (C)__ldg(&B0[n]);
    Db[0][c] = (C)__ldg(&B0[n + sx]) - (C)__ldg(&B0[n - sx]);
    Db[1][c] = (C)__ldg(&B0[n + sy]) - (C)__ldg(&B0[n - sy]);
    Db[2][c] = (C)__ldg(&B0[n + sz]) - (C)__ldg(&B0[n - sz]);
  }
  // cofactors of G: row i of cof is (row i+1 of G) x (row i+2 of G)
  C cof[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
    cof[i][0] = g[1][i1] * g[2][i2] - g[2][i1] * g[1][i2];
    cof[i][1] = g[2][i1] * g[0][i2] - g[0][i1] * g[2][i2];
    cof[i][2] = g[0][i1] * g[1][i2] - g[1][i1] * g[0][i2];
  }
  const C det = det3(g[0], g[1], g[2]);
  if (le_zero(det))  // NaN: reported by the error norm
    atomicOr(&a.st->flags, S == 0 ? FLAG_COLLAPSED : FLAG_FOLDED_TRIAL);
  const C r = recip(det);
  C V[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) V[i] = g[0][i] * b[0] + g[1][i] * b[1] + g[2][i] * b[2];
  // D_c B = D_c V / det - V D_c det / det^2, with
  // D_c V = sum_a S_ac b_a + g_a D_c b_a and D_c det = sum_ia cof_ia (S_ac)_i
  C DB[3][3];
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    C Dd = (C)0;
#pragma unroll
    for (int aa = 0; aa < 3; ++aa)
#pragma unroll
      for (int i = 0; i < 3; ++i) Dd = fma(cof[i][aa], Sd[aa][c][i], Dd);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      C DV = (C)0;
#pragma unroll
      for (int aa = 0; aa < 3; ++aa) DV = fma(Sd[aa][c][i], b[aa], fma(g[aa][i], Db[c][aa], DV));
      DB[c][i] = (DV - V[i] * Dd * r) * r;
    }
  }
  // grad B (gB[i][l] = dB_i/dx_l) = sum_c D_c B_i (G^-1)_cl, G^-1 = cof^T / det
  C gB[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int l = 0; l < 3; ++l)
      gB[i][l] = (DB[0][i] * cof[l][0] + DB[1][i] * cof[l][1] + DB[2][i] * cof[l][2]) * r;
  C J[3], B[3], u[3];
  J[0] = gB[2][1] - gB[1][2];
  J[1] = gB[0][2] - gB[2][0];
  J[2] = gB[1][0] - gB[0][1];
#pragma unroll
  for (int i = 0; i < 3; ++i) B[i] = V[i] * r;
  u[0] = J[1] * B[2] - J[2] * B[1];
  u[1] = J[2] * B[0] - J[0] * B[2];
  u[2] = J[0] * B[1] - J[1] * B[0];
  emit_centre<T, C, S>(a, n, u, J, B, ce, dout, an, st, diag, acc);
}

// Stage S (0..5) of Cash-Karp with the direct current.  Like the mimetic
// kernel, stage s reads only its input y_s on the tile (halo 1) and writes
// k_s and y_{s+1} pointwise.  Shared memory holds a ring of 4 planes of y_s
// ([3][DP] each): iteration m evaluates plane m from planes m-1 .. m+1 and
// loads plane m+2 (issued before, committed after the arithmetic).
template <typename T, typename C, int S, int MINB>
__global__ void __launch_bounds__(NT, MINB) k_stage_direct(const StageArgs<T> a) {
  constexpr bool FINAL = S == 5;
  pdl_wait();
  const DevState* st = a.st;
  if (!a.force && (st->status != ST_OK || st->n_accept >= st->target)) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ double red[NT / 32];
  C* xs = reinterpret_cast<C*>(smem_raw);  // [4 planes][3][DP]
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY;
  const int k0 = blockIdx.z * a.kz, k1 = min(a.nz, k0 + a.kz);
  const int N = a.nx * a.ny * a.nz, nxy = a.nx * a.ny;
  const int cur = st->cur;
  const T* d = a.d[cur];
  T* dout = const_cast<T*>(a.d[cur ^ 1]);
  const T* y = S == 0 ? d : a.ys[S & 1];
  C an[S < 5 ? S + 1 : 1];  // dt a_{S+1, j}: the next stage input
#pragma unroll
  for (int j = 0; j < (S < 5 ? S + 1 : 0); ++j) an[j] = coef_a<C>(st, S + 1, j);
  const bool diag = a.diag != 0;
  Acc<C> acc;
  LoadPts<DW, DH, 1> pts;
  pts.init(i0, j0, a.nx, a.ny);
  using Raw = PlaneSoA<T, C, LoadPts<DW, DH, 1>::LP>;
  const int gi = i0 + threadIdx.x % TX, gj = j0 + threadIdx.x / TX;
  const bool out_xy = gi >= 1 && gi <= a.nx - 2 && gj >= 1 && gj <= a.ny - 2;
  const int nxy_out = gj * a.nx + gi;
  for (int q = k0 - 1; q <= k0 + 1; ++q) {
    if (q < 0 || q >= a.nz || q > k1) continue;
    Raw raw;
    raw.issue(y, N, nxy, pts.off, q);
    raw.template commit<DP>(pts.off, xs + (q & 3) * 3 * DP);
  }
  __syncthreads();
  for (int m = k0; m < k1; ++m) {
    const int ql = m + 2;  // plane loaded in this iteration
    const bool load = ql < a.nz && ql <= k1;
    Raw raw;
    if (load) raw.issue(y, N, nxy, pts.off, ql);
    const bool out = out_xy && m >= 1 && m <= a.nz - 2;
    const int n = m * nxy + nxy_out;
    Centre<T, C, S> ce;
    if (out) {
      ce.issue(a, d, N, n);
      direct_out<T, C, S>(a, n, xs + ((m - 1) & 3) * 3 * DP, xs + (m & 3) * 3 * DP,
                          xs + ((m + 1) & 3) * 3 * DP, ce, dout, an, st, diag, acc);
    }
    if (load) raw.template commit<DP>(pts.off, xs + (ql & 3) * 3 * DP);
    __syncthreads();
  }
  pdl_trigger();
  write_partials<T, C>(a, FINAL, diag, acc, red);
}

// ------------------------------------------------------------ launchers

inline size_t stage_smem_bytes(int curl, size_t csize) {
  return curl == 0 ? (size_t)(XRING * XP + BRING * BP) * 4 * csize
                   : (size_t)(4 * 3 * DP) * csize;
}

// Launch stage `stage` (0..5) of the current `CURL` (0 mimetic, 1 direct).
template <typename T, typename C, int CURL, int MINB>
cudaError_t launch_stage_t(const StageArgs<T>& a, int stage, dim3 grid, cudaStream_t s) {
  const size_t smem = stage_smem_bytes(CURL, sizeof(C));
#define GLEMUR_STAGE_CASE(SS)                                                     \
  case SS:                                                                        \
    if constexpr (CURL == 0)                                                      \
      return launch_pdl(k_stage_mimetic<T, C, SS, MINB>, grid, dim3(NT), smem, s, a); \
    else                                                                          \
      return launch_pdl(k_stage_direct<T, C, SS, MINB>, grid, dim3(NT), smem, s, a);
  switch (stage) {
    GLEMUR_STAGE_CASE(0)
    GLEMUR_STAGE_CASE(1)
    GLEMUR_STAGE_CASE(2)
    GLEMUR_STAGE_CASE(3)
    GLEMUR_STAGE_CASE(4)
    GLEMUR_STAGE_CASE(5)
    default:
      return cudaErrorInvalidValue;
  }
#undef GLEMUR_STAGE_CASE
}

template <typename T, typename C, int CURL, int MINB>
cudaError_t prepare_stage_t() {
  const int sm = (int)stage_smem_bytes(CURL, sizeof(C));
  cudaError_t e = cudaSuccess;
#define GLEMUR_PREP(SS)                                                                  \
  if (e == cudaSuccess) {                                                                \
    if constexpr (CURL == 0)                                                             \
      e = cudaFuncSetAttribute(k_stage_mimetic<T, C, SS, MINB>,                          \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, sm);         \
    else                                                                                 \
      e = cudaFuncSetAttribute(k_stage_direct<T, C, SS, MINB>,                           \
                               cudaFuncAttributeMaxDynamicSharedMemorySize, sm);         \
  }
  GLEMUR_PREP(0)
  GLEMUR_PREP(1)
  GLEMUR_PREP(2)
  GLEMUR_PREP(3)
  GLEMUR_PREP(4)
  GLEMUR_PREP(5)
#undef GLEMUR_PREP
  return e;
}

template <typename T, typename C, int CURL, int MINB>
int stage_ctas_per_sm_t() {
  int n = 0;
  const size_t s = stage_smem_bytes(CURL, sizeof(C));
  if constexpr (CURL == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_mimetic<T, C, 3, MINB>, NT, s);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_stage_direct<T, C, 3, MINB>, NT, s);
  return n;
}

}  // namespace glemur
