// Hand-written adjoint (reverse mode) of the relaxation step, FP64.
//
// Forward (one Cash-Karp step of fixed size dt, section "Time Stepping"):
//   y_s = x + dt sum_{j<s} a_sj k_j,  k_s = f(y_s; B0),
//   x' = x + dt sum_j b_j k_j,
// with f(y)_n = J_n x B_n at interior nodes (eq. "magneto friction"),
// B = G B0s / det G at every node (eq. "B transformation" in index-space
// form), and the compact mimetic current J = (c_0 g_0 + c_1 g_1 + c_2 g_2) /
// det G, c_a = P_{a+1}.g_{a+2} - P_{a+2}.g_{a+1}, g_a and P_a the central
// differences of y and B (section "Mimetic Operators").
//
// Reverse: given lam' = dL/dx', lam_k_j = dt b_j lam', and for s = 6..1 the
// stage VJP lam_y = (df/dy)^T lam_k_s, mu += (df/dB0s)^T lam_k_s, then
// lam_k_j += dt a_sj lam_y (j < s) and lam += lam_y; finally lam += lam'.
// The stage VJP runs as node-local kernels and gathers (no atomics):
//   1. reverse of u = J x B and of the current at each interior node ->
//      per-node adjoints of P_a, g_a, 1/det G and the centre B;
//   2. at every node, gather the adjoint of B from the P adjoints of its
//      interior neighbours, reverse the pull-back -> adjoint of g_a, mu;
//   3. at every node, gather the adjoint of y from the g_a adjoints of the
//      nodes whose difference stencils contain it (central inside, one-sided
//      on boundary faces); in the reverse step the same kernel applies the
//      Runge-Kutta combine (lam, lam_k_j) to it directly.
// Boundary nodes are line-tied: their position adjoint is not propagated.
// Every kernel here is launched as a programmatic dependent of the one
// before it (launch_pdl) and starts with pdl_wait(), before any memory
// access.
#include <cuda_runtime.h>

#include <climits>
#include <cmath>

#include "glemur.h"
#include "glemur_dev.cuh"

namespace glemur {

// Cash-Karp table (Cash & Karp, ACM TOMS 16, 1990) for the reverse combine.
__constant__ double AD_A[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0, 253.0 / 4096.0,
     0}};
__constant__ double AD_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0,
                                512.0 / 1771.0};

struct AdjGeom {
  int nx, ny, nz;
  double h2[3];  // 2 h_a
  double s[3];   // B0s_a = B0_a s_a
};

__device__ __forceinline__ int stencil(int i, int n) {  // 0 central, 1 lower, 2 upper
  return i == 0 ? 1 : (i == n - 1 ? 2 : 0);
}

// Column a of G = index-space differences of y (displacement) + 2 h_a e_a.
// FACE = false: central differences only (the node is interior); kept apart
// so that the one-sided variants are not evaluated under predicates at
// interior nodes (predicated-off FP64 instructions still take FP64-pipe
// slots on GB300).
template <bool FACE = true, typename T>
__device__ __forceinline__ void gcol(const AdjGeom& g, const T* y, int N, int a, int i, int j,
                                     int k, double out[3]) {
  const int id[3] = {i, j, k};
  const int n[3] = {g.nx, g.ny, g.nz};
  const int st[3] = {1, g.nx, g.nx * g.ny};
  const int c0 = (k * g.ny + j) * g.nx + i;
  const int sa = st[a];
  const int kind = FACE ? stencil(id[a], n[a]) : 0;
  for (int c = 0; c < 3; ++c) {
    const T* v = y + c * N;
    double d;
    if (!FACE || kind == 0)
      d = (double)v[c0 + sa] - (double)v[c0 - sa];
    else if (kind == 1)
      d = (4.0 * (double)v[c0 + sa] - 3.0 * (double)v[c0]) - (double)v[c0 + 2 * sa];
    else
      d = (3.0 * (double)v[c0] - 4.0 * (double)v[c0 - sa]) + (double)v[c0 - 2 * sa];
    out[c] = d;
  }
  out[a] += g.h2[a];
}

__device__ __forceinline__ void cross3(const double a[3], const double b[3], double o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double dot(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

#define NODE_LOOP(N)                                                                      \
  for (int n = blockIdx.x * blockDim.x + threadIdx.x; n < (N); n += gridDim.x * blockDim.x)

// Dense enumerations of node sets, so that a warp's 32 lanes all run the
// same stencil code: the interior box [1, n-2]^3, the boundary (faces, face
// by face), and the interior split into the deep box [3, n-4]^3 and the
// shell between them.
__device__ __forceinline__ int node_at(const AdjGeom& g, int i, int j, int k) {
  return (k * g.ny + j) * g.nx + i;
}
__device__ __forceinline__ int adj_interior(const AdjGeom& g, int t, int& i, int& j, int& k) {
  const int nxi = g.nx - 2, nyi = g.ny - 2;
  i = 1 + t % nxi;
  const int r = t / nxi;
  j = 1 + r % nyi;
  k = 1 + r / nyi;
  return node_at(g, i, j, k);
}
__device__ __forceinline__ int adj_boundary(const AdjGeom& g, int b, int& i, int& j, int& k) {
  const int nx = g.nx, ny = g.ny, nz = g.nz;
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
  return node_at(g, i, j, k);
}
// the deep box exists when every extent is at least 7
__device__ __forceinline__ bool has_deep(const AdjGeom& g) {
  return g.nx >= 7 && g.ny >= 7 && g.nz >= 7;
}
__device__ __forceinline__ int adj_deep(const AdjGeom& g, int t, int& i, int& j, int& k) {
  const int dx = g.nx - 6, dy = g.ny - 6;
  i = 3 + t % dx;
  const int r = t / dx;
  j = 3 + r % dy;
  k = 3 + r / dy;
  return node_at(g, i, j, k);
}
// shell: planes k in {1, 2, nz-3, nz-2} of the interior box, then rows
// j in {1, 2, ny-3, ny-2} with 3 <= k <= nz-4, then columns i in {1, 2,
// nx-3, nx-2} with 3 <= j <= ny-4, 3 <= k <= nz-4 (all extents >= 7)
__device__ __forceinline__ int adj_shell(const AdjGeom& g, int s, int& i, int& j, int& k) {
  const int ix = g.nx - 2, iy = g.ny - 2, dy = g.ny - 6, dz = g.nz - 6;
  if (s < 4 * ix * iy) {
    const int q = s / (ix * iy), r = s - q * ix * iy;
    k = q < 2 ? 1 + q : g.nz - 5 + q;
    j = 1 + r / ix;
    i = 1 + r % ix;
  } else if (s < 4 * ix * iy + 4 * ix * dz) {
    const int s1 = s - 4 * ix * iy;
    const int q = s1 / (ix * dz), r = s1 - q * ix * dz;
    j = q < 2 ? 1 + q : g.ny - 5 + q;
    k = 3 + r / ix;
    i = 1 + r % ix;
  } else {
    const int s2 = s - 4 * ix * iy - 4 * ix * dz;
    const int q = s2 / (dy * dz), r = s2 - q * dy * dz;
    i = q < 2 ? 1 + q : g.nx - 5 + q;
    k = 3 + r / dy;
    j = 3 + r % dy;
  }
  return node_at(g, i, j, k);
}
#define GRID_LOOP(v, count) \
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < (count); v += gridDim.x * blockDim.x)

// y = d + sum_{j<s} dt a_sj k_j (stage input as a displacement), all nodes.
template <int S, typename T>
__device__ __forceinline__ void adj_stage_input_s(int N3, const T* d, const T* const* k, double dt,
                                                  double* y) {
  double c[S > 0 ? S : 1];
#pragma unroll
  for (int j = 0; j < S; ++j) c[j] = dt * AD_A[S][j];
  NODE_LOOP(N3) {
    double v = (double)d[n];
#pragma unroll
    for (int j = 0; j < S; ++j) v += c[j] * (double)k[j][n];
    y[n] = v;
  }
}

template <typename T>
__global__ void k_adj_stage_input(int N3, const T* d, const T* const* k, int s, double dt,
                                  double* y) {
  pdl_wait();
  pdl_trigger();
  switch (s) {  // stage-uniform: the loop over j unrolls without predicates
    case 0: adj_stage_input_s<0>(N3, d, k, dt, y); break;
    case 1: adj_stage_input_s<1>(N3, d, k, dt, y); break;
    case 2: adj_stage_input_s<2>(N3, d, k, dt, y); break;
    case 3: adj_stage_input_s<3>(N3, d, k, dt, y); break;
    case 4: adj_stage_input_s<4>(N3, d, k, dt, y); break;
    default: adj_stage_input_s<5>(N3, d, k, dt, y); break;
  }
}

// B = G B0s / det G and 1/det G at node n of the stage input y.
template <bool FACE, typename T>
__device__ __forceinline__ void fwd_B_node(const AdjGeom& g, const double* y, const T* B0s,
                                           double* Bb, double* rb, int N, int n, int i, int j,
                                           int k) {
  double G[3][3];
  for (int a = 0; a < 3; ++a) gcol<FACE>(g, y, N, a, i, j, k, G[a]);
  double m[3];
  cross3(G[1], G[2], m);
  const double r = 1.0 / dot(G[0], m);
  const double b0 = (double)B0s[n], b1 = (double)B0s[N + n], b2 = (double)B0s[2 * N + n];
  for (int c = 0; c < 3; ++c) Bb[c * N + n] = (G[0][c] * b0 + G[1][c] * b1 + G[2][c] * b2) * r;
  rb[n] = r;
}

// B = G B0s / det G and 1/det G at every node (interior, then boundary).
template <typename T>
__global__ void k_adj_fwd_B(AdjGeom g, const double* y, const T* B0s, double* Bb, double* rb) {
  pdl_wait();
  pdl_trigger();
  const int N = g.nx * g.ny * g.nz, NI = (g.nx - 2) * (g.ny - 2) * (g.nz - 2);
  GRID_LOOP(t, NI) {
    int i, j, k;
    const int n = adj_interior(g, t, i, j, k);
    fwd_B_node<false>(g, y, B0s, Bb, rb, N, n, i, j, k);
  }
  GRID_LOOP(b, N - NI) {
    int i, j, k;
    const int n = adj_boundary(g, b, i, j, k);
    fwd_B_node<true>(g, y, B0s, Bb, rb, N, n, i, j, k);
  }
}

__device__ __forceinline__ bool interior(const AdjGeom& g, int i, int j, int k) {
  return i > 0 && j > 0 && k > 0 && i < g.nx - 1 && j < g.ny - 1 && k < g.nz - 1;
}

// Forward current at an interior node from y and the B buffer.
__device__ __forceinline__ void current_at(const AdjGeom& g, const double* y, const double* Bb,
                                           const double* rb, int n, int i, int j, int k,
                                           double G[3][3], double P[3][3], double cc[3],
                                           double V[3], double J[3]) {
  const int N = g.nx * g.ny * g.nz;
  const int st[3] = {1, g.nx, g.nx * g.ny};
  for (int a = 0; a < 3; ++a) {
    gcol<false>(g, y, N, a, i, j, k, G[a]);  // interior node: central
    for (int c = 0; c < 3; ++c) P[a][c] = Bb[c * N + n + st[a]] - Bb[c * N + n - st[a]];
  }
  cc[0] = dot(P[1], G[2]) - dot(P[2], G[1]);
  cc[1] = dot(P[2], G[0]) - dot(P[0], G[2]);
  cc[2] = dot(P[0], G[1]) - dot(P[1], G[0]);
  const double r = rb[n];
  for (int c = 0; c < 3; ++c) {
    V[c] = cc[0] * G[0][c] + cc[1] * G[1][c] + cc[2] * G[2][c];
    J[c] = V[c] * r;
  }
}

// Step 1: reverse of u = J x B and of the current at interior nodes.
// lam_u: adjoint of the stage velocity (3N).  Outputs (zero off the
// interior): lamP [3 axes][3 comp][N], lamg [3][3][N] (current part),
// lamr [N] (adjoint of 1/det G from the current), lamB [3][N] (centre B).
__global__ void k_adj_current(AdjGeom g, const double* y, const double* Bb, const double* rb,
                              const double* lam_u, double* lamP, double* lamg, double* lamr,
                              double* lamB) {
  pdl_wait();
  pdl_trigger();
  const int N = g.nx * g.ny * g.nz, NI = (g.nx - 2) * (g.ny - 2) * (g.nz - 2);
  GRID_LOOP(t, NI) {
    int i, j, k;
    const int n = adj_interior(g, t, i, j, k);
    double lP[3][3] = {{0}}, lg[3][3] = {{0}}, lr = 0.0, lB[3] = {0, 0, 0};
    double G[3][3], P[3][3], cc[3], V[3], J[3];
    current_at(g, y, Bb, rb, n, i, j, k, G, P, cc, V, J);
    const double r = rb[n];
    const double lu[3] = {lam_u[n], lam_u[N + n], lam_u[2 * N + n]};
    const double B[3] = {Bb[n], Bb[N + n], Bb[2 * N + n]};
    double lJ[3];
    cross3(B, lu, lJ);  // u = J x B: lam_J = B x lam_u, lam_B = lam_u x J
    cross3(lu, J, lB);
    double lV[3];
    for (int c = 0; c < 3; ++c) lV[c] = lJ[c] * r;
    lr = dot(lJ, V);
    double lc[3];
    for (int a = 0; a < 3; ++a) {
      lc[a] = dot(lV, G[a]);
      for (int c = 0; c < 3; ++c) lg[a][c] += cc[a] * lV[c];
    }
    // c_a = P_{a+1} . g_{a+2} - P_{a+2} . g_{a+1}
    for (int a = 0; a < 3; ++a) {
      const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
      for (int c = 0; c < 3; ++c) {
        lP[a1][c] += lc[a] * G[a2][c];
        lg[a2][c] += lc[a] * P[a1][c];
        lP[a2][c] -= lc[a] * G[a1][c];
        lg[a1][c] -= lc[a] * P[a2][c];
      }
    }
    for (int a = 0; a < 3; ++a)
      for (int c = 0; c < 3; ++c) {
        lamP[(a * 3 + c) * N + n] = lP[a][c];
        lamg[(a * 3 + c) * N + n] = lg[a][c];
      }
    lamr[n] = lr;
    for (int c = 0; c < 3; ++c) lamB[c * N + n] = lB[c];
  }
  GRID_LOOP(b, N - NI) {  // boundary nodes carry no current
    int i, j, k;
    const int n = adj_boundary(g, b, i, j, k);
    for (int q = 0; q < 9; ++q) {
      lamP[q * N + n] = 0.0;
      lamg[q * N + n] = 0.0;
    }
    lamr[n] = 0.0;
    for (int c = 0; c < 3; ++c) lamB[c * N + n] = 0.0;
  }
}

// The pull-back reverse at node n = (i, j, k).  FACE = false: an interior
// node (all six neighbours exist, central differences).
template <bool FACE, typename T>
__device__ __forceinline__ void pullback_node(const AdjGeom& g, const double* y, const T* B0s,
                                              const double* rb, const double* lamP, double* lamg,
                                              const double* lamr, const double* lamB, double wE,
                                              double* mu, int N, int n, int i, int j, int k) {
  const int st[3] = {1, g.nx, g.nx * g.ny};
  const int id[3] = {i, j, k};
  const int ext[3] = {g.nx, g.ny, g.nz};
  // adjoint of B(n): the centre term plus, since P_a(m) = B(m + e_a) -
  // B(m - e_a), +lamP_a(n - e_a) and -lamP_a(n + e_a) (zero unless that
  // neighbour is interior).
  double lB[3] = {lamB[n], lamB[N + n], lamB[2 * N + n]};
  for (int a = 0; a < 3; ++a) {
    if (!FACE || id[a] - 1 >= 0)
      for (int c = 0; c < 3; ++c) lB[c] += lamP[(a * 3 + c) * N + n - st[a]];
    if (!FACE || id[a] + 1 < ext[a])
      for (int c = 0; c < 3; ++c) lB[c] -= lamP[(a * 3 + c) * N + n + st[a]];
  }
  double G[3][3];
  for (int a = 0; a < 3; ++a) gcol<FACE>(g, y, N, a, i, j, k, G[a]);
  const double r = rb[n];
  const double b[3] = {(double)B0s[n], (double)B0s[N + n], (double)B0s[2 * N + n]};
  double W[3];
  for (int c = 0; c < 3; ++c) W[c] = G[0][c] * b[0] + G[1][c] * b[1] + G[2][c] * b[2];
  // B = W r
  double lW[3];
  for (int c = 0; c < 3; ++c) lW[c] = lB[c] * r;
  double lr = dot(lB, W) + lamr[n];
  if (wE != 0.0) {
    int nb = (i == 0 || i == g.nx - 1) + (j == 0 || j == g.ny - 1) + (k == 0 || k == g.nz - 1);
    const double zeta = nb == 0 ? 1.0 : nb == 1 ? 0.5 : nb == 2 ? 0.25 : 0.125;
    for (int c = 0; c < 3; ++c) lW[c] += wE * zeta * W[c] * r / 8.0;
    lr += wE * zeta * dot(W, W) / 16.0;
  }
  // W = sum_a g_a b_a ; r = 1 / det G, d det / d g_a = g_{a+1} x g_{a+2}
  const double ldet = -lr * r * r;
  for (int a = 0; a < 3; ++a) {
    mu[a * N + n] += dot(lW, G[a]);
    double cr[3];
    cross3(G[(a + 1) % 3], G[(a + 2) % 3], cr);
    for (int c = 0; c < 3; ++c) lamg[(a * 3 + c) * N + n] += b[a] * lW[c] + ldet * cr[c];
  }
}

// Step 2: gather the adjoint of B, reverse the pull-back, add the energy
// loss (weight wE; E_M = sum zeta |G B0s|^2 / det G / 16) and the current's
// g and 1/det adjoints.  lamg is updated in place to the total adjoint of
// the columns g_a; mu (adjoint of B0s) is accumulated.  Interior nodes,
// then boundary nodes.
template <typename T>
__global__ void k_adj_pullback(AdjGeom g, const double* y, const T* B0s, const double* rb,
                               const double* lamP, double* lamg, const double* lamr,
                               const double* lamB, double wE, double* mu) {
  pdl_wait();
  pdl_trigger();
  const int N = g.nx * g.ny * g.nz, NI = (g.nx - 2) * (g.ny - 2) * (g.nz - 2);
  GRID_LOOP(t, NI) {
    int i, j, k;
    const int n = adj_interior(g, t, i, j, k);
    pullback_node<false>(g, y, B0s, rb, lamP, lamg, lamr, lamB, wE, mu, N, n, i, j, k);
  }
  GRID_LOOP(b, N - NI) {
    int i, j, k;
    const int n = adj_boundary(g, b, i, j, k);
    pullback_node<true>(g, y, B0s, rb, lamP, lamg, lamr, lamB, wE, mu, N, n, i, j, k);
  }
}

// Coefficient of y(p) in the difference g_a(m) along axis a (index m of the
// stencil's node, p of the position), extent n.
__device__ __forceinline__ double gcoef(int m, int p, int n) {
  const int kind = stencil(m, n);
  if (kind == 0) return p == m + 1 ? 1.0 : (p == m - 1 ? -1.0 : 0.0);
  if (kind == 1) return p == 0 ? -3.0 : (p == 1 ? 4.0 : (p == 2 ? -1.0 : 0.0));
  return p == n - 1 ? 3.0 : (p == n - 2 ? -4.0 : (p == n - 3 ? 1.0 : 0.0));
}

// Adjoint of the stage input at interior node n = (i, j, k), general
// form: the g_a adjoints of every stencil (central or one-sided) that
// contains the node.
__device__ __forceinline__ void positions_general(const AdjGeom& g, const double* lamg, int N,
                                                  int n, int i, int j, int k, double ly[3]) {
  const int st[3] = {1, g.nx, g.nx * g.ny};
  const int id[3] = {i, j, k};
  const int ext[3] = {g.nx, g.ny, g.nz};
  ly[0] = ly[1] = ly[2] = 0.0;
  for (int a = 0; a < 3; ++a)
    for (int dm = -2; dm <= 2; ++dm) {
      const int m = id[a] + dm;
      if (m < 0 || m >= ext[a]) continue;
      const double w = gcoef(m, id[a], ext[a]);
      if (w == 0.0) continue;
      const int nm = n + dm * st[a];
      for (int c = 0; c < 3; ++c) ly[c] += w * lamg[(a * 3 + c) * N + nm];
    }
}

// Where the stage-input adjoint ly of interior node n goes.  S < 0: into
// lam_y.  S = 0..5: straight into the reverse Runge-Kutta combine after
// stage S (lam += ly, lam_k_j += dt a_Sj ly for j < S), with no round trip
// through lam_y.
template <int S>
__device__ __forceinline__ void positions_out(int N, int n, const double ly[3], double* lam_y,
                                              const double* cj, double* lam,
                                              double* const* lam_k) {
  if constexpr (S < 0) {
    for (int c = 0; c < 3; ++c) lam_y[c * N + n] = ly[c];
  } else {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int q = c * N + n;
      lam[q] += ly[c];
#pragma unroll
      for (int j = 0; j < S; ++j) lam_k[j][q] += cj[j] * ly[c];
    }
  }
}

// Step 3: adjoint of the stage input at interior nodes (0 on the boundary).
// Nodes at least 3 from every face are touched by central stencils only:
// lam_y = sum_a lamg_a(n - e_a) - lamg_a(n + e_a); the shell between them
// and the faces takes the general form.  S >= 0: combined with the reverse
// Runge-Kutta step of stage S (positions_out); boundary nodes then add
// nothing (line-tied: their adjoint is 0).
template <int S>
__device__ __forceinline__ void adj_positions_s(const AdjGeom& g, const double* lamg,
                                                double* lam_y, double dt, double* lam,
                                                double* const* lam_k) {
  const int N = g.nx * g.ny * g.nz, NI = (g.nx - 2) * (g.ny - 2) * (g.nz - 2);
  const int st[3] = {1, g.nx, g.nx * g.ny};
  double cj[S > 0 ? S : 1];
#pragma unroll
  for (int j = 0; j < (S > 0 ? S : 0); ++j) cj[j] = dt * AD_A[S][j];
  if (has_deep(g)) {
    const int ND = (g.nx - 6) * (g.ny - 6) * (g.nz - 6);
    GRID_LOOP(t, ND) {
      int i, j, k;
      const int n = adj_deep(g, t, i, j, k);
      double ly[3] = {0, 0, 0};
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c)
          ly[c] += lamg[(a * 3 + c) * N + n - st[a]] - lamg[(a * 3 + c) * N + n + st[a]];
      positions_out<S>(N, n, ly, lam_y, cj, lam, lam_k);
    }
    GRID_LOOP(sidx, NI - ND) {
      int i, j, k;
      const int n = adj_shell(g, sidx, i, j, k);
      double ly[3];
      positions_general(g, lamg, N, n, i, j, k, ly);
      positions_out<S>(N, n, ly, lam_y, cj, lam, lam_k);
    }
  } else {
    GRID_LOOP(t, NI) {
      int i, j, k;
      const int n = adj_interior(g, t, i, j, k);
      double ly[3];
      positions_general(g, lamg, N, n, i, j, k, ly);
      positions_out<S>(N, n, ly, lam_y, cj, lam, lam_k);
    }
  }
  if constexpr (S < 0) {
    GRID_LOOP(b, N - NI) {  // line-tied: no position adjoint
      int i, j, k;
      const int n = adj_boundary(g, b, i, j, k);
      for (int c = 0; c < 3; ++c) lam_y[c * N + n] = 0.0;
    }
  }
}

// s < 0: the stage-input adjoint into lam_y; s = 0..5: combined with the
// reverse Runge-Kutta step of stage s.
__global__ void k_adj_positions(AdjGeom g, const double* lamg, double* lam_y, int s, double dt,
                                double* lam, double* const* lam_k) {
  pdl_wait();
  pdl_trigger();
  switch (s) {  // stage-uniform: the loop over j unrolls without predicates
    case 0: adj_positions_s<0>(g, lamg, lam_y, dt, lam, lam_k); break;
    case 1: adj_positions_s<1>(g, lamg, lam_y, dt, lam, lam_k); break;
    case 2: adj_positions_s<2>(g, lamg, lam_y, dt, lam, lam_k); break;
    case 3: adj_positions_s<3>(g, lamg, lam_y, dt, lam, lam_k); break;
    case 4: adj_positions_s<4>(g, lamg, lam_y, dt, lam, lam_k); break;
    case 5: adj_positions_s<5>(g, lamg, lam_y, dt, lam, lam_k); break;
    default: adj_positions_s<-1>(g, lamg, lam_y, dt, lam, lam_k); break;
  }
}

// Seeds of one step's reverse: lam_k_j = dt b_j lam', lam = lam'.
__global__ void k_adj_seed(int N3, const double* lam_next, double dt, double* lam,
                           double* const* lam_k) {
  pdl_wait();
  pdl_trigger();
  NODE_LOOP(N3) {
    const double v = lam_next[n];
    lam[n] = v;
    for (int j = 0; j < 6; ++j) lam_k[j][n] = dt * AD_B5[j] * v;
  }
}

// Per-CTA (value, index) of xi = |J x B| / |B|^2 over interior nodes.
__global__ void k_adj_xi_partial(AdjGeom g, const double* y, const double* Bb, const double* rb,
                                 double* pv, int* pi) {
  pdl_wait();
  pdl_trigger();
  const int N = g.nx * g.ny * g.nz;
  double best = -1.0;
  int arg = -1;
  NODE_LOOP(N) {
    const int i = n % g.nx, j = (n / g.nx) % g.ny, k = n / (g.nx * g.ny);
    if (!interior(g, i, j, k)) continue;
    double G[3][3], P[3][3], cc[3], V[3], J[3], u[3];
    current_at(g, y, Bb, rb, n, i, j, k, G, P, cc, V, J);
    const double B[3] = {Bb[n], Bb[N + n], Bb[2 * N + n]};
    cross3(J, B, u);
    const double v = sqrt(dot(u, u)) / dot(B, B);
    if (v > best || (v == best && n < arg)) {
      best = v;
      arg = n;
    }
  }
  __shared__ double sv[256];
  __shared__ int si[256];
  sv[threadIdx.x] = best;
  si[threadIdx.x] = arg;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      const double v2 = sv[threadIdx.x + o];
      const int i2 = si[threadIdx.x + o];
      if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 >= 0 && i2 < si[threadIdx.x])) {
        sv[threadIdx.x] = v2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = sv[0];
    pi[blockIdx.x] = si[0];
  }
}

// Seed of the xi loss at its argmax node: lam_u = u / (|u| |B|^2) and the
// direct B dependence -2 |u| B / |B|^4; writes the value to out[0].
__global__ void k_adj_xi_seed(AdjGeom g, const double* y, const double* Bb, const double* rb,
                              const double* pv, const int* pi, int nb, double* lam_u,
                              double* lamB_extra, double* out) {
  pdl_wait();
  pdl_trigger();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int N = g.nx * g.ny * g.nz;
  double best = -1.0;
  int n = -1;
  for (int b = 0; b < nb; ++b)
    if (pv[b] > best || (pv[b] == best && pi[b] >= 0 && pi[b] < n)) {
      best = pv[b];
      n = pi[b];
    }
  out[0] = best;
  if (n < 0) return;
  const int i = n % g.nx, j = (n / g.nx) % g.ny, k = n / (g.nx * g.ny);
  double G[3][3], P[3][3], cc[3], V[3], J[3], u[3];
  current_at(g, y, Bb, rb, n, i, j, k, G, P, cc, V, J);
  const double B[3] = {Bb[n], Bb[N + n], Bb[2 * N + n]};
  cross3(J, B, u);
  const double um = sqrt(dot(u, u)), b2 = dot(B, B);
  for (int c = 0; c < 3; ++c) {
    lam_u[c * N + n] = um > 0.0 ? u[c] / (um * b2) : 0.0;
    lamB_extra[c * N + n] = -2.0 * um * B[c] / (b2 * b2);
  }
}

__global__ void k_adj_add(int M, const double* a, double* b) {
  pdl_wait();
  pdl_trigger();
  NODE_LOOP(M) b[n] += a[n];
}

__global__ void k_adj_zero(int M, double* a) {
  pdl_wait();
  pdl_trigger();
  NODE_LOOP(M) a[n] = 0.0;
}

// mu (adjoint of B0s) -> adjoint of B0: B0s_a = s_a B0_a.
__global__ void k_adj_mu_out(AdjGeom g, const double* mu, double* mu_B0) {
  pdl_wait();
  pdl_trigger();
  const int N = g.nx * g.ny * g.nz;
  NODE_LOOP(N) for (int c = 0; c < 3; ++c) mu_B0[c * N + n] += g.s[c] * mu[c * N + n];
}

// Parameter contraction out[p] = sum_m dB[p][m] mu[m] (fixed-order sums).
__global__ void k_param_contract(long long M, const double* dB, const double* mu,
                                 double* out) {
  pdl_wait();
  pdl_trigger();
  const int p = blockIdx.x;
  double s = 0.0;
  for (long long m = threadIdx.x; m < M; m += blockDim.x) s += dB[p * M + m] * mu[m];
  __shared__ double sh[256];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) out[p] = sh[0];
}

}  // namespace glemur

// ------------------------------------------------------------ host side

namespace glemur {
// Provided by glemur.cu.
int ctx_recompute_stages(glemur_ctx* c, double dt, void* k6);
int ctx_recompute_stages_saved(glemur_ctx* c, double dt, void* k6, double* const* yS,
                               double* const* BS, double* const* RS);
int ctx_info(glemur_ctx* c, int* nx, int* ny, int* nz, double h[3], int* precision,
             void** d_cur, void** B0s, void** k, void** stream);
}  // namespace glemur

using namespace glemur;

namespace {

size_t al(size_t v) { return (v + 255) & ~(size_t)255; }

// Adjoint workspace: k6 (storage type), FP64 stage input, B, 1/det, six
// stage adjoints, the stage-input adjoint, the P and g adjoints, the
// 1/det, centre-B, extra-B and velocity adjoints, mu (adjoint of B0s), the
// xi partials and two small pointer tables.
struct AdjLayout {
  size_t k6, y, Bb, rb, lamk, lamy, lamP, lamg, lamr, lamB, lamB2, lamu, mu, pv, pi, ptr,
      yS, BS, RS, total, fstride, rstride;
};

constexpr int kXiBlocks = 1024;

AdjLayout adj_layout(int nx, int ny, int nz, int precision) {
  const size_t N = (size_t)nx * ny * nz;
  const size_t es = precision == GLEMUR_MIXED ? 4 : 8;
  AdjLayout L{};
  size_t o = 0;
  L.fstride = al(3 * N * 8);
  L.k6 = o; o += al(3 * N * es);
  L.y = o; o += L.fstride;
  L.Bb = o; o += L.fstride;
  L.rb = o; o += al(N * 8);
  L.lamk = o; o += 6 * L.fstride;
  L.lamy = o; o += L.fstride;
  L.lamP = o; o += al(9 * N * 8);
  L.lamg = o; o += al(9 * N * 8);
  L.lamr = o; o += al(N * 8);
  L.lamB = o; o += L.fstride;
  L.lamB2 = o; o += L.fstride;
  L.lamu = o; o += L.fstride;
  L.mu = o; o += L.fstride;
  L.pv = o; o += al(kXiBlocks * 8 + 8);
  L.pi = o; o += al(kXiBlocks * 4);
  L.ptr = o; o += 256;
  // FP64: every stage's input (y_1..y_5), B and 1/det G, kept by the
  // forward recompute so the reverse loop need not form them again
  L.rstride = al(N * 8);
  if (precision == GLEMUR_FP64) {
    L.yS = o; o += 5 * L.fstride;
    L.BS = o; o += 6 * L.fstride;
    L.RS = o; o += 6 * L.rstride;
  }
  L.total = o;
  return L;
}

struct Adj {
  int N, precision;
  AdjGeom g;
  void* d;
  void* B0s;
  void* k[5];
  cudaStream_t s;
  unsigned char* ws;
  AdjLayout L;
  double* P(size_t off) const { return (double*)(ws + off); }
};

int adj_open(glemur_ctx* c, void* ws, size_t bytes, Adj* A) {
  if (!c || !ws || ((uintptr_t)ws & 255)) return GLEMUR_ERR_BADARG;
  double h[3];
  void* stream = nullptr;
  int nx, ny, nz;
  int rc = ctx_info(c, &nx, &ny, &nz, h, &A->precision, &A->d, &A->B0s, A->k, &stream);
  if (rc) return rc;
  A->s = (cudaStream_t)stream;
  A->N = nx * ny * nz;
  A->L = adj_layout(nx, ny, nz, A->precision);
  if (bytes < A->L.total) return GLEMUR_ERR_WORKSPACE;
  A->ws = (unsigned char*)ws;
  A->g.nx = nx;
  A->g.ny = ny;
  A->g.nz = nz;
  for (int a = 0; a < 3; ++a) A->g.h2[a] = 2.0 * h[a];
  A->g.s[0] = 4.0 * h[1] * h[2];
  A->g.s[1] = 4.0 * h[2] * h[0];
  A->g.s[2] = 4.0 * h[0] * h[1];
  return GLEMUR_OK;
}

int nblk(long long n) {
  long long b = (n + 255) / 256;
  return (int)(b < 8192 ? (b < 1 ? 1 : b) : 8192);
}

// Five stage-input buffers (pointers by value).
struct YSave {
  double* p[5];
};

// Boundary entries of the saved stage inputs y_1..y_5: the fixed boundary
// positions (the forward passes write interior nodes only).
__global__ void k_adj_seed_boundary(AdjGeom g, const double* d, YSave ys) {
  pdl_wait();
  pdl_trigger();
  const int N = g.nx * g.ny * g.nz, NI = (g.nx - 2) * (g.ny - 2) * (g.nz - 2);
  GRID_LOOP(b, N - NI) {
    int i, j, k;
    const int n = adj_boundary(g, b, i, j, k);
    for (int c = 0; c < 3; ++c) {
      const double v = d[c * N + n];
      for (int q = 0; q < 5; ++q) ys.p[q][c * N + n] = v;
    }
  }
}

// The stage VJP at the stage input y (B and 1/det G in Bb, rb; formed here
// when form_B): lam_u -> lam_y, mu +=.  rk_s >= 0: the stage-input adjoint
// goes straight into the reverse Runge-Kutta combine of stage rk_s (lam,
// lam_k) instead of lam_y.
template <typename T>
void stage_vjp(const Adj& A, const double* y, double* Bb, double* rb, bool form_B,
               const double* lam_u, const double* extra_lamB, double wE, int rk_s = -1,
               double dt = 0.0, double* lam = nullptr, double* const* lam_k = nullptr) {
  const int N = A.N;
  if (form_B) launch_pdl(k_adj_fwd_B<T>, dim3(nblk(N)), dim3(256), 0, A.s, A.g, y, (const T*)A.B0s,
                         Bb, rb);
  if (lam_u) {
    launch_pdl(k_adj_current, dim3(nblk(N)), dim3(256), 0, A.s, A.g, y, Bb, rb, lam_u,
               A.P(A.L.lamP), A.P(A.L.lamg), A.P(A.L.lamr), A.P(A.L.lamB));
  } else {
    launch_pdl(k_adj_zero, dim3(nblk(9 * N)), dim3(256), 0, A.s, 9 * N, A.P(A.L.lamP));
    launch_pdl(k_adj_zero, dim3(nblk(9 * N)), dim3(256), 0, A.s, 9 * N, A.P(A.L.lamg));
    launch_pdl(k_adj_zero, dim3(nblk(N)), dim3(256), 0, A.s, N, A.P(A.L.lamr));
    launch_pdl(k_adj_zero, dim3(nblk(3 * N)), dim3(256), 0, A.s, 3 * N, A.P(A.L.lamB));
  }
  if (extra_lamB) launch_pdl(k_adj_add, dim3(nblk(3 * N)), dim3(256), 0, A.s, 3 * N, extra_lamB,
                             A.P(A.L.lamB));
  launch_pdl(k_adj_pullback<T>, dim3(nblk(N)), dim3(256), 0, A.s, A.g, y, (const T*)A.B0s, rb,
             A.P(A.L.lamP), A.P(A.L.lamg), A.P(A.L.lamr), A.P(A.L.lamB), wE, A.P(A.L.mu));
  launch_pdl(k_adj_positions, dim3(nblk(N)), dim3(256), 0, A.s, A.g, (const double*)A.P(A.L.lamg),
             A.P(A.L.lamy), rk_s, dt, lam, lam_k);
}

template <typename T>
int vjp_step_t(glemur_ctx* c, const Adj& A, double dt, const double* lam_next, double* lam,
               double* mu_B0) {
  const int N3 = 3 * A.N;
  // FP64 two-pass contexts: the recompute keeps every stage's input, B and
  // 1/det G; otherwise the reverse loop forms them again
  double* yS[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  double* BS[6];
  double* RS[6];
  bool saved = false;
  if (A.precision == GLEMUR_FP64) {
    YSave ysave;
    for (int q = 1; q < 6; ++q) ysave.p[q - 1] = yS[q] = A.P(A.L.yS + (q - 1) * A.L.fstride);
    for (int q = 0; q < 6; ++q) {
      BS[q] = A.P(A.L.BS + q * A.L.fstride);
      RS[q] = A.P(A.L.RS + q * A.L.rstride);
    }
    launch_pdl(k_adj_seed_boundary, dim3(nblk(A.N)), dim3(256), 0, A.s, A.g, (const double*)A.d,
               ysave);
    const int rs = ctx_recompute_stages_saved(c, dt, A.ws + A.L.k6, yS, BS, RS);
    if (rs != GLEMUR_OK && rs != GLEMUR_ERR_BADARG) return rs;
    saved = rs == GLEMUR_OK;
  }
  int rc = saved ? GLEMUR_OK : ctx_recompute_stages(c, dt, A.ws + A.L.k6);
  if (rc) return rc;
  double* lamk_h[6];
  for (int j = 0; j < 6; ++j) lamk_h[j] = A.P(A.L.lamk + j * A.L.fstride);
  const T* kp[6] = {(const T*)A.k[0], (const T*)A.k[1], (const T*)A.k[2], (const T*)A.k[3],
                    (const T*)A.k[4], (const T*)(A.ws + A.L.k6)};
  double** lamk_d = (double**)(A.ws + A.L.ptr);
  const T** kp_d = (const T**)(A.ws + A.L.ptr + 64);
  cudaError_t e = cudaMemcpyAsync(lamk_d, lamk_h, sizeof(lamk_h), cudaMemcpyHostToDevice, A.s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kp_d, kp, sizeof(kp), cudaMemcpyHostToDevice, A.s);
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  launch_pdl(k_adj_zero, dim3(nblk(N3)), dim3(256), 0, A.s, N3, A.P(A.L.mu));
  launch_pdl(k_adj_seed, dim3(nblk(N3)), dim3(256), 0, A.s, N3, lam_next, dt, lam, lamk_d);
  for (int s = 5; s >= 0; --s) {
    if (saved) {
      stage_vjp<T>(A, s == 0 ? (const double*)A.d : yS[s], BS[s], RS[s], false, lamk_h[s],
                   nullptr, 0.0, s, dt, lam, lamk_d);
    } else {
      launch_pdl(k_adj_stage_input<T>, dim3(nblk(N3)), dim3(256), 0, A.s, N3, (const T*)A.d, kp_d,
                 s, dt, A.P(A.L.y));
      stage_vjp<T>(A, A.P(A.L.y), A.P(A.L.Bb), A.P(A.L.rb), true, lamk_h[s], nullptr, 0.0, s,
                   dt, lam, lamk_d);
    }
  }
  launch_pdl(k_adj_mu_out, dim3(nblk(A.N)), dim3(256), 0, A.s, A.g, A.P(A.L.mu), mu_B0);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(A.s);  // pointer tables are host stack
  return e == cudaSuccess ? GLEMUR_OK : GLEMUR_ERR_CUDA;
}

template <typename T>
int loss_grad_t(glemur_ctx* c, const Adj& A, int loss, double* value, double* lam,
                double* mu_B0) {
  const int N = A.N, N3 = 3 * N;
  const T* kp[1] = {nullptr};
  const T** kp_d = (const T**)(A.ws + A.L.ptr + 64);
  if (cudaMemcpyAsync(kp_d, kp, sizeof(kp), cudaMemcpyHostToDevice, A.s)) return GLEMUR_ERR_CUDA;
  launch_pdl(k_adj_zero, dim3(nblk(N3)), dim3(256), 0, A.s, N3, A.P(A.L.mu));
  launch_pdl(k_adj_stage_input<T>, dim3(nblk(N3)), dim3(256), 0, A.s, N3, (const T*)A.d, kp_d, 0,
             0.0, A.P(A.L.y));
  double v = 0.0;
  if (loss == 0) {
    stage_vjp<T>(A, A.P(A.L.y), A.P(A.L.Bb), A.P(A.L.rb), true, nullptr, nullptr, 1.0);
    int rc = glemur_energy(c, &v);
    if (rc) return rc;
  } else {
    double* Bb = A.P(A.L.Bb);
    double* rb = A.P(A.L.rb);
    launch_pdl(k_adj_fwd_B<T>, dim3(nblk(N)), dim3(256), 0, A.s, A.g, A.P(A.L.y), (const T*)A.B0s,
               Bb, rb);
    const int nb = nblk(N) < kXiBlocks ? nblk(N) : kXiBlocks;
    double* pv = A.P(A.L.pv);
    int* pi = (int*)(A.ws + A.L.pi);
    launch_pdl(k_adj_xi_partial, dim3(nb), dim3(256), 0, A.s, A.g, A.P(A.L.y), Bb, rb, pv, pi);
    launch_pdl(k_adj_zero, dim3(nblk(N3)), dim3(256), 0, A.s, N3, A.P(A.L.lamu));
    launch_pdl(k_adj_zero, dim3(nblk(N3)), dim3(256), 0, A.s, N3, A.P(A.L.lamB2));
    double* out = pv + kXiBlocks;
    launch_pdl(k_adj_xi_seed, dim3(1), dim3(32), 0, A.s, A.g, A.P(A.L.y), Bb, rb, pv, pi, nb,
               A.P(A.L.lamu), A.P(A.L.lamB2), out);
    stage_vjp<T>(A, A.P(A.L.y), A.P(A.L.Bb), A.P(A.L.rb), false, A.P(A.L.lamu), A.P(A.L.lamB2),
                 0.0);
    if (cudaMemcpyAsync(&v, out, sizeof(double), cudaMemcpyDeviceToHost, A.s))
      return GLEMUR_ERR_CUDA;
  }
  cudaMemcpyAsync(lam, A.P(A.L.lamy), sizeof(double) * N3, cudaMemcpyDeviceToDevice, A.s);
  launch_pdl(k_adj_mu_out, dim3(nblk(N)), dim3(256), 0, A.s, A.g, A.P(A.L.mu), mu_B0);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(A.s);
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  if (value) *value = v;
  return GLEMUR_OK;
}

}  // namespace

extern "C" {

size_t glemur_adjoint_workspace_bytes(int nx, int ny, int nz, int precision) {
  if (nx < 3 || ny < 3 || nz < 3 || 9LL * nx * ny * nz >= (1LL << 31)) return 0;
  if (precision != GLEMUR_FP64 && precision != GLEMUR_MIXED) return 0;
  return adj_layout(nx, ny, nz, precision).total;
}

int glemur_vjp_step(glemur_ctx* c, double dt, const double* lam_next, double* lam,
                    double* mu_B0, void* adj_ws, size_t adj_bytes) {
  if (!lam_next || !lam || !mu_B0 || !(dt > 0) || !std::isfinite(dt)) return GLEMUR_ERR_BADARG;
  Adj A;
  int rc = adj_open(c, adj_ws, adj_bytes, &A);
  if (rc) return rc;
  return A.precision == GLEMUR_MIXED ? vjp_step_t<float>(c, A, dt, lam_next, lam, mu_B0)
                                     : vjp_step_t<double>(c, A, dt, lam_next, lam, mu_B0);
}

int glemur_loss_grad(glemur_ctx* c, int loss, double* value, double* lam, double* mu_B0,
                     void* adj_ws, size_t adj_bytes) {
  if (!lam || !mu_B0 || (loss != GLEMUR_LOSS_ENERGY && loss != GLEMUR_LOSS_XI))
    return GLEMUR_ERR_BADARG;
  Adj A;
  int rc = adj_open(c, adj_ws, adj_bytes, &A);
  if (rc) return rc;
  return A.precision == GLEMUR_MIXED ? loss_grad_t<float>(c, A, loss, value, lam, mu_B0)
                                     : loss_grad_t<double>(c, A, loss, value, lam, mu_B0);
}

size_t glemur_adjoint_segment_bytes(glemur_ctx* c, int n_steps, int every) {
  if (!c || n_steps < 0 || every < 1) return 0;
  int nx, ny, nz, prec;
  double h[3];
  void *d, *B0s, *k[5], *stream;
  if (ctx_info(c, &nx, &ny, &nz, h, &prec, &d, &B0s, k, &stream)) return 0;
  const size_t S = (glemur_state_bytes(c) + 255) & ~(size_t)255;
  const size_t F = (sizeof(double) * 3 * (size_t)nx * ny * nz + 255) & ~(size_t)255;
  const size_t nseg = n_steps > 0 ? ((size_t)n_steps + every - 1) / every : 1;
  const size_t per = (size_t)(n_steps < every ? n_steps : every);
  return (nseg + per) * S + F;
}

int glemur_adjoint_segment(glemur_ctx* c, const double* x0, const double* dts, int n, int every,
                           int loss, double* value, double* lam_x0, double* mu_B0, void* adj_ws,
                           size_t adj_bytes, void* seg_ws, size_t seg_bytes) {
  if (!c || !x0 || !value || !lam_x0 || !mu_B0 || n < 0 || every < 1 || (n > 0 && !dts) ||
      (loss != GLEMUR_LOSS_ENERGY && loss != GLEMUR_LOSS_XI))
    return GLEMUR_ERR_BADARG;
  for (int i = 0; i < n; ++i)
    if (!(dts[i] > 0) || !std::isfinite(dts[i])) return GLEMUR_ERR_BADARG;
  const size_t need = glemur_adjoint_segment_bytes(c, n, every);
  if (!need || !seg_ws || ((uintptr_t)seg_ws & 255) || seg_bytes < need)
    return GLEMUR_ERR_WORKSPACE;
  int nx, ny, nz, prec;
  double h[3];
  void *d, *B0s, *k[5], *stream;
  int rc = ctx_info(c, &nx, &ny, &nz, h, &prec, &d, &B0s, k, &stream);
  if (rc) return rc;
  const cudaStream_t s = (cudaStream_t)stream;
  const size_t S = (glemur_state_bytes(c) + 255) & ~(size_t)255;
  const size_t F3 = sizeof(double) * 3 * (size_t)nx * ny * nz;
  const long long nseg = n > 0 ? ((long long)n + every - 1) / every : 1;
  const int per = n < every ? n : every;
  unsigned char* base = (unsigned char*)seg_ws;
  unsigned char* states = base + (size_t)nseg * S;  // the states after each step of a segment
  double* scratch = (double*)(states + (size_t)per * S);
  auto ckpt = [&](long long q) { return (void*)(base + (size_t)q * S); };
  // forward: checkpoints at steps 0, every, 2 every, ... (< n); x0 is read
  // before the outputs are cleared, so it may share a buffer with them
  glemur_stats st;
  if ((rc = glemur_set_x(c, x0, GLEMUR_MEM_DEVICE))) return rc;
  if ((rc = glemur_get_state(c, ckpt(0)))) return rc;
  cudaError_t e = cudaMemsetAsync(mu_B0, 0, F3, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(lam_x0, 0, F3, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(scratch, 0, F3, s);
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  for (int i = 0; i < n; ++i) {
    if ((rc = glemur_step_fixed(c, dts[i], &st))) return rc;
    if ((i + 1) % every == 0 && i + 1 < n && (rc = glemur_get_state(c, ckpt((i + 1) / every))))
      return rc;
  }
  if (n == 0) {
    if ((rc = glemur_set_state(c, ckpt(0)))) return rc;
    return glemur_loss_grad(c, loss, value, lam_x0, mu_B0, adj_ws, adj_bytes);
  }
  // backward, segment by segment from the last
  double* lam_next = lam_x0;
  double* lam = scratch;
  bool seeded = false;
  for (long long q = nseg - 1; q >= 0; --q) {
    const int start = (int)(q * every), end = start + every < n ? start + every : n;
    if ((rc = glemur_set_state(c, ckpt(q)))) return rc;
    for (int i = start; i < end; ++i) {
      if ((rc = glemur_step_fixed(c, dts[i], &st))) return rc;
      if ((rc = glemur_get_state(c, states + (size_t)(i - start) * S))) return rc;
    }
    if (!seeded) {  // the context is at the final state
      if ((rc = glemur_loss_grad(c, loss, value, lam_next, mu_B0, adj_ws, adj_bytes))) return rc;
      seeded = true;
    }
    for (int i = end - 1; i >= start; --i) {
      const void* xi = i == start ? ckpt(q) : (const void*)(states + (size_t)(i - start - 1) * S);
      if ((rc = glemur_set_state(c, xi))) return rc;
      if ((rc = glemur_vjp_step(c, dts[i], lam_next, lam, mu_B0, adj_ws, adj_bytes))) return rc;
      double* t = lam_next;
      lam_next = lam;
      lam = t;
    }
  }
  if (lam_next != lam_x0) e = cudaMemcpyAsync(lam_x0, lam_next, F3, cudaMemcpyDeviceToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  return e == cudaSuccess ? GLEMUR_OK : GLEMUR_ERR_CUDA;
}

int glemur_param_contract(int n_params, long long m, const double* dB0, const double* mu,
                          double* out, void* stream) {
  if (n_params < 1 || m < 1 || !dB0 || !mu || !out) return GLEMUR_ERR_BADARG;
  launch_pdl(k_param_contract, dim3(n_params), dim3(256), 0, (cudaStream_t)stream, m, dB0, mu, out);
  return cudaGetLastError() == cudaSuccess ? GLEMUR_OK : GLEMUR_ERR_CUDA;
}

}  // extern "C"
