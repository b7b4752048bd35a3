// Validation diagnostics of section "Diagnostics" beyond E_M and xi, on the
// accepted state of a context:
//   * the deviation from a known equilibrium (section "Deviation from the
//     Exact Known Equilibrium"): sigma_x and sigma_B, the root mean square
//     over all nodes of |x - x_ref| and |B - B_ref|;
//   * alpha* = J.B / B^2 along a line of nodes and eq. "epsilon star", the
//     largest a_r (alpha*_k - alpha*_l) / |X_k - X_l| over pairs of its
//     nodes (section "Force-Freeness"), with the context's current;
//   * the convexity kappa of eq. "convexity" at every node (section
//     "Convexity"): +1 when every trihedron of index neighbours has a
//     determinant of sign di dj dk, else -1.
// They run on demand, not inside the step: one thread per node, FP64
// arithmetic whatever the storage precision, deterministic fixed-order
// sums.  B = G B0s / det G with the index-space columns g_a = 2 h_a dx/dX_a
// and the pre-scaled B0s (see glemur_dev.cuh); the current is the compact
// form of the nearest-neighbour loops, J = (c_0 g_0 + c_1 g_1 + c_2 g_2) /
// det G with c_a = P_{a+1}.g_{a+2} - P_{a+2}.g_{a+1} and P_a the central
// differences of B, or the classic product-rule current.
#include <cuda_runtime.h>

#include <cmath>

#include "glemur.h"
#include "glemur_dev.cuh"

namespace glemur {

int ctx_diag(glemur_ctx* c, DiagCtx* out);  // glemur.cu

namespace {

struct DG {
  int nx, ny, nz;
  double lo[3], h[3], h2[3];
  int periodic;  // periodic in z: ghost planes carry their partner's B
};

__device__ __forceinline__ int nid(const DG& g, int i, int j, int k) {
  return (k * g.ny + j) * g.nx + i;
}

// Column a of G at node (i, j, k) from the displacement d: central
// differences inside, second-order one-sided on the faces, + 2 h_a e_a.
template <typename T>
__device__ void gcol_d(const DG& g, const T* d, int N, int a, int i, int j, int k,
                       double out[3]) {
  const int id[3] = {i, j, k};
  const int n[3] = {g.nx, g.ny, g.nz};
  const int st[3] = {1, g.nx, g.nx * g.ny};
  const int c0 = nid(g, i, j, k), sa = st[a];
  for (int c = 0; c < 3; ++c) {
    const T* v = d + c * N;
    double r;
    if (id[a] > 0 && id[a] < n[a] - 1)
      r = (double)v[c0 + sa] - (double)v[c0 - sa];
    else if (id[a] == 0)
      r = (4.0 * (double)v[c0 + sa] - 3.0 * (double)v[c0]) - (double)v[c0 + 2 * sa];
    else
      r = (3.0 * (double)v[c0] - 4.0 * (double)v[c0 - sa]) + (double)v[c0 - 2 * sa];
    out[c] = r;
  }
  out[a] += g.h2[a];
}

__device__ __forceinline__ double ddot(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

__device__ __forceinline__ double ddet(const double g0[3], const double g1[3],
                                       const double g2[3]) {
  return g0[0] * (g1[1] * g2[2] - g1[2] * g2[1]) + g0[1] * (g1[2] * g2[0] - g1[0] * g2[2]) +
         g0[2] * (g1[0] * g2[1] - g1[1] * g2[0]);
}

// Eq. "B transformation" at node (i, j, k): B and det G; G's columns in g.
// Periodic in z, a ghost plane's B is its partner's (section "Boundary
// Conditions").
template <typename T>
__device__ double pull_B(const DG& g, const T* d, const T* B0s, int N, int i, int j, int k,
                         double G[3][3], double B[3]) {
  if (g.periodic) k = k == 0 ? g.nz - 2 : (k == g.nz - 1 ? 1 : k);
  gcol_d(g, d, N, 0, i, j, k, G[0]);
  gcol_d(g, d, N, 1, i, j, k, G[1]);
  gcol_d(g, d, N, 2, i, j, k, G[2]);
  const double det = ddet(G[0], G[1], G[2]);
  const int n = nid(g, i, j, k);
  const double b0 = (double)B0s[n], b1 = (double)B0s[N + n], b2 = (double)B0s[2 * N + n];
  for (int c = 0; c < 3; ++c) B[c] = (G[0][c] * b0 + G[1][c] * b1 + G[2][c] * b2) / det;
  return det;
}

// Nearest-neighbour mimetic current at interior node (i, j, k) (compact
// form of the three Stokes loops) and B there.
template <typename T>
__device__ void current_mimetic(const DG& g, const T* d, const T* B0s, int N, int i, int j,
                                int k, double J[3], double B[3]) {
  double G[3][3], Gn[3][3], Bp[3], Bm[3], P[3][3];
  const double det = pull_B(g, d, B0s, N, i, j, k, G, B);
  for (int a = 0; a < 3; ++a) {
    const int e[3] = {a == 0, a == 1, a == 2};
    pull_B(g, d, B0s, N, i + e[0], j + e[1], k + e[2], Gn, Bp);
    pull_B(g, d, B0s, N, i - e[0], j - e[1], k - e[2], Gn, Bm);
    for (int c = 0; c < 3; ++c) P[a][c] = Bp[c] - Bm[c];
  }
  double cc[3];
  for (int a = 0; a < 3; ++a) {
    const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
    cc[a] = ddot(P[a1], G[a2]) - ddot(P[a2], G[a1]);
  }
  for (int c = 0; c < 3; ++c) J[c] = (cc[0] * G[0][c] + cc[1] * G[1][c] + cc[2] * G[2][c]) / det;
}

// Next-nearest-neighbour current at interior node (i, j, k): in each index
// surface r (spanned by p = r+1, q = r+2) the octilateral through the eight
// in-plane neighbours, counter-clockwise about +r from the corner
// +e_p - e_q, edge-mean B for the circulation, the four corner triangles
// (/ 2) and the inner quadrilateral through the face neighbours (/ 4) for
// the vector area; M J = c solved by the adjugate.
template <typename T>
__device__ void current_nnn(const DG& g, const T* d, const T* B0s, int N, int i, int j, int k,
                            double J[3], double B[3]) {
  const int op[8] = {1, 1, 1, 0, -1, -1, -1, 0};
  const int oq[8] = {-1, 0, 1, 1, 1, 0, -1, -1};
  const int n = nid(g, i, j, k);
  double Gc[3][3], M[3][3], cr[3];
  pull_B(g, d, B0s, N, i, j, k, Gc, B);
  for (int r = 0; r < 3; ++r) {
    const int p = (r + 1) % 3, q = (r + 2) % 3;
    double xv[8][3], Bv[8][3], Gn[3][3];
    for (int m = 0; m < 8; ++m) {
      int id[3] = {i, j, k};
      id[p] += op[m];
      id[q] += oq[m];
      const int nn = nid(g, id[0], id[1], id[2]);
      for (int c = 0; c < 3; ++c) xv[m][c] = (double)d[c * N + nn] - (double)d[c * N + n];
      xv[m][p] += op[m] * g.h[p];
      xv[m][q] += oq[m] * g.h[q];
      pull_B(g, d, B0s, N, id[0], id[1], id[2], Gn, Bv[m]);
    }
    double circ = 0.0, dx[8][3];
    for (int m = 0; m < 8; ++m)
      for (int c = 0; c < 3; ++c) {
        dx[m][c] = xv[(m + 1) % 8][c] - xv[m][c];
        circ += 0.5 * (Bv[m][c] + Bv[(m + 1) % 8][c]) * dx[m][c];
      }
    double area[3] = {0.0, 0.0, 0.0};
    for (int t = 0; t < 4; ++t) {
      const double* e0 = dx[2 * t + 1];
      const double* e1 = dx[(2 * t + 2) % 8];
      area[0] += 0.5 * (e0[1] * e1[2] - e0[2] * e1[1]);
      area[1] += 0.5 * (e0[2] * e1[0] - e0[0] * e1[2]);
      area[2] += 0.5 * (e0[0] * e1[1] - e0[1] * e1[0]);
    }
    double qd[4][3];
    for (int c = 0; c < 3; ++c) {
      qd[0][c] = xv[3][c] - xv[1][c];
      qd[1][c] = xv[5][c] - xv[3][c];
      qd[2][c] = xv[7][c] - xv[5][c];
      qd[3][c] = xv[1][c] - xv[7][c];
    }
    for (int t = 0; t < 4; ++t) {
      const double* e0 = qd[t];
      const double* e1 = qd[(t + 1) % 4];
      area[0] += 0.25 * (e0[1] * e1[2] - e0[2] * e1[1]);
      area[1] += 0.25 * (e0[2] * e1[0] - e0[0] * e1[2]);
      area[2] += 0.25 * (e0[0] * e1[1] - e0[1] * e1[0]);
    }
    cr[r] = circ;
    for (int c = 0; c < 3; ++c) M[r][c] = area[c];
  }
  double adj[3][3];
  for (int r = 0; r < 3; ++r) {
    const double* u = M[(r + 1) % 3];
    const double* v = M[(r + 2) % 3];
    adj[r][0] = u[1] * v[2] - u[2] * v[1];
    adj[r][1] = u[2] * v[0] - u[0] * v[2];
    adj[r][2] = u[0] * v[1] - u[1] * v[0];
  }
  const double detM = ddot(M[0], adj[0]);
  for (int c = 0; c < 3; ++c)
    J[c] = (cr[0] * adj[0][c] + cr[1] * adj[1][c] + cr[2] * adj[2][c]) / detM;
}

// Classic current at interior node (i, j, k): dB/dX by the product rule on
// B = G B0s / det G (second differences of x, central differences of B0s,
// Jacobi's formula for the derivative of det G), then dB/dx = dB/dX (dx/dX)^-1
// and J = curl_x B; all differences in index space.
template <typename T>
__device__ void current_direct(const DG& g, const T* d, const T* B0s, int N, int i, int j,
                               int k, double J[3], double B[3]) {
  const int st[3] = {1, g.nx, g.nx * g.ny};
  const int n = nid(g, i, j, k);
  double G[3][3], S[3][3][3], b[3], Db[3][3];
  for (int a = 0; a < 3; ++a) gcol_d(g, d, N, a, i, j, k, G[a]);
  for (int c = 0; c < 3; ++c) {
    const T* v = d + c * N;
    const double xc = (double)v[n];
    for (int a = 0; a < 3; ++a) {
      const int sa = st[a];
      // the label grid is linear: its second differences vanish
      S[a][a][c] = 4.0 * (((double)v[n + sa] + (double)v[n - sa]) - 2.0 * xc);
      for (int e = a + 1; e < 3; ++e) {
        const int se = st[e];
        const double s = ((double)v[n + sa + se] - (double)v[n + sa - se]) -
                         ((double)v[n - sa + se] - (double)v[n - sa - se]);
        S[a][e][c] = s;
        S[e][a][c] = s;
      }
    }
  }
  for (int c = 0; c < 3; ++c) {
    const T* B0 = B0s + c * N;
    b[c] = (double)B0[n];
    for (int a = 0; a < 3; ++a) Db[a][c] = (double)B0[n + st[a]] - (double)B0[n - st[a]];
  }
  double cof[3][3];
  for (int r = 0; r < 3; ++r) {
    const int r1 = (r + 1) % 3, r2 = (r + 2) % 3;
    cof[r][0] = G[1][r1] * G[2][r2] - G[2][r1] * G[1][r2];
    cof[r][1] = G[2][r1] * G[0][r2] - G[0][r1] * G[2][r2];
    cof[r][2] = G[0][r1] * G[1][r2] - G[1][r1] * G[0][r2];
  }
  const double det = ddet(G[0], G[1], G[2]);
  double V[3];
  for (int r = 0; r < 3; ++r) V[r] = G[0][r] * b[0] + G[1][r] * b[1] + G[2][r] * b[2];
  double DB[3][3];
  for (int c = 0; c < 3; ++c) {
    double Dd = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int r = 0; r < 3; ++r) Dd += cof[r][a] * S[a][c][r];
    for (int r = 0; r < 3; ++r) {
      double DV = 0.0;
      for (int a = 0; a < 3; ++a) DV += S[a][c][r] * b[a] + G[a][r] * Db[c][a];
      DB[c][r] = (DV - V[r] * Dd / det) / det;
    }
  }
  double gB[3][3];
  for (int r = 0; r < 3; ++r)
    for (int l = 0; l < 3; ++l)
      gB[r][l] = (DB[0][r] * cof[l][0] + DB[1][r] * cof[l][1] + DB[2][r] * cof[l][2]) / det;
  J[0] = gB[2][1] - gB[1][2];
  J[1] = gB[0][2] - gB[2][0];
  J[2] = gB[1][0] - gB[0][1];
  for (int r = 0; r < 3; ++r) B[r] = V[r] / det;
}

constexpr int DT = 256;

__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < DT / 32; ++w) t += sh[w];
  return t;
}

__device__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < DT / 32; ++w) t = fmax(t, sh[w]);
  return t;
}

// Sums of |x - x_ref|^2 and |B - B_ref|^2 per CTA.
template <typename T>
__global__ void __launch_bounds__(DT) k_deviation(DG g, const void* const* dbuf,
                                                  const DevState* st, const T* B0s,
                                                  const double* __restrict__ xref,
                                                  const double* __restrict__ Bref,
                                                  double* part) {
  __shared__ double sh[DT / 32];
  const T* d = (const T*)dbuf[st->cur];
  const int N = g.nx * g.ny * g.nz;
  double sx = 0.0, sb = 0.0;
  for (int n = blockIdx.x * DT + threadIdx.x; n < N; n += gridDim.x * DT) {
    const int i = n % g.nx, r = n / g.nx, j = r % g.ny, k = r / g.ny;
    const double X[3] = {g.lo[0] + i * g.h[0], g.lo[1] + j * g.h[1], g.lo[2] + k * g.h[2]};
    double G[3][3], B[3];
    pull_B(g, d, B0s, N, i, j, k, G, B);
    for (int c = 0; c < 3; ++c) {
      const double ex = (X[c] + (double)d[c * N + n]) - xref[c * N + n];
      const double eb = B[c] - Bref[c * N + n];
      sx += ex * ex;
      sb += eb * eb;
    }
  }
  sx = block_sum(sx, sh);
  sb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = sx;
    part[gridDim.x + blockIdx.x] = sb;
  }
}

__global__ void __launch_bounds__(DT) k_deviation_final(const double* part, int nb, double N,
                                                        double* out) {
  __shared__ double sh[DT / 32];
  double sx = 0.0, sb = 0.0;
  for (int b = threadIdx.x; b < nb; b += DT) {
    sx += part[b];
    sb += part[nb + b];
  }
  sx = block_sum(sx, sh);
  sb = block_sum(sb, sh);
  if (threadIdx.x == 0) {
    out[0] = sqrt(sx / N);
    out[1] = sqrt(sb / N);
  }
}

// alpha* at the interior nodes of the line (i, j, .) into out[0 .. nz-1]
// (NaN at the two boundary nodes) and epsilon* into out[nz]; one CTA,
// dynamic shared memory of nz doubles.
template <typename T, int CURL>
__global__ void __launch_bounds__(DT) k_alpha_line(DG g, const void* const* dbuf,
                                                   const DevState* st, const T* B0s, int i,
                                                   int j, double a_r, double* out) {
  extern __shared__ double al[];
  __shared__ double sh[DT / 32];
  const T* d = (const T*)dbuf[st->cur];
  const int N = g.nx * g.ny * g.nz;
  for (int k = threadIdx.x; k < g.nz; k += DT) {
    double a = NAN;
    if (k >= 1 && k <= g.nz - 2) {
      double J[3], B[3];
      if (CURL == GLEMUR_CURL_DIRECT)
        current_direct(g, d, B0s, N, i, j, k, J, B);
      else if (CURL == GLEMUR_CURL_NNN)
        current_nnn(g, d, B0s, N, i, j, k, J, B);
      else
        current_mimetic(g, d, B0s, N, i, j, k, J, B);
      a = ddot(J, B) / ddot(B, B);
    }
    al[k] = a;
    out[k] = a;
  }
  __syncthreads();
  double e = 0.0;
  for (int k = 1 + threadIdx.x; k <= g.nz - 2; k += DT)
    for (int l = 1; l <= g.nz - 2; ++l) {
      if (l == k) continue;
      const double v = a_r * (al[k] - al[l]) / (fabs((double)(k - l)) * g.h[2]);
      e = fmax(e, v);
    }
  e = block_max(e, sh);
  if (threadIdx.x == 0) out[g.nz] = e;
}

// kappa at every node (into kappa when non-null) and the number of concave
// nodes per CTA.
template <typename T>
__global__ void __launch_bounds__(DT) k_convexity(DG g, const void* const* dbuf,
                                                  const DevState* st, signed char* kappa,
                                                  double* part) {
  __shared__ double sh[DT / 32];
  const T* d = (const T*)dbuf[st->cur];
  const int N = g.nx * g.ny * g.nz;
  const int stp[3] = {1, g.nx, g.nx * g.ny};
  double cnt = 0.0;
  for (int n = blockIdx.x * DT + threadIdx.x; n < N; n += gridDim.x * DT) {
    const int id[3] = {n % g.nx, (n / g.nx) % g.ny, n / (g.nx * g.ny)};
    const int ext[3] = {g.nx, g.ny, g.nz};
    // x(neighbour) - x(node) along axis a, direction s: d difference + s h_a e_a
    bool ok = true;
    for (int oct = 0; oct < 8; ++oct) {
      const int sg[3] = {(oct & 1) ? 1 : -1, (oct & 2) ? 1 : -1, (oct & 4) ? 1 : -1};
      bool inside = true;
      for (int a = 0; a < 3; ++a) inside = inside && id[a] + sg[a] >= 0 && id[a] + sg[a] < ext[a];
      if (!inside) continue;
      double v[3][3];
      for (int a = 0; a < 3; ++a) {
        const int m = n + sg[a] * stp[a];
        for (int c = 0; c < 3; ++c) v[a][c] = (double)d[c * N + m] - (double)d[c * N + n];
        v[a][a] += sg[a] * g.h[a];
      }
      const double D = ddet(v[0], v[1], v[2]);
      const int sgn = D > 0.0 ? 1 : (D < 0.0 ? -1 : 0);
      if (sgn != sg[0] * sg[1] * sg[2]) ok = false;
    }
    if (kappa) kappa[n] = ok ? 1 : -1;
    if (!ok) cnt += 1.0;
  }
  cnt = block_sum(cnt, sh);
  if (threadIdx.x == 0) part[blockIdx.x] = cnt;
}

__global__ void __launch_bounds__(DT) k_count_final(const double* part, int nb, double* out) {
  __shared__ double sh[DT / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += DT) s += part[b];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

DG geom_of(const DiagCtx& c) {
  DG g;
  g.nx = c.nx;
  g.ny = c.ny;
  g.nz = c.nz;
  for (int a = 0; a < 3; ++a) {
    g.lo[a] = c.lo[a];
    g.h[a] = c.h[a];
    g.h2[a] = 2.0 * c.h[a];
  }
  g.periodic = c.periodic;
  return g;
}

int grid_blocks(const DiagCtx& c) {
  const long long N = (long long)c.nx * c.ny * c.nz;
  long long b = (N + DT - 1) / DT;
  if (b > c.max_blocks) b = c.max_blocks;
  if (b > 4096) b = 4096;
  return (int)(b < 1 ? 1 : b);
}

int finish(const DiagCtx& c, cudaError_t e, double* host, int count) {
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(host, c.stage, sizeof(double) * count, cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  return e == cudaSuccess ? GLEMUR_OK : GLEMUR_ERR_CUDA;
}

}  // namespace
}  // namespace glemur

using namespace glemur;

extern "C" {

int glemur_deviation(glemur_ctx* ctx, const double* x_ref, const double* B_ref,
                     double* sigma_x, double* sigma_B) {
  if (!ctx || !x_ref || !B_ref || !sigma_x || !sigma_B) return GLEMUR_ERR_BADARG;
  DiagCtx c;
  int rc = ctx_diag(ctx, &c);
  if (rc) return rc;
  const DG g = geom_of(c);
  const int nb = grid_blocks(c);
  if (c.precision == GLEMUR_MIXED)
    k_deviation<float><<<nb, DT, 0, c.s>>>(g, c.dbuf_dev, c.st, (const float*)c.B0s, x_ref,
                                           B_ref, c.part);
  else
    k_deviation<double><<<nb, DT, 0, c.s>>>(g, c.dbuf_dev, c.st, (const double*)c.B0s, x_ref,
                                            B_ref, c.part);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) {
    k_deviation_final<<<1, DT, 0, c.s>>>(c.part, nb, (double)c.nx * c.ny * c.nz, c.stage);
  }
  double out[2];
  rc = finish(c, e, out, 2);
  if (rc) return rc;
  *sigma_x = out[0];
  *sigma_B = out[1];
  return GLEMUR_OK;
}

int glemur_alpha_line(glemur_ctx* ctx, int i, int j, double a_r, double* alpha,
                      double* eps_star) {
  if (!ctx || !eps_star) return GLEMUR_ERR_BADARG;
  DiagCtx c;
  int rc = ctx_diag(ctx, &c);
  if (rc) return rc;
  // the line's alpha* values sit in shared memory (at most 48 KiB)
  if (i < 1 || i > c.nx - 2 || j < 1 || j > c.ny - 2 || !(a_r > 0) || c.nz > 6144)
    return GLEMUR_ERR_BADARG;
  const DG g = geom_of(c);
  const size_t sm = sizeof(double) * c.nz;
  const bool direct = c.curl == GLEMUR_CURL_DIRECT;
  if (c.curl == GLEMUR_CURL_NNN) {  // FP64 contexts only
    k_alpha_line<double, 2><<<1, DT, sm, c.s>>>(g, c.dbuf_dev, c.st, (const double*)c.B0s, i, j,
                                                a_r, c.stage);
  } else if (c.precision == GLEMUR_MIXED) {
    if (direct)
      k_alpha_line<float, 1><<<1, DT, sm, c.s>>>(g, c.dbuf_dev, c.st, (const float*)c.B0s, i, j,
                                                 a_r, c.stage);
    else
      k_alpha_line<float, 0><<<1, DT, sm, c.s>>>(g, c.dbuf_dev, c.st, (const float*)c.B0s, i, j,
                                                 a_r, c.stage);
  } else {
    if (direct)
      k_alpha_line<double, 1><<<1, DT, sm, c.s>>>(g, c.dbuf_dev, c.st, (const double*)c.B0s, i,
                                                  j, a_r, c.stage);
    else
      k_alpha_line<double, 0><<<1, DT, sm, c.s>>>(g, c.dbuf_dev, c.st, (const double*)c.B0s, i,
                                                  j, a_r, c.stage);
  }
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && alpha)
    e = cudaMemcpyAsync(alpha, c.stage, sizeof(double) * c.nz, cudaMemcpyDeviceToHost, c.s);
  double out;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&out, c.stage + c.nz, sizeof(double), cudaMemcpyDeviceToHost, c.s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.s);
  if (e != cudaSuccess) return GLEMUR_ERR_CUDA;
  *eps_star = out;
  return GLEMUR_OK;
}

int glemur_convexity(glemur_ctx* ctx, long long* n_concave, signed char* kappa) {
  if (!ctx || !n_concave) return GLEMUR_ERR_BADARG;
  DiagCtx c;
  int rc = ctx_diag(ctx, &c);
  if (rc) return rc;
  const DG g = geom_of(c);
  const int nb = grid_blocks(c);
  if (c.precision == GLEMUR_MIXED)
    k_convexity<float><<<nb, DT, 0, c.s>>>(g, c.dbuf_dev, c.st, kappa, c.part);
  else
    k_convexity<double><<<nb, DT, 0, c.s>>>(g, c.dbuf_dev, c.st, kappa, c.part);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) k_count_final<<<1, DT, 0, c.s>>>(c.part, nb, c.stage);
  double out;
  rc = finish(c, e, &out, 1);
  if (rc) return rc;
  *n_concave = (long long)out;
  return GLEMUR_OK;
}

}  // extern "C"
