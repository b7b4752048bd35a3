/*
 * FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY (see glemur_oracle.h).
 *
 * Plain restatement of the paper's method, in the paper's order and notation:
 *   section "Magnetic Field Relaxation", eq. "B transformation"  -> pull-back
 *   section "Mimetic Operators", eqs. "current discrete" ... "current matrix
 *       equation"                                                -> mimetic J
 *   eq. "magneto friction" (gamma = 1, mu_0 = 1)                  -> u = J x B
 *   section "Time Stepping", eq. "time stepping"                 -> Cash-Karp
 *       RK 5(4) with error-controlled step
 *   section "Boundary Conditions" (line-tied: u = 0 on the boundary)
 *   section "Diagnostics", eq. "magnetic energy" and the measure xi.
 * No blocking, fusion or algebraic shortcut is used: every quantity is built
 * the way the text defines it.  Built with -ffp-contract=off so that it
 * rounds identically on every host.
 */
#include "glemur_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ indexing */

static long n_nodes(const ora_grid* g) {
  return (long)g->nx * g->ny * g->nz;
}

static long node(const ora_grid* g, int i, int j, int k) {
  return ((long)k * g->ny + j) * g->nx + i;
}

static int extent(const ora_grid* g, int a) {
  return a == 0 ? g->nx : (a == 1 ? g->ny : g->nz);
}

static void get3(const ora_grid* g, const double* v, int i, int j, int k,
                 double out[3]) {
  long N = n_nodes(g), n = node(g, i, j, k);
  out[0] = v[n];
  out[1] = v[N + n];
  out[2] = v[2 * N + n];
}

static int is_interior(const ora_grid* g, int i, int j, int k) {
  return i > 0 && j > 0 && k > 0 && i < g->nx - 1 && j < g->ny - 1 &&
         k < g->nz - 1;
}

/* ------------------------------------------------- periodic boundaries */

/* Section "Boundary Conditions", periodic in z: the ghost planes k = 0 and
 * k = nz-1 repeat the last and first inner planes (f = 1, l = nz-2),
 * shifted by L_z + dZ, where L_z = Z_l - Z_f is the extent of the inner
 * planes and dZ the initial spacing: (nz - 3) h_z + h_z. */
static double period_z(const ora_grid* g) {
  return (double)(g->nz - 3) * g->h[2] + g->h[2];
}

static void refresh_ghosts(const ora_grid* g, double* x) {
  if (!g->periodic_z) return;
  long N = (long)g->nx * g->ny * g->nz;
  double P = period_z(g);
  for (int j = 0; j < g->ny; ++j)
    for (int i = 0; i < g->nx; ++i) {
      long f = ((long)1 * g->ny + j) * g->nx + i;
      long l = ((long)(g->nz - 2) * g->ny + j) * g->nx + i;
      long gf = ((long)0 * g->ny + j) * g->nx + i;
      long gl = ((long)(g->nz - 1) * g->ny + j) * g->nx + i;
      for (int c = 0; c < 3; ++c) {
        x[c * N + gf] = x[c * N + l] - (c == 2 ? P : 0.0);
        x[c * N + gl] = x[c * N + f] + (c == 2 ? P : 0.0);
      }
    }
}

/* The plane whose B a node's plane carries: ghosts carry their partner's
 * (B(X_{f-1}) = B(X_l), B(X_{l+1}) = B(X_f)). */
static int b_plane(const ora_grid* g, int k) {
  if (!g->periodic_z) return k;
  return k == 0 ? g->nz - 2 : (k == g->nz - 1 ? 1 : k);
}

/* ------------------------------------------------------------ 3-vectors */

static void cross(const double a[3], const double b[3], double out[3]) {
  out[0] = a[1] * b[2] - a[2] * b[1];
  out[1] = a[2] * b[0] - a[0] * b[2];
  out[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double norm(const double a[3]) { return sqrt(dot(a, a)); }

static double det3(const double F[9]) {
  return F[0] * (F[4] * F[8] - F[5] * F[7]) -
         F[1] * (F[3] * F[8] - F[5] * F[6]) +
         F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* Solve M y = r (3x3) by Gaussian elimination with partial pivoting.
 * Returns 0 on success, -1 if M is singular. */
static int solve3(const double Min[9], const double rin[3], double y[3]) {
  double M[3][4];
  for (int r = 0; r < 3; ++r) {
    for (int c = 0; c < 3; ++c) M[r][c] = Min[r * 3 + c];
    M[r][3] = rin[r];
  }
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
    if (M[piv][col] == 0.0) return -1;
    if (piv != col)
      for (int c = 0; c < 4; ++c) {
        double t = M[col][c];
        M[col][c] = M[piv][c];
        M[piv][c] = t;
      }
    for (int r = col + 1; r < 3; ++r) {
      double f = M[r][col] / M[col][col];
      for (int c = col; c < 4; ++c) M[r][c] -= f * M[col][c];
    }
  }
  for (int r = 2; r >= 0; --r) {
    double s = M[r][3];
    for (int c = r + 1; c < 3; ++c) s -= M[r][c] * y[c];
    y[r] = s / M[r][r];
  }
  return 0;
}

/* ------------------------------------------------------------ Jacobian */

/* d x / d X_b by second-order finite differences in index space: central
 * (x_{+1} - x_{-1}) / (2h) at interior indices, one-sided
 * (-3 x_0 + 4 x_1 - x_2) / (2h) on the lower face and its mirror image on the
 * upper face.  (The paper does not state the stencil; the second-order
 * one-sided form keeps affine maps exact on boundary nodes.) */
void ora_jacobian_at(const ora_grid* g, const double* x, int i, int j, int k,
                     double F[9]) {
  int idx[3] = {i, j, k};
  for (int b = 0; b < 3; ++b) {
    int n = extent(g, b);
    int p0[3] = {i, j, k}, p1[3] = {i, j, k}, p2[3] = {i, j, k};
    double w0, w1, w2;
    if (idx[b] > 0 && idx[b] < n - 1) {
      p0[b] = idx[b] - 1;
      p1[b] = idx[b] + 1;
      p2[b] = idx[b];
      w0 = -1.0;
      w1 = 1.0;
      w2 = 0.0;
    } else if (idx[b] == 0) {
      p0[b] = 0;
      p1[b] = 1;
      p2[b] = 2;
      w0 = -3.0;
      w1 = 4.0;
      w2 = -1.0;
    } else {
      p0[b] = n - 1;
      p1[b] = n - 2;
      p2[b] = n - 3;
      w0 = 3.0;
      w1 = -4.0;
      w2 = 1.0;
    }
    double x0[3], x1[3], x2[3];
    get3(g, x, p0[0], p0[1], p0[2], x0);
    get3(g, x, p1[0], p1[1], p1[2], x1);
    get3(g, x, p2[0], p2[1], p2[2], x2);
    for (int a = 0; a < 3; ++a)
      F[a * 3 + b] = (w0 * x0[a] + w1 * x1[a] + w2 * x2[a]) / (2.0 * g->h[b]);
  }
}

/* Eq. "B transformation": B_i = (1/Delta) sum_j (dx_i/dX_j) B_j(X, 0). */
static int pullback_at(const ora_grid* g, const double* x, const double* B0,
                       int i, int j, int k, double B[3], double* Delta) {
  double F[9], b0[3];
  ora_jacobian_at(g, x, i, j, k, F);
  get3(g, B0, i, j, k, b0);
  double D = det3(F);
  for (int a = 0; a < 3; ++a)
    B[a] = (F[a * 3 + 0] * b0[0] + F[a * 3 + 1] * b0[1] +
            F[a * 3 + 2] * b0[2]) / D;
  if (Delta) *Delta = D;
  return D <= 0.0 ? ORA_ERR_COLLAPSED : ORA_OK; /* NaN: left to the error norm */
}

int ora_pullback(const ora_grid* g, const double* x, const double* B0,
                 double* B, double* Delta) {
  long N = n_nodes(g);
  int rc = ORA_OK;
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double b[3], D;
        if (pullback_at(g, x, B0, i, j, b_plane(g, k), b, &D) != ORA_OK)
          rc = ORA_ERR_COLLAPSED;
        long n = node(g, i, j, k);
        B[n] = b[0];
        B[N + n] = b[1];
        B[2 * N + n] = b[2];
        if (Delta) Delta[n] = D;
      }
  return rc;
}

/* ------------------------------------------------------------ mimetic J */

/* The surfaces through node ijk: r = 0 is the jk grid surface (its normal
 * points along +X on an undistorted grid), r = 1 the ki surface, r = 2 the ij
 * surface; each is spanned by index directions (p, q) = (r+1, r+2) mod 3,
 * the cyclic permutation of the ij case drawn in the paper's first figure.
 * Loop vertices I..IV are the in-plane nearest neighbours +e_p, +e_q, -e_p,
 * -e_q, visited counter-clockwise about the +r direction. */
static void loop_vertices(int r, const int c[3], int v[4][3]) {
  int p = (r + 1) % 3, q = (r + 2) % 3;
  for (int m = 0; m < 4; ++m) {
    v[m][0] = c[0];
    v[m][1] = c[1];
    v[m][2] = c[2];
  }
  v[0][p] += 1; /* I   */
  v[1][q] += 1; /* II  */
  v[2][p] -= 1; /* III */
  v[3][q] -= 1; /* IV  */
}

/* One Stokes loop: eq. "current discrete" for the circulation and eqs.
 * "four surfaces" / "sum of triangles" for the vector area. */
static void stokes_loop(const double xv[4][3], const double Bv[4][3],
                        const double xc[3], double* circ, double nA[3],
                        double nA_four[3]) {
  double dx[4][3], Bm[4][3];
  for (int r = 0; r < 4; ++r)
    for (int a = 0; a < 3; ++a) {
      dx[r][a] = xv[(r + 1) % 4][a] - xv[r][a];           /* dx_1 = x_II - x_I */
      Bm[r][a] = (Bv[r][a] + Bv[(r + 1) % 4][a]) / 2.0;   /* B_1 = (B_I+B_II)/2 */
    }
  *circ = 0.0;
  for (int r = 0; r < 4; ++r) *circ += dot(Bm[r], dx[r]);
  /* eq. "sum of triangles" */
  nA[0] = nA[1] = nA[2] = 0.0;
  for (int r = 0; r < 4; ++r) {
    double t[3];
    cross(dx[r], dx[(r + 1) % 4], t);
    for (int a = 0; a < 3; ++a) nA[a] += t[a];
  }
  for (int a = 0; a < 3; ++a) nA[a] /= 4.0;
  /* eq. "four surfaces" (apex at x_ijk), kept as a self-check */
  nA_four[0] = nA_four[1] = nA_four[2] = 0.0;
  for (int r = 0; r < 4; ++r) {
    double s0[3], s1[3], t[3];
    for (int a = 0; a < 3; ++a) {
      s0[a] = xv[r][a] - xc[a];
      s1[a] = xv[(r + 1) % 4][a] - xc[a];
    }
    cross(s0, s1, t);
    for (int a = 0; a < 3; ++a) nA_four[a] += t[a] / 2.0;
  }
}

/* Eq. "current matrix equation" for the three surfaces: J . (n A)_r = c_r,
 * i.e. M J = c with the vector areas as rows of M.  (Solving with the
 * un-normalised areas is the same linear system as normalising each row by
 * its area A_r.) */
static int mimetic_solve(const double xv[3][4][3], const double Bv[3][4][3],
                         const double xc[3], double c[3], double M[9],
                         double J[3], double* gap) {
  for (int r = 0; r < 3; ++r) {
    double nA[3], nA4[3];
    stokes_loop(xv[r], Bv[r], xc, &c[r], nA, nA4);
    for (int a = 0; a < 3; ++a) M[r * 3 + a] = nA[a];
    if (gap) {
      double d[3] = {nA[0] - nA4[0], nA[1] - nA4[1], nA[2] - nA4[2]};
      double rel = norm(d) / norm(nA);
      if (!(rel <= *gap)) *gap = rel;
    }
  }
  if (solve3(M, c, J) != 0) return ORA_ERR_COLLAPSED;
  return ORA_OK;
}

int ora_mimetic_loops_at(const ora_grid* g, const double* x, const double* B,
                         int i, int j, int k, double c[3], double M[9],
                         double J[3]) {
  if (!is_interior(g, i, j, k)) return ORA_ERR_BADARG;
  int ctr[3] = {i, j, k};
  double xv[3][4][3], Bv[3][4][3], xc[3];
  get3(g, x, i, j, k, xc);
  for (int r = 0; r < 3; ++r) {
    int v[4][3];
    loop_vertices(r, ctr, v);
    for (int m = 0; m < 4; ++m) {
      get3(g, x, v[m][0], v[m][1], v[m][2], xv[r][m]);
      get3(g, B, v[m][0], v[m][1], v[m][2], Bv[r][m]);
    }
  }
  return mimetic_solve(xv, Bv, xc, c, M, J, NULL);
}

int ora_curl_mimetic(const ora_grid* g, const double* x, const double* B,
                     double* J, double* area_gap) {
  long N = n_nodes(g);
  int rc = ORA_OK;
  if (area_gap) *area_gap = 0.0;
  memset(J, 0, sizeof(double) * 3 * N);
  for (int k = 1; k < g->nz - 1; ++k)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        int ctr[3] = {i, j, k};
        double xv[3][4][3], Bv[3][4][3], xc[3], c[3], M[9], Jn[3];
        get3(g, x, i, j, k, xc);
        for (int r = 0; r < 3; ++r) {
          int v[4][3];
          loop_vertices(r, ctr, v);
          for (int m = 0; m < 4; ++m) {
            get3(g, x, v[m][0], v[m][1], v[m][2], xv[r][m]);
            get3(g, B, v[m][0], v[m][1], v[m][2], Bv[r][m]);
          }
        }
        if (mimetic_solve(xv, Bv, xc, c, M, Jn, area_gap) != ORA_OK)
          rc = ORA_ERR_COLLAPSED;
        long n = node(g, i, j, k);
        J[n] = Jn[0];
        J[N + n] = Jn[1];
        J[2 * N + n] = Jn[2];
      }
  return rc;
}

/* ---------------------------------------------------- next-nearest J */

/* The octilateral of section "Next Nearest Neighbor Mimetic Approach" in
 * surface r (spanned by index directions p = r+1, q = r+2 mod 3, as for the
 * nearest-neighbour loops): the eight in-plane neighbours visited
 * counter-clockwise about +r, starting at a corner,
 *   V1 = +e_p - e_q, V2 = +e_p, V3 = +e_p + e_q, V4 = +e_q,
 *   V5 = -e_p + e_q, V6 = -e_p, V7 = -e_p - e_q, V8 = -e_q,
 * so that edges 2 and 3, 4 and 5, 6 and 7, 8 and 1 meet at the four
 * corners, as the corner triangles of eq. "eight surfaces" need. */
static void octilateral_vertices(int r, const int c[3], int v[8][3]) {
  static const int off[8][2] = {{1, -1}, {1, 0},  {1, 1},   {0, 1},
                                {-1, 1}, {-1, 0}, {-1, -1}, {0, -1}};
  int p = (r + 1) % 3, q = (r + 2) % 3;
  for (int m = 0; m < 8; ++m) {
    v[m][0] = c[0];
    v[m][1] = c[1];
    v[m][2] = c[2];
    v[m][p] += off[m][0];
    v[m][q] += off[m][1];
  }
}

/* Eq. "current discrete" over the octilateral (edge-mean B, eight
 * contributions) and its vector area by eq. "sum of eight triangles": the
 * four corner triangles dx_2 x dx_3 / 2, ..., dx_8 x dx_1 / 2 and the inner
 * quadrilateral through V2, V4, V6, V8 with edges dx_A .. dx_D, whose area
 * is (dx_A x dx_B + dx_B x dx_C + dx_C x dx_D + dx_D x dx_A) / 4. */
static void octilateral_loop(const double xv[8][3], const double Bv[8][3],
                             double* circ, double nA[3]) {
  double dx[8][3];
  *circ = 0.0;
  for (int r = 0; r < 8; ++r) {
    double Bm[3];
    for (int a = 0; a < 3; ++a) {
      dx[r][a] = xv[(r + 1) % 8][a] - xv[r][a];
      Bm[a] = (Bv[r][a] + Bv[(r + 1) % 8][a]) / 2.0;
    }
    *circ += dot(Bm, dx[r]);
  }
  nA[0] = nA[1] = nA[2] = 0.0;
  /* corner triangles: (dx_2, dx_3), (dx_4, dx_5), (dx_6, dx_7), (dx_8, dx_1) */
  for (int t = 0; t < 4; ++t) {
    double c[3];
    cross(dx[2 * t + 1], dx[(2 * t + 2) % 8], c);
    for (int a = 0; a < 3; ++a) nA[a] += c[a] / 2.0;
  }
  /* inner quadrilateral V2 -> V4 -> V6 -> V8 */
  double q[4][3];
  for (int a = 0; a < 3; ++a) {
    q[0][a] = xv[3][a] - xv[1][a]; /* dx_A */
    q[1][a] = xv[5][a] - xv[3][a]; /* dx_B */
    q[2][a] = xv[7][a] - xv[5][a]; /* dx_C */
    q[3][a] = xv[1][a] - xv[7][a]; /* dx_D */
  }
  for (int t = 0; t < 4; ++t) {
    double c[3];
    cross(q[t], q[(t + 1) % 4], c);
    for (int a = 0; a < 3; ++a) nA[a] += c[a] / 4.0;
  }
}

/* Next-nearest-neighbour current at interior node (i, j, k): the three
 * octilaterals' vector areas as the rows of M and their circulations as c
 * in eq. "current matrix equation", M J = c. */
static int nnn_at(const ora_grid* g, const double* x, const double* B, int i,
                  int j, int k, double J[3]) {
  int ctr[3] = {i, j, k};
  double M[9], c[3];
  for (int r = 0; r < 3; ++r) {
    int v[8][3];
    double xv[8][3], Bv[8][3], nA[3];
    octilateral_vertices(r, ctr, v);
    for (int m = 0; m < 8; ++m) {
      get3(g, x, v[m][0], v[m][1], v[m][2], xv[m]);
      get3(g, B, v[m][0], v[m][1], v[m][2], Bv[m]);
    }
    octilateral_loop(xv, Bv, &c[r], nA);
    for (int a = 0; a < 3; ++a) M[r * 3 + a] = nA[a];
  }
  return solve3(M, c, J) == 0 ? ORA_OK : ORA_ERR_COLLAPSED;
}

int ora_curl_nnn(const ora_grid* g, const double* x, const double* B,
                 double* J) {
  long N = n_nodes(g);
  int rc = ORA_OK;
  memset(J, 0, sizeof(double) * 3 * N);
  for (int k = 1; k < g->nz - 1; ++k)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        double Jn[3];
        if (nnn_at(g, x, B, i, j, k, Jn) != ORA_OK) rc = ORA_ERR_COLLAPSED;
        long n = node(g, i, j, k);
        J[n] = Jn[0];
        J[N + n] = Jn[1];
        J[2 * N + n] = Jn[2];
      }
  return rc;
}

/* ------------------------------------------------------------ direct J */

/* Classic current at one interior node.  With W = F B0 and B = W / Delta,
 *   dW_a/dX_c     = sum_b (d2 x_a / dX_b dX_c) B0_b + F_ab dB0_b/dX_c
 *   dDelta/dX_c   = sum_ab cof(F)_ab d2 x_a / dX_b dX_c      (Jacobi)
 *   dB_a/dX_c     = dW_a/dX_c / Delta - W_a dDelta/dX_c / Delta^2
 *   dB_a/dx_l     = sum_c dB_a/dX_c (F^-1)_cl
 *   J             = curl_x B.
 * Derivatives are second-order central differences in index space. */
static int direct_at(const ora_grid* g, const double* x, const double* B0,
                     int i, int j, int k, double J[3], double Bc[3]) {
  int ctr[3] = {i, j, k};
  double F[9], xc[3], b0c[3];
  ora_jacobian_at(g, x, i, j, k, F);
  get3(g, x, i, j, k, xc);
  get3(g, B0, i, j, k, b0c);
  /* second derivatives H[a][b][c] = d2 x_a / dX_b dX_c */
  double H[3][3][3];
  for (int b = 0; b < 3; ++b)
    for (int c = 0; c < 3; ++c) {
      double val[3];
      if (b == c) {
        int pp[3] = {i, j, k}, mm[3] = {i, j, k};
        pp[b] += 1;
        mm[b] -= 1;
        double xp[3], xm[3];
        get3(g, x, pp[0], pp[1], pp[2], xp);
        get3(g, x, mm[0], mm[1], mm[2], xm);
        for (int a = 0; a < 3; ++a)
          val[a] = (xp[a] - 2.0 * xc[a] + xm[a]) / (g->h[b] * g->h[b]);
      } else {
        int s[4][3];
        double sg[4] = {1.0, -1.0, -1.0, 1.0};
        int db[4] = {1, 1, -1, -1}, dc[4] = {1, -1, 1, -1};
        double acc[3] = {0.0, 0.0, 0.0};
        for (int m = 0; m < 4; ++m) {
          s[m][0] = ctr[0];
          s[m][1] = ctr[1];
          s[m][2] = ctr[2];
          s[m][b] += db[m];
          s[m][c] += dc[m];
          double xs[3];
          get3(g, x, s[m][0], s[m][1], s[m][2], xs);
          for (int a = 0; a < 3; ++a) acc[a] += sg[m] * xs[a];
        }
        for (int a = 0; a < 3; ++a)
          val[a] = acc[a] / (4.0 * g->h[b] * g->h[c]);
      }
      for (int a = 0; a < 3; ++a) H[a][b][c] = val[a];
    }
  /* dB0_b / dX_c */
  double dB0[3][3];
  for (int c = 0; c < 3; ++c) {
    int pp[3] = {i, j, k}, mm[3] = {i, j, k};
    pp[c] += 1;
    mm[c] -= 1;
    double bp[3], bm[3];
    get3(g, B0, pp[0], pp[1], pp[2], bp);
    get3(g, B0, mm[0], mm[1], mm[2], bm);
    for (int b = 0; b < 3; ++b) dB0[b][c] = (bp[b] - bm[b]) / (2.0 * g->h[c]);
  }
  /* cofactors: rows of cof(F) are cross products of the rows of F */
  double cof[9], r0[3] = {F[0], F[1], F[2]}, r1[3] = {F[3], F[4], F[5]},
                 r2[3] = {F[6], F[7], F[8]};
  cross(r1, r2, &cof[0]);
  cross(r2, r0, &cof[3]);
  cross(r0, r1, &cof[6]);
  double D = det3(F);
  if (D <= 0.0) return ORA_ERR_COLLAPSED;
  double W[3];
  for (int a = 0; a < 3; ++a)
    W[a] = F[a * 3 + 0] * b0c[0] + F[a * 3 + 1] * b0c[1] + F[a * 3 + 2] * b0c[2];
  double dW[3][3], dD[3], dB[3][3];
  for (int c = 0; c < 3; ++c) {
    dD[c] = 0.0;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) dD[c] += cof[a * 3 + b] * H[a][b][c];
    for (int a = 0; a < 3; ++a) {
      dW[a][c] = 0.0;
      for (int b = 0; b < 3; ++b)
        dW[a][c] += H[a][b][c] * b0c[b] + F[a * 3 + b] * dB0[b][c];
    }
  }
  for (int a = 0; a < 3; ++a)
    for (int c = 0; c < 3; ++c)
      dB[a][c] = dW[a][c] / D - W[a] * dD[c] / (D * D);
  /* F^-1 = adj(F) / Delta, adj(F)_{cb} = cof(F)_{bc} */
  double Finv[3][3];
  for (int c = 0; c < 3; ++c)
    for (int l = 0; l < 3; ++l) Finv[c][l] = cof[l * 3 + c] / D;
  double gB[3][3]; /* gB[a][l] = dB_a / dx_l */
  for (int a = 0; a < 3; ++a)
    for (int l = 0; l < 3; ++l) {
      gB[a][l] = 0.0;
      for (int c = 0; c < 3; ++c) gB[a][l] += dB[a][c] * Finv[c][l];
    }
  J[0] = gB[2][1] - gB[1][2];
  J[1] = gB[0][2] - gB[2][0];
  J[2] = gB[1][0] - gB[0][1];
  if (Bc)
    for (int a = 0; a < 3; ++a) Bc[a] = W[a] / D;
  return ORA_OK;
}

int ora_curl_direct(const ora_grid* g, const double* x, const double* B0,
                    double* J) {
  long N = n_nodes(g);
  int rc = ORA_OK;
  memset(J, 0, sizeof(double) * 3 * N);
  for (int k = 1; k < g->nz - 1; ++k)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        double Jn[3];
        if (direct_at(g, x, B0, i, j, k, Jn, NULL) != ORA_OK) {
          rc = ORA_ERR_COLLAPSED;
          Jn[0] = Jn[1] = Jn[2] = 0.0;
        }
        long n = node(g, i, j, k);
        J[n] = Jn[0];
        J[N + n] = Jn[1];
        J[2 * N + n] = Jn[2];
      }
  return rc;
}

/* ------------------------------------------------------------ velocity */

/* J of the selected current at every interior node (0 elsewhere), B the
 * pulled-back field on the same positions. */
static int curl_of(const ora_grid* g, int curl, const double* x, const double* B0,
                   const double* B, double* J) {
  if (curl == ORA_CURL_DIRECT) return ora_curl_direct(g, x, B0, J);
  if (curl == ORA_CURL_NNN) return ora_curl_nnn(g, x, B, J);
  return ora_curl_mimetic(g, x, B, J, NULL);
}

/* B (eq. "B transformation") and J of state x; with periodic z the ghost
 * planes of (a copy of) x are first set from the inner planes. */
static int state_fields(const ora_grid* g, int curl, const double* x,
                        const double* B0, double* B, double* J) {
  long n = 3 * n_nodes(g);
  const double* xs = x;
  double* xc = NULL;
  if (g->periodic_z) {
    xc = (double*)malloc(sizeof(double) * n);
    if (!xc) return ORA_ERR_BADARG;
    memcpy(xc, x, sizeof(double) * n);
    refresh_ghosts(g, xc);
    xs = xc;
  }
  int rc = ora_pullback(g, xs, B0, B, NULL);
  int rc2 = curl_of(g, curl, xs, B0, B, J);
  free(xc);
  return rc == ORA_OK ? rc2 : rc;
}

void ora_lorentz_velocity(const ora_grid* g, const double* J, const double* B,
                          double* u) {
  long N = n_nodes(g);
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        long n = node(g, i, j, k);
        double un[3] = {0.0, 0.0, 0.0};
        if (is_interior(g, i, j, k)) {
          double Jn[3], Bn[3];
          get3(g, J, i, j, k, Jn);
          get3(g, B, i, j, k, Bn);
          cross(Jn, Bn, un); /* gamma = 1 */
        }
        u[n] = un[0];
        u[N + n] = un[1];
        u[2 * N + n] = un[2];
      }
}

int ora_velocity(const ora_grid* g, int curl, const double* x,
                 const double* B0, double* u) {
  long N = n_nodes(g);
  double* B = (double*)malloc(sizeof(double) * 3 * N);
  double* J = (double*)malloc(sizeof(double) * 3 * N);
  if (!B || !J) {
    free(B);
    free(J);
    return ORA_ERR_BADARG;
  }
  int rc = state_fields(g, curl, x, B0, B, J);
  ora_lorentz_velocity(g, J, B, u);
  free(B);
  free(J);
  return rc;
}

int ora_velocity_at(const ora_grid* g, int curl, const double* x,
                    const double* B0, int i, int j, int k, double u[3]) {
  if (g->periodic_z) return ORA_ERR_BADARG; /* whole-grid ora_velocity only */
  if (!is_interior(g, i, j, k)) {
    u[0] = u[1] = u[2] = 0.0;
    return ORA_OK;
  }
  double J[3], Bc[3];
  if (curl == ORA_CURL_DIRECT) {
    int rc = direct_at(g, x, B0, i, j, k, J, Bc);
    if (rc != ORA_OK) return rc;
  } else if (curl == ORA_CURL_NNN) {
    /* B at the node's 3x3x3 neighbourhood (a small local copy) */
    ora_grid lg = {3, 3, 3, {g->h[0], g->h[1], g->h[2]}, 0};
    double lx[81], lB[81];
    for (int c = 0; c < 3; ++c)
      for (int dk = 0; dk < 3; ++dk)
        for (int dj = 0; dj < 3; ++dj)
          for (int di = 0; di < 3; ++di) {
            long m = node(&lg, di, dj, dk);
            lx[c * 27 + m] = x[c * n_nodes(g) + node(g, i + di - 1, j + dj - 1, k + dk - 1)];
          }
    for (int dk = 0; dk < 3; ++dk)
      for (int dj = 0; dj < 3; ++dj)
        for (int di = 0; di < 3; ++di) {
          double b[3];
          if (pullback_at(g, x, B0, i + di - 1, j + dj - 1, k + dk - 1, b, NULL) != ORA_OK)
            return ORA_ERR_COLLAPSED;
          long m = node(&lg, di, dj, dk);
          for (int c = 0; c < 3; ++c) lB[c * 27 + m] = b[c];
        }
    int rc = nnn_at(&lg, lx, lB, 1, 1, 1, J);
    if (rc != ORA_OK) return rc;
    if (pullback_at(g, x, B0, i, j, k, Bc, NULL) != ORA_OK)
      return ORA_ERR_COLLAPSED;
  } else {
    int ctr[3] = {i, j, k};
    double xv[3][4][3], Bv[3][4][3], xc[3], c[3], M[9];
    get3(g, x, i, j, k, xc);
    for (int r = 0; r < 3; ++r) {
      int v[4][3];
      loop_vertices(r, ctr, v);
      for (int m = 0; m < 4; ++m) {
        get3(g, x, v[m][0], v[m][1], v[m][2], xv[r][m]);
        if (pullback_at(g, x, B0, v[m][0], v[m][1], v[m][2], Bv[r][m], NULL) !=
            ORA_OK)
          return ORA_ERR_COLLAPSED;
      }
    }
    int rc = mimetic_solve(xv, Bv, xc, c, M, J, NULL);
    if (rc != ORA_OK) return rc;
    if (pullback_at(g, x, B0, i, j, k, Bc, NULL) != ORA_OK)
      return ORA_ERR_COLLAPSED;
  }
  cross(J, Bc, u);
  return ORA_OK;
}

/* ------------------------------------------------------------ Cash-Karp */

/* Embedded Runge-Kutta 5(4) pair of Cash & Karp (ACM TOMS 16, 1990), the
 * scheme the paper cites for its time stepping. */
void ora_cash_karp_tableau(double c[6], double a[36], double b5[6],
                           double b4[6]) {
  static const double C[6] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 3.0 / 5.0, 1.0,
                              7.0 / 8.0};
  static const double A[6][6] = {
      {0, 0, 0, 0, 0, 0},
      {1.0 / 5.0, 0, 0, 0, 0, 0},
      {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
      {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0, 0},
      {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0, 0},
      {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0,
       253.0 / 4096.0, 0}};
  static const double B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0,
                               125.0 / 594.0, 0.0, 512.0 / 1771.0};
  static const double B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0,
                               13525.0 / 55296.0, 277.0 / 14336.0, 1.0 / 4.0};
  for (int s = 0; s < 6; ++s) {
    c[s] = C[s];
    b5[s] = B5[s];
    b4[s] = B4[s];
    for (int j = 0; j < 6; ++j) a[s * 6 + j] = A[s][j];
  }
}

int ora_ck_attempt(long n, const double* y, double dt, ora_rhs_fn f,
                   void* ctx, double* ynew, double* yerr, double* kout) {
  double c[6], a[36], b5[6], b4[6];
  ora_cash_karp_tableau(c, a, b5, b4);
  double* k = kout ? kout : (double*)malloc(sizeof(double) * 6 * n);
  double* ys = (double*)malloc(sizeof(double) * n);
  if (!k || !ys) {
    if (!kout) free(k);
    free(ys);
    return ORA_ERR_BADARG;
  }
  int rc = ORA_OK;
  for (int s = 0; s < 6; ++s) {
    /* stage input y_s = y + dt sum_{j<s} a_sj k_j */
    for (long m = 0; m < n; ++m) {
      double acc = 0.0;
      for (int j = 0; j < s; ++j) acc += a[s * 6 + j] * k[(long)j * n + m];
      ys[m] = y[m] + dt * acc;
    }
    int r = f(ctx, ys, &k[(long)s * n]);
    if (r != ORA_OK && rc == ORA_OK) rc = r;
  }
  for (long m = 0; m < n; ++m) {
    double acc5 = 0.0, acce = 0.0;
    for (int j = 0; j < 6; ++j) {
      acc5 += b5[j] * k[(long)j * n + m];
      acce += (b5[j] - b4[j]) * k[(long)j * n + m];
    }
    ynew[m] = y[m] + dt * acc5;
    yerr[m] = dt * acce;
  }
  if (!kout) free(k);
  free(ys);
  return rc;
}

/* Eq. "time stepping" with the acceptance rule around it. */
int ora_step_control(const ora_control_opts* o, double lambda, double dt,
                     int consecutive_rejects, double* dt_next, int* accept) {
  if (!isfinite(lambda) || !isfinite(dt)) {
    *accept = 0;
    *dt_next = dt;
    return ORA_ERR_NONFINITE;
  }
  if (lambda > o->lambda0) {
    double fac = o->safety * pow(o->lambda0 / lambda, 0.2);
    if (fac < o->shrink_min) fac = o->shrink_min;
    *accept = 0;
    *dt_next = dt * fac;
    if (consecutive_rejects + 1 > o->max_rejects || *dt_next < o->dt_min)
      return ORA_ERR_DT_UNDERFLOW;
    return ORA_OK;
  }
  *accept = 1;
  double fac = 1.0;
  if (lambda < 0.5 * o->lambda0) {
    fac = lambda > 0.0 ? o->safety * pow(o->lambda0 / lambda, 0.2) : o->grow_max;
    if (fac > o->grow_max) fac = o->grow_max;
  }
  *dt_next = dt * fac;
  return ORA_OK;
}

/* ------------------------------------------------------------ relaxation */

typedef struct {
  const ora_grid* g;
  int curl;
  const double* B0;
} rhs_ctx;

static int grid_rhs(void* vctx, const double* y, double* dydt) {
  rhs_ctx* c = (rhs_ctx*)vctx;
  return ora_velocity(c->g, c->curl, y, c->B0, dydt);
}

/* ORA_ERR_COLLAPSED if det(dx/dX) <= 0 at some node of x. */
static int pullback_status(const ora_grid* g, const double* x,
                           const double* B0) {
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double b[3];
        if (pullback_at(g, x, B0, i, j, b_plane(g, k), b, NULL) != ORA_OK)
          return ORA_ERR_COLLAPSED;
      }
  return ORA_OK;
}

static double max_abs(long n, const double* v) {
  double m = 0.0;
  for (long i = 0; i < n; ++i) {
    double a = fabs(v[i]);
    if (!(a <= m)) m = a; /* NaN propagates */
  }
  return m;
}

int ora_step_fixed(const ora_grid* g, int curl, double* x, const double* B0,
                   double dt, double* lambda) {
  long n = 3 * n_nodes(g);
  double* xn = (double*)malloc(sizeof(double) * n);
  double* er = (double*)malloc(sizeof(double) * n);
  if (!xn || !er) {
    free(xn);
    free(er);
    return ORA_ERR_BADARG;
  }
  rhs_ctx c = {g, curl, B0};
  int rc = ora_ck_attempt(n, x, dt, grid_rhs, &c, xn, er, NULL);
  if (lambda) *lambda = max_abs(n, er);
  memcpy(x, xn, sizeof(double) * n);
  refresh_ghosts(g, x);
  free(xn);
  free(er);
  return rc;
}

int ora_relax(const ora_grid* g, int curl, const ora_control_opts* o,
              double* x, const double* B0, int n_accept, double* dt,
              double* dt_log, ora_stats* st) {
  long n = 3 * n_nodes(g);
  double* xn = (double*)malloc(sizeof(double) * n);
  double* er = (double*)malloc(sizeof(double) * n);
  if (!xn || !er) {
    free(xn);
    free(er);
    return ORA_ERR_BADARG;
  }
  rhs_ctx c = {g, curl, B0};
  int acc = 0, rej = 0, consec = 0, rc = ORA_OK;
  double t = st ? st->t : 0.0, lam = 0.0;
  while (acc < n_accept) {
    rc = ora_ck_attempt(n, x, *dt, grid_rhs, &c, xn, er, NULL);
    double dt_next;
    int accept;
    if (rc == ORA_ERR_COLLAPSED) {
      /* A stage input folded the grid.  If the accepted state itself is
       * folded the run cannot continue; otherwise the attempt is rejected
       * with the largest shrink (its error is unbounded), which is how the
       * step size collapses before a blow-up (section "Grid Convexity and
       * Stability"). */
      if (pullback_status(g, x, B0) != ORA_OK) break;
      lam = INFINITY;
      rc = ora_step_control(o, DBL_MAX, *dt, consec, &dt_next, &accept);
    } else {
      if (rc != ORA_OK) break;
      lam = max_abs(n, er); /* Lambda: maximum error in x */
      rc = ora_step_control(o, lam, *dt, consec, &dt_next, &accept);
    }
    if (rc != ORA_OK) {
      if (!accept) ++rej;
      break;
    }
    if (accept) {
      memcpy(x, xn, sizeof(double) * n);
      refresh_ghosts(g, x);
      t += *dt;
      if (dt_log) dt_log[acc] = *dt;
      ++acc;
      consec = 0;
    } else {
      ++rej;
      ++consec;
    }
    *dt = dt_next;
  }
  if (st) {
    st->accepted = acc;
    st->rejected = rej;
    st->dt = *dt;
    st->t = t;
    st->lambda = lam;
  }
  free(xn);
  free(er);
  return rc;
}

/* ------------------------------------------------------------ diagnostics */

int ora_energy(const ora_grid* g, const double* x, const double* B0,
               double* E) {
  double sum = 0.0;
  int rc = ORA_OK;
  /* periodic in z: one period, the inner planes, none of them on a z face */
  int k0 = g->periodic_z ? 1 : 0, k1 = g->periodic_z ? g->nz - 1 : g->nz;
  for (int k = k0; k < k1; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double B[3], D;
        if (pullback_at(g, x, B0, i, j, k, B, &D) != ORA_OK)
          rc = ORA_ERR_COLLAPSED;
        /* zeta = 1, 1/2, 1/4, 1/8 inside, on faces, edges, corners */
        double zeta = 1.0;
        if (i == 0 || i == g->nx - 1) zeta *= 0.5;
        if (j == 0 || j == g->ny - 1) zeta *= 0.5;
        if (!g->periodic_z && (k == 0 || k == g->nz - 1)) zeta *= 0.5;
        sum += zeta * dot(B, B) * D;
      }
  *E = 0.5 * sum * g->h[0] * g->h[1] * g->h[2];
  return rc;
}

int ora_forcefree(const ora_grid* g, int curl, const double* x,
                  const double* B0, double* xi, double* xi_sin) {
  long N = n_nodes(g);
  double* B = (double*)malloc(sizeof(double) * 3 * N);
  double* J = (double*)malloc(sizeof(double) * 3 * N);
  if (!B || !J) {
    free(B);
    free(J);
    return ORA_ERR_BADARG;
  }
  int rc = state_fields(g, curl, x, B0, B, J);
  double m1 = 0.0, m2 = 0.0;
  for (int k = 1; k < g->nz - 1; ++k)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        double Jn[3], Bn[3], f[3];
        get3(g, J, i, j, k, Jn);
        get3(g, B, i, j, k, Bn);
        cross(Jn, Bn, f);
        double fm = norm(f), b2 = dot(Bn, Bn), jb = norm(Jn) * norm(Bn);
        double r1 = fm / b2;
        if (!(r1 <= m1)) m1 = r1;
        if (jb > 1e-300) {
          double r2 = fm / jb;
          if (!(r2 <= m2)) m2 = r2;
        }
      }
  *xi = m1;
  *xi_sin = m2;
  free(B);
  free(J);
  return rc;
}

/* ------------------------------------------- validation diagnostics */

/* Section "Deviation from the Exact Known Equilibrium": sigma_x and sigma_B,
 * root-mean-square over all N nodes of |x - x_ref| and |B - B_ref|. */
int ora_deviation(const ora_grid* g, const double* x, const double* B0,
                  const double* x_ref, const double* B_ref, double* sigma_x,
                  double* sigma_B) {
  long N = n_nodes(g);
  double* B = (double*)malloc(sizeof(double) * 3 * N);
  if (!B) return ORA_ERR_BADARG;
  int rc = ora_pullback(g, x, B0, B, NULL);
  double sx = 0.0, sb = 0.0;
  for (long n = 0; n < N; ++n)
    for (int c = 0; c < 3; ++c) {
      double dx = x[c * N + n] - x_ref[c * N + n];
      double db = B[c * N + n] - B_ref[c * N + n];
      sx += dx * dx;
      sb += db * db;
    }
  *sigma_x = sqrt(sx / (double)N);
  *sigma_B = sqrt(sb / (double)N);
  free(B);
  return rc;
}

/* Section "Force-Freeness": alpha* = J.B / B^2 at the interior nodes
 * (i, j, k), k = 1 .. nz-2, of the node line through (i, j) (alpha[k]; the
 * two boundary entries, where the current is not defined, are NaN), and
 * eq. "epsilon star": the largest a_r (alpha*_k - alpha*_l) / |X_k - X_l|
 * over pairs of those nodes, |X_k - X_l| = |k - l| h_z on the line. */
int ora_alpha_line(const ora_grid* g, int curl, const double* x,
                   const double* B0, int i, int j, double a_r, double* alpha,
                   double* eps_star) {
  if (i < 1 || i > g->nx - 2 || j < 1 || j > g->ny - 2) return ORA_ERR_BADARG;
  long N = n_nodes(g);
  double* B = (double*)malloc(sizeof(double) * 3 * N);
  double* J = (double*)malloc(sizeof(double) * 3 * N);
  if (!B || !J) {
    free(B);
    free(J);
    return ORA_ERR_BADARG;
  }
  int rc = state_fields(g, curl, x, B0, B, J);
  alpha[0] = alpha[g->nz - 1] = NAN;
  for (int k = 1; k < g->nz - 1; ++k) {
    double Jn[3], Bn[3];
    get3(g, J, i, j, k, Jn);
    get3(g, B, i, j, k, Bn);
    alpha[k] = dot(Jn, Bn) / dot(Bn, Bn);
  }
  double e = 0.0;
  for (int k = 1; k < g->nz - 1; ++k)
    for (int l = 1; l < g->nz - 1; ++l) {
      if (l == k) continue;
      double v = a_r * (alpha[k] - alpha[l]) / (fabs((double)(k - l)) * g->h[2]);
      if (!(v <= e)) e = v;
    }
  *eps_star = e;
  free(B);
  free(J);
  return rc;
}

/* Section "Convexity", eq. "convexity": at node (i, j, k) the trihedra of
 * dx^lambda = x(i+di, j, k) - x, dx^mu = x(i, j+dj, k) - x and
 * dx^nu = x(i, j, k+dk) - x for the eight sign choices (di, dj, dk); the
 * node is convex (kappa = +1) when the determinant of every trihedron whose
 * three neighbours exist has the sign di dj dk, else kappa = -1.  kappa
 * (N ints) may be NULL; *n_concave counts the nodes with kappa = -1. */
int ora_convexity(const ora_grid* g, const double* x, int* kappa,
                  long* n_concave) {
  long cnt = 0;
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        double xc[3];
        get3(g, x, i, j, k, xc);
        int ok = 1;
        for (int di = -1; di <= 1; di += 2)
          for (int dj = -1; dj <= 1; dj += 2)
            for (int dk = -1; dk <= 1; dk += 2) {
              if (i + di < 0 || i + di >= g->nx || j + dj < 0 || j + dj >= g->ny ||
                  k + dk < 0 || k + dk >= g->nz)
                continue;
              double a[3], b[3], c[3], F[9];
              get3(g, x, i + di, j, k, a);
              get3(g, x, i, j + dj, k, b);
              get3(g, x, i, j, k + dk, c);
              for (int r = 0; r < 3; ++r) {
                F[r * 3 + 0] = a[r] - xc[r];
                F[r * 3 + 1] = b[r] - xc[r];
                F[r * 3 + 2] = c[r] - xc[r];
              }
              double D = det3(F);
              int sgn = D > 0.0 ? 1 : (D < 0.0 ? -1 : 0);
              if (sgn != di * dj * dk) ok = 0;
            }
        if (kappa) kappa[node(g, i, j, k)] = ok ? 1 : -1;
        if (!ok) ++cnt;
      }
  *n_concave = cnt;
  return ORA_OK;
}
