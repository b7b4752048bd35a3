/*
 * Complex-step derivatives of the relaxation -- TEST INFRASTRUCTURE ONLY.
 *
 * The same plain restatement of the method as glemur_oracle.c (pull-back of
 * eq. "B transformation", the nearest-neighbour loops of eqs. "current
 * discrete" / "sum of triangles" / "current matrix equation", u = J x B of
 * eq. "magneto friction" with line-tied boundaries, Cash-Karp stages of
 * section "Time Stepping" at a given step-size schedule, eq. "magnetic
 * energy" and xi), evaluated in complex arithmetic.  Perturbing an input by
 * i*h (h tiny) gives f(z + i h v) = f(z) + i h f'(z) v + O(h^2) with no
 * subtractive cancellation, so Im(f)/h is the directional derivative to
 * rounding accuracy (Squire & Trapp, SIAM Review 40, 1998).  Every operation
 * used is complex-analytic: magnitudes are sqrt(sum of squares) without
 * conjugation, comparisons (pivoting, max) use real parts.
 *
 * Only the mimetic current is provided; the step-size schedule is fixed
 * (the control law is piecewise constant in the inputs).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "glemur_oracle.h"

typedef double complex cplx;

static long nn(const ora_grid* g) { return (long)g->nx * g->ny * g->nz; }
static long nd(const ora_grid* g, int i, int j, int k) {
  return ((long)k * g->ny + j) * g->nx + i;
}
static int ext(const ora_grid* g, int a) {
  return a == 0 ? g->nx : (a == 1 ? g->ny : g->nz);
}
static void get3c(const ora_grid* g, const cplx* v, int i, int j, int k, cplx o[3]) {
  long N = nn(g), n = nd(g, i, j, k);
  o[0] = v[n];
  o[1] = v[N + n];
  o[2] = v[2 * N + n];
}
static int interior(const ora_grid* g, int i, int j, int k) {
  return i > 0 && j > 0 && k > 0 && i < g->nx - 1 && j < g->ny - 1 && k < g->nz - 1;
}
static void crossc(const cplx a[3], const cplx b[3], cplx o[3]) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static cplx dotc(const cplx a[3], const cplx b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* Jacobian at a node: central inside, second-order one-sided on faces. */
static void jac(const ora_grid* g, const cplx* x, int i, int j, int k, cplx F[9]) {
  int id[3] = {i, j, k};
  for (int b = 0; b < 3; ++b) {
    int n = ext(g, b);
    int p0[3] = {i, j, k}, p1[3] = {i, j, k}, p2[3] = {i, j, k};
    double w0, w1, w2;
    if (id[b] > 0 && id[b] < n - 1) {
      p0[b] -= 1; p1[b] += 1; w0 = -1.0; w1 = 1.0; w2 = 0.0;
    } else if (id[b] == 0) {
      p1[b] = 1; p2[b] = 2; w0 = -3.0; w1 = 4.0; w2 = -1.0;
    } else {
      p1[b] = n - 2; p2[b] = n - 3; w0 = 3.0; w1 = -4.0; w2 = 1.0;
    }
    cplx x0[3], x1[3], x2[3];
    get3c(g, x, p0[0], p0[1], p0[2], x0);
    get3c(g, x, p1[0], p1[1], p1[2], x1);
    get3c(g, x, p2[0], p2[1], p2[2], x2);
    for (int a = 0; a < 3; ++a)
      F[a * 3 + b] = (w0 * x0[a] + w1 * x1[a] + w2 * x2[a]) / (2.0 * g->h[b]);
  }
}

static cplx det3c(const cplx F[9]) {
  return F[0] * (F[4] * F[8] - F[5] * F[7]) - F[1] * (F[3] * F[8] - F[5] * F[6]) +
         F[2] * (F[3] * F[7] - F[4] * F[6]);
}

/* Eq. "B transformation" at every node; Delta optional. */
static void pullback(const ora_grid* g, const cplx* x, const cplx* B0, cplx* B, cplx* D) {
  long N = nn(g);
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        cplx F[9], b0[3];
        jac(g, x, i, j, k, F);
        get3c(g, B0, i, j, k, b0);
        cplx d = det3c(F);
        long n = nd(g, i, j, k);
        for (int a = 0; a < 3; ++a)
          B[a * N + n] = (F[a * 3] * b0[0] + F[a * 3 + 1] * b0[1] + F[a * 3 + 2] * b0[2]) / d;
        if (D) D[n] = d;
      }
}

/* Gaussian elimination with pivoting on the real parts. */
static int solve3c(const cplx Min[9], const cplx r[3], cplx y[3]) {
  cplx M[3][4];
  for (int a = 0; a < 3; ++a) {
    for (int b = 0; b < 3; ++b) M[a][b] = Min[a * 3 + b];
    M[a][3] = r[a];
  }
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int a = col + 1; a < 3; ++a)
      if (fabs(creal(M[a][col])) > fabs(creal(M[piv][col]))) piv = a;
    if (creal(M[piv][col]) == 0.0) return -1;
    for (int c = 0; c < 4; ++c) {
      cplx t = M[col][c];
      M[col][c] = M[piv][c];
      M[piv][c] = t;
    }
    for (int a = col + 1; a < 3; ++a) {
      cplx f = M[a][col] / M[col][col];
      for (int c = col; c < 4; ++c) M[a][c] -= f * M[col][c];
    }
  }
  for (int a = 2; a >= 0; --a) {
    cplx s = M[a][3];
    for (int c = a + 1; c < 3; ++c) s -= M[a][c] * y[c];
    y[a] = s / M[a][a];
  }
  return 0;
}

/* Mimetic current at every interior node (loops through +e_p, +e_q, -e_p,
 * -e_q of the surfaces jk, ki, ij; eq. "sum of triangles" areas). */
static int curl_mimetic(const ora_grid* g, const cplx* x, const cplx* B, cplx* J) {
  long N = nn(g);
  int rc = 0;
  memset(J, 0, sizeof(cplx) * 3 * N);
  for (int k = 1; k < g->nz - 1; ++k)
    for (int j = 1; j < g->ny - 1; ++j)
      for (int i = 1; i < g->nx - 1; ++i) {
        cplx M[9], c[3], Jn[3];
        for (int r = 0; r < 3; ++r) {
          int p = (r + 1) % 3, q = (r + 2) % 3;
          int v[4][3];
          for (int m = 0; m < 4; ++m) {
            v[m][0] = i;
            v[m][1] = j;
            v[m][2] = k;
          }
          v[0][p] += 1;
          v[1][q] += 1;
          v[2][p] -= 1;
          v[3][q] -= 1;
          cplx xv[4][3], Bv[4][3];
          for (int m = 0; m < 4; ++m) {
            get3c(g, x, v[m][0], v[m][1], v[m][2], xv[m]);
            get3c(g, B, v[m][0], v[m][1], v[m][2], Bv[m]);
          }
          cplx circ = 0.0, nA[3] = {0.0, 0.0, 0.0};
          for (int m = 0; m < 4; ++m) {
            cplx dx[3], dx2[3], Bm[3], t[3];
            for (int a = 0; a < 3; ++a) {
              dx[a] = xv[(m + 1) % 4][a] - xv[m][a];
              dx2[a] = xv[(m + 2) % 4][a] - xv[(m + 1) % 4][a];
              Bm[a] = (Bv[m][a] + Bv[(m + 1) % 4][a]) / 2.0;
            }
            circ += dotc(Bm, dx);
            crossc(dx, dx2, t);
            for (int a = 0; a < 3; ++a) nA[a] += t[a] / 4.0;
          }
          c[r] = circ;
          for (int a = 0; a < 3; ++a) M[r * 3 + a] = nA[a];
        }
        if (solve3c(M, c, Jn) != 0) rc = ORA_ERR_COLLAPSED;
        long n = nd(g, i, j, k);
        for (int a = 0; a < 3; ++a) J[a * N + n] = Jn[a];
      }
  return rc;
}

/* u = J x B inside, 0 on the line-tied boundary. */
int orc_velocity(const ora_grid* g, const cplx* x, const cplx* B0, cplx* u) {
  long N = nn(g);
  cplx* B = (cplx*)malloc(sizeof(cplx) * 3 * N);
  cplx* J = (cplx*)malloc(sizeof(cplx) * 3 * N);
  if (!B || !J) {
    free(B);
    free(J);
    return ORA_ERR_BADARG;
  }
  pullback(g, x, B0, B, NULL);
  int rc = curl_mimetic(g, x, B, J);
  for (int k = 0; k < g->nz; ++k)
    for (int j = 0; j < g->ny; ++j)
      for (int i = 0; i < g->nx; ++i) {
        long n = nd(g, i, j, k);
        cplx un[3] = {0.0, 0.0, 0.0};
        if (interior(g, i, j, k)) {
          cplx Jn[3], Bn[3];
          get3c(g, J, i, j, k, Jn);
          get3c(g, B, i, j, k, Bn);
          crossc(Jn, Bn, un);
        }
        for (int a = 0; a < 3; ++a) u[a * N + n] = un[a];
      }
  free(B);
  free(J);
  return rc;
}

/* One Cash-Karp step of size dt (5th-order solution), in place. */
static int ck_step(const ora_grid* g, cplx* x, const cplx* B0, double dt) {
  double c[6], a[36], b5[6], b4[6];
  ora_cash_karp_tableau(c, a, b5, b4);
  long n = 3 * nn(g);
  cplx* k = (cplx*)malloc(sizeof(cplx) * 6 * n);
  cplx* ys = (cplx*)malloc(sizeof(cplx) * n);
  if (!k || !ys) {
    free(k);
    free(ys);
    return ORA_ERR_BADARG;
  }
  int rc = 0;
  for (int s = 0; s < 6; ++s) {
    for (long m = 0; m < n; ++m) {
      cplx acc = 0.0;
      for (int j = 0; j < s; ++j) acc += a[s * 6 + j] * k[(long)j * n + m];
      ys[m] = x[m] + dt * acc;
    }
    int r = orc_velocity(g, ys, B0, &k[(long)s * n]);
    if (r && !rc) rc = r;
  }
  for (long m = 0; m < n; ++m) {
    cplx acc = 0.0;
    for (int j = 0; j < 6; ++j) acc += b5[j] * k[(long)j * n + m];
    x[m] += dt * acc;
  }
  free(k);
  free(ys);
  return rc;
}

/* Steps with the given schedule, then loss 0 = E_M (eq. "magnetic energy"),
 * 1 = xi = max |J x B| / B^2 (by real part).  x is advanced in place. */
int orc_relax_loss(const ora_grid* g, cplx* x, const cplx* B0, const double* dts, int nsteps,
                   int loss, cplx* value) {
  int rc = 0;
  for (int s = 0; s < nsteps && !rc; ++s) rc = ck_step(g, x, B0, dts[s]);
  long N = nn(g);
  cplx* B = (cplx*)malloc(sizeof(cplx) * 3 * N);
  cplx* D = (cplx*)malloc(sizeof(cplx) * N);
  cplx* J = (cplx*)malloc(sizeof(cplx) * 3 * N);
  if (!B || !D || !J) {
    free(B);
    free(D);
    free(J);
    return ORA_ERR_BADARG;
  }
  pullback(g, x, B0, B, D);
  if (loss == 0) {
    cplx sum = 0.0;
    for (int k = 0; k < g->nz; ++k)
      for (int j = 0; j < g->ny; ++j)
        for (int i = 0; i < g->nx; ++i) {
          double zeta = 1.0;
          if (i == 0 || i == g->nx - 1) zeta *= 0.5;
          if (j == 0 || j == g->ny - 1) zeta *= 0.5;
          if (k == 0 || k == g->nz - 1) zeta *= 0.5;
          cplx Bn[3];
          get3c(g, B, i, j, k, Bn);
          sum += zeta * dotc(Bn, Bn) * D[nd(g, i, j, k)];
        }
    *value = 0.5 * sum * g->h[0] * g->h[1] * g->h[2];
  } else {
    int r = curl_mimetic(g, x, B, J);
    if (r && !rc) rc = r;
    cplx best = 0.0;
    for (int k = 1; k < g->nz - 1; ++k)
      for (int j = 1; j < g->ny - 1; ++j)
        for (int i = 1; i < g->nx - 1; ++i) {
          cplx Jn[3], Bn[3], f[3];
          get3c(g, J, i, j, k, Jn);
          get3c(g, B, i, j, k, Bn);
          crossc(Jn, Bn, f);
          cplx v = csqrt(dotc(f, f)) / dotc(Bn, Bn);
          if (creal(v) > creal(best)) best = v;
        }
    *value = best;
  }
  free(B);
  free(D);
  free(J);
  return rc;
}
