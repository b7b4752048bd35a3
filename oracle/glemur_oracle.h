/*
 * FP64 CPU oracle for Lagrangian magneto-frictional relaxation with the
 * mimetic current (Candelaresi, Pontin & Hornig, "Mimetic Methods for
 * Lagrangian Relaxation of Magnetic Fields").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the plain, slow, obviously correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the test-suite, the package's smoke check and the CPU-baseline leg of the
 * benchmark may load it.  It shares no source, header, table or helper with
 * the CUDA library.
 *
 * Conventions.  Grid of nx*ny*nz nodes, node (i,j,k) has linear index
 * n = (k*ny + j)*nx + i; a vector field is stored as three consecutive
 * scalar fields (SoA): component c of node n at v[c*N + n], N = nx*ny*nz.
 * h[a] is the label spacing along axis a (X_ijk = lo + (i h0, j h1, k h2)).
 *
 * Parity notes (unpinned parts): the direct-derivative current of the
 * "classic" method is a reading of the paper (the paper cites but does not
 * print the formula); its pins are closed forms only (exactness on affine
 * maps, second-order convergence on a smooth nonlinear map).
 */
#ifndef GLEMUR_ORACLE_H
#define GLEMUR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int nx, ny, nz;
  double h[3];
  /* 0: line-tied on every face (section "Boundary Conditions").  1: periodic
   * in z: planes k = 0 and k = nz-1 are ghosts of the last and first inner
   * planes shifted by the period L_z + dZ = (nz - 2) h_z along z,
   * x(i,j,0) = x(i,j,nz-2) - (L_z + dZ) e_z and x(i,j,nz-1) = x(i,j,1) +
   * (L_z + dZ) e_z, so that B is periodic; the x and y faces stay
   * line-tied.  B0 must be periodic with the same period. */
  int periodic_z;
} ora_grid;

enum { ORA_CURL_MIMETIC = 0, ORA_CURL_DIRECT = 1, ORA_CURL_NNN = 2 };

enum {
  ORA_OK = 0,
  ORA_ERR_BADARG = -1,
  ORA_ERR_COLLAPSED = -3,   /* det(dx/dX) <= 0 or a singular loop matrix */
  ORA_ERR_NONFINITE = -4,
  ORA_ERR_DT_UNDERFLOW = -5
};

typedef struct {
  double lambda0;     /* tolerance Lambda_0 on the max error in x */
  double dt_min;      /* give up below this step */
  double grow_max;    /* clamp on dt'/dt when growing */
  double shrink_min;  /* clamp on dt'/dt when shrinking */
  int max_rejects;    /* consecutive rejects before giving up */
  double safety;      /* factor s on the adjusted step, s dt (L0/L)^0.2;
                         1 is the law as printed */
} ora_control_opts;

/* --- spatial operator (section "Magnetic Field Relaxation", "Mimetic
 *     Operators") -------------------------------------------------------- */

/* dx/dX at node (i,j,k): F[a*3+b] = d x_a / d X_b.  Second-order central
 * differences inside, second-order one-sided differences on boundary
 * faces. */
void ora_jacobian_at(const ora_grid* g, const double* x, int i, int j, int k,
                     double F[9]);

/* Eq. "B transformation": B = (dx/dX) B0 / det(dx/dX) at every node; also
 * returns Delta = det(dx/dX) when Delta != NULL.  Returns ORA_ERR_COLLAPSED
 * if some Delta <= 0. */
int ora_pullback(const ora_grid* g, const double* x, const double* B0,
                 double* B, double* Delta);

/* Eqs. "current discrete", "sum of triangles", "current matrix equation":
 * nearest-neighbour mimetic current at every interior node (0 elsewhere).
 * If area_gap != NULL it receives the largest relative difference between
 * the four-triangle area of eq. "four surfaces" and eq. "sum of
 * triangles" over all loops. */
int ora_curl_mimetic(const ora_grid* g, const double* x, const double* B,
                     double* J, double* area_gap);

/* The three Stokes loops at one interior node: circulation c[r] and vector
 * area M[r*3+.] (eq. "sum of triangles") for r = 0 (jk surface), 1 (ki),
 * 2 (ij), and J solving M J = c. */
int ora_mimetic_loops_at(const ora_grid* g, const double* x, const double* B,
                         int i, int j, int k, double c[3], double M[9],
                         double J[3]);

/* Classic current: J = curl_x B with dB/dX from the product rule on
 * B = F B0 / Delta (first and second derivatives of x, first derivatives
 * of B0), at every interior node (0 elsewhere). */
int ora_curl_direct(const ora_grid* g, const double* x, const double* B0,
                    double* J);

/* Section "Next Nearest Neighbor Mimetic Approach": the octilateral loops
 * through the eight in-plane neighbours (face and edge-diagonal) of each
 * index surface, eqs. "eight surfaces" / "sum of eight triangles" for
 * their vector areas, M J = c (eq. "current matrix equation") at every
 * interior node (0 elsewhere). */
int ora_curl_nnn(const ora_grid* g, const double* x, const double* B,
                 double* J);

/* u = J x B (gamma = 1) at interior nodes, u = 0 on line-tied boundary
 * nodes (eq. "magneto friction"; section "Boundary Conditions"). */
void ora_lorentz_velocity(const ora_grid* g, const double* J, const double* B,
                          double* u);

/* Full right-hand side dx/dt = u(x) of eq. "x integration". */
int ora_velocity(const ora_grid* g, int curl, const double* x,
                 const double* B0, double* u);

/* Velocity at one interior node, recomputing every quantity it needs from
 * x and B0 (used to spot-check large grids one node at a time). */
int ora_velocity_at(const ora_grid* g, int curl, const double* x,
                    const double* B0, int i, int j, int k, double u[3]);

/* --- time stepping (section "Time Stepping") ---------------------------- */

/* Right-hand side callback for the generic Cash-Karp stepper. */
typedef int (*ora_rhs_fn)(void* ctx, const double* y, double* dydt);

/* The Cash-Karp embedded 5(4) coefficients: c[6], a[6*6] (row s, col j),
 * b5[6], b4[6]. */
void ora_cash_karp_tableau(double c[6], double a[36], double b5[6],
                           double b4[6]);

/* One Cash-Karp attempt of size dt from y (length n): ynew gets the
 * fifth-order solution, yerr the embedded error estimate dt*sum(b5-b4)k.
 * k (6*n doubles) receives the stage derivatives when non-NULL. */
int ora_ck_attempt(long n, const double* y, double dt, ora_rhs_fn f,
                   void* ctx, double* ynew, double* yerr, double* k);

/* Eq. "time stepping": accept iff lambda <= lambda0; the next step is
 * dt*(lambda0/lambda)^0.2 when rejecting or when lambda < lambda0/2, else
 * dt.  Returns ORA_OK or an error code; *accept is 0/1. */
int ora_step_control(const ora_control_opts* o, double lambda, double dt,
                     int consecutive_rejects, double* dt_next, int* accept);

typedef struct {
  int accepted, rejected;
  double dt;       /* step size that will be tried next */
  double t;        /* time of the accepted state */
  double lambda;   /* error of the last attempt */
} ora_stats;

/* Advance x (3N, in place) by n_accept accepted steps from the step size
 * *dt, with the error-controlled Cash-Karp scheme.  The accepted step sizes
 * are written to dt_log (capacity n_accept) when non-NULL. */
int ora_relax(const ora_grid* g, int curl, const ora_control_opts* o,
              double* x, const double* B0, int n_accept, double* dt,
              double* dt_log, ora_stats* st);

/* One attempt of a given size, always taken (replaying a step-size
 * schedule); *lambda receives its error estimate. */
int ora_step_fixed(const ora_grid* g, int curl, double* x, const double* B0,
                   double dt, double* lambda);

/* --- diagnostics (section "Diagnostics") --------------------------------- */

/* Eq. "magnetic energy": E_M = 1/2 sum zeta B^2 Delta dX dY dZ. */
int ora_energy(const ora_grid* g, const double* x, const double* B0,
               double* E);

/* xi = max |J x B| / B^2 over interior nodes, and the sine form
 * max |J x B| / (|J| |B|). */
int ora_forcefree(const ora_grid* g, int curl, const double* x,
                  const double* B0, double* xi, double* xi_sin);

/* --- validation diagnostics (section "Diagnostics") ---------------------- */

/* Section "Deviation from the Exact Known Equilibrium": sigma_x and sigma_B,
 * the root mean square over all N nodes of |x - x_ref| and |B - B_ref|
 * (B the pull-back of B0 on x). */
int ora_deviation(const ora_grid* g, const double* x, const double* B0,
                  const double* x_ref, const double* B_ref, double* sigma_x,
                  double* sigma_B);

/* Section "Force-Freeness": alpha* = J.B/B^2 along the node line (i, j, k),
 * k = 1 .. nz-2 (alpha has nz entries, the boundary ones NaN), and
 * epsilon* = max over pairs of a_r (alpha_k - alpha_l) / |X_k - X_l|. */
int ora_alpha_line(const ora_grid* g, int curl, const double* x,
                   const double* B0, int i, int j, double a_r, double* alpha,
                   double* eps_star);

/* Section "Convexity", eq. "convexity": kappa = +1 at a node when every
 * trihedron of its index neighbours (di, dj, dk = +-1, neighbours inside
 * the grid) has a determinant of sign di dj dk, else -1; *n_concave counts
 * the -1 nodes (kappa may be NULL). */
int ora_convexity(const ora_grid* g, const double* x, int* kappa,
                  long* n_concave);

#ifdef __cplusplus
}
#endif
#endif
