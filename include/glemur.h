/*
 * glemur.h -- C ABI of the GB300 (sm_103a) library for Lagrangian
 * magneto-frictional relaxation with the mimetic current (Candelaresi,
 * Pontin & Hornig, "Mimetic Methods for Lagrangian Relaxation of Magnetic
 * Fields", SIAM J. Sci. Comput.).
 *
 * The state is the position x(X, t) of every node of a logically
 * rectangular grid of labels X_ijk = lo + (i h_x, j h_y, k h_z),
 * h_a = (hi_a - lo_a) / (n_a - 1).  One relaxation step (section "Time
 * Stepping") advances dx/dt = u (eq. "x integration") with the frictional
 * velocity u = J x B (eq. "magneto friction", gamma = 1, mu_0 = 1), where
 * B = (dx/dX) B0 / det(dx/dX) is the pull-back of the initial field
 * (eq. "B transformation") and J = curl B comes from Stokes loops through
 * the nearest neighbours (section "Mimetic Operators", eqs. "current
 * discrete" to "current matrix equation") or, switchably, from direct
 * derivatives (the classic method the paper compares against).  Nodes on
 * the boundary are line-tied: they never move (section "Boundary
 * Conditions").
 *
 * Layout.  Every nodal vector field crossing this ABI is float64, SoA:
 * component c of node (i, j, k) at v[c*N + (k*ny + j)*nx + i],
 * N = nx*ny*nz.
 *
 * Memory.  The library never allocates device memory.  The caller passes a
 * device workspace of at least glemur_workspace_bytes() bytes (for example
 * a torch.uint8 tensor) and keeps it alive until glemur_destroy().  Host
 * pointers passed with GLEMUR_MEM_HOST may be pageable or pinned: pageable
 * buffers go through a device staging buffer, page-locked ones are read
 * (glemur_set_x, glemur_set_B0) or written (glemur_get_x, glemur_velocity)
 * in place by the conversion kernels.  An input buffer is read
 * asynchronously on the stream; the caller keeps it unchanged until the
 * stream has passed the call.  Output calls synchronise the stream.
 *
 * Streams.  All device work runs on the cudaStream_t given to
 * glemur_init_grid (NULL = the legacy default stream).  Calls that return
 * host scalars (glemur_step, glemur_energy, glemur_forcefree_err,
 * glemur_get_stats) synchronise that stream; glemur_attempts does not.
 *
 * Errors.  Every int-returning call returns GLEMUR_OK (0) or a negative
 * GLEMUR_ERR_* code; glemur_strerror() names it.  After an error status
 * from the step (COLLAPSED, NONFINITE, DT_UNDERFLOW, TIMEOUT) the context keeps the
 * last accepted state and refuses further steps until glemur_set_x().
 */
#ifndef GLEMUR_H
#define GLEMUR_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum glemur_precision {
  GLEMUR_FP64 = 0,  /* FP64 storage and arithmetic throughout */
  GLEMUR_MIXED = 1  /* FP32 displacement, B0 and stage fields with FP32
                       stencil arithmetic; determinants, reductions and the
                       step-size control carried at >= 44-bit precision */
};

enum glemur_curl {
  GLEMUR_CURL_MIMETIC = 0, /* nearest-neighbour Stokes loops (default) */
  GLEMUR_CURL_DIRECT = 1,  /* direct derivatives of B = F B0 / det F */
  GLEMUR_CURL_NNN = 2      /* next-nearest-neighbour (octilateral) loops of
                              section "Next Nearest Neighbor Mimetic
                              Approach", eqs. "eight surfaces" and "sum of
                              eight triangles"; GLEMUR_FP64 only, no adjoint.
                              The paper finds it unstable in all but one of
                              its runs. */
};

enum glemur_mem { GLEMUR_MEM_DEVICE = 0, GLEMUR_MEM_HOST = 1 };

enum glemur_status {
  GLEMUR_OK = 0,
  GLEMUR_ERR_BADARG = -1,       /* invalid argument or context state */
  GLEMUR_ERR_CUDA = -2,         /* a CUDA runtime call failed */
  GLEMUR_ERR_COLLAPSED = -3,    /* det(dx/dX) <= 0 somewhere: grid folded */
  GLEMUR_ERR_NONFINITE = -4,    /* NaN/Inf in the error estimate */
  GLEMUR_ERR_DT_UNDERFLOW = -5, /* step shrank below dt_min or too many
                                   consecutive rejections */
  GLEMUR_ERR_WORKSPACE = -6,    /* workspace missing, misaligned or small */
  GLEMUR_ERR_TOO_LARGE = -7,    /* grid larger than a fixed-scratch entry
                                   point supports */
  GLEMUR_ERR_TIMEOUT = -8       /* a bounded device-side wait for a tile
                                   load gave up; the state is not advanced */
};

typedef struct glemur_ctx glemur_ctx;

/* Options; glemur_default_opts() fills the defaults given here.  The paper
 * fixes the control law dt' = dt |Lambda_0/Lambda|^0.2 (eq. "time
 * stepping") but no tolerance, initial step or clamps. */
typedef struct {
  int precision;      /* glemur_precision, default GLEMUR_FP64 */
  int curl;           /* glemur_curl, default GLEMUR_CURL_MIMETIC */
  double lambda0;     /* Lambda_0: tolerance on the max error in x, 1e-7 */
  double dt0;         /* first step size, 1e-3 */
  double dt_min;      /* smallest step before GLEMUR_ERR_DT_UNDERFLOW, 1e-14 */
  double grow_max;    /* clamp on dt'/dt when growing, 5 */
  double shrink_min;  /* clamp on dt'/dt when shrinking, 0.1 */
  int max_rejects;    /* consecutive rejections allowed, 64 */
  int diag_each_attempt; /* 1: every attempt also reduces E_M and xi of the
                            state it starts from (default 1) */
  double safety;      /* factor s on the adjusted step: s dt (Lambda_0/
                         Lambda)^0.2 when rejecting or growing; 1 (default)
                         is the law as printed.  s < 1 (0.9 in Numerical
                         Recipes' stepper) ends rejection streaks when the
                         error falls more slowly than dt^5 */
  int periodic_z;     /* 0 (default): every face line-tied.  1: periodic in
                         z as in section "Boundary Conditions": node planes
                         k = 0 and k = nz-1 are ghosts of the last and first
                         inner planes (f = 1, l = nz-2) shifted by
                         L_z + dZ = (nz - 2) h_z along z, so the period is
                         the nz - 2 inner planes; glemur_set_x takes the
                         ghost positions from their partners, glemur_energy
                         sums one period.  The x and y faces stay
                         line-tied; B0 must be periodic.  GLEMUR_FP64 with
                         the nearest- or next-nearest-neighbour current;
                         no adjoint. */
} glemur_opts;

typedef struct {
  long long accepted;   /* accepted steps since glemur_set_x */
  long long rejected;   /* rejected attempts since glemur_set_x */
  double t;             /* time of the accepted state */
  double dt;            /* step size of the next attempt */
  double lambda;        /* error estimate Lambda of the last attempt */
  double energy;        /* E_M of the state the last attempt started from
                           (when diag_each_attempt is on, else 0; NaN with
                           the direct current -- use glemur_energy) */
  double xi;            /* xi = max |J x B| / B^2 of that state */
  double xi_sin;        /* max |J x B| / (|J| |B|) of that state */
  int status;           /* GLEMUR_OK or the error that stopped stepping */
  double dt_last;       /* size of the last accepted step (replay schedules) */
} glemur_stats;

/* Fill *o with the defaults listed in glemur_opts. */
void glemur_default_opts(glemur_opts* o);

/* Device workspace needed for an nx*ny*nz grid at the given precision
 * (bytes, a multiple of 256).  Returns 0 for invalid sizes. */
size_t glemur_workspace_bytes(int nx, int ny, int nz, int precision);

/* Create a context for an nx*ny*nz node grid (each >= 3) with labels on the
 * box [lo, hi] (hi_a > lo_a).  `opts` may be NULL for the defaults.
 * `stream` is a cudaStream_t (or NULL).  `workspace` is caller-owned
 * device memory of ws_bytes >= glemur_workspace_bytes(), 256-byte aligned.
 * The positions start at x = X and B0 = 0; call glemur_set_x/glemur_set_B0.
 * On success *out receives the context.  Errors: BADARG, WORKSPACE, CUDA.
 *
 * Kernel selection happens here, once per context; these environment
 * variables, read at this call, override it (all results stay within the
 * same tolerances):
 *   GLEMUR_TMA=0          mixed precision: register-staged tile loads even
 *                         where TMA tiles apply (nx a multiple of 4, nx >= 40,
 *                         ny >= 12)
 *   GLEMUR_F64_FUSED=1    FP64: single-kernel mimetic stages (halo
 *                         recomputation) instead of the two-pass stages
 *   GLEMUR_KZ=k           z-planes per CTA of the stage kernels instead of
 *                         the cost model's choice
 *   GLEMUR_PERSIST=1      FP64 two-pass stages, line-tied, loop currents:
 *                         whole attempts (twelve passes and the control) in
 *                         one persistent cooperative launch with per-plane
 *                         waits instead of one launch per pass (same
 *                         results bit for bit; measured about 5 % slower)
 *   GLEMUR_TEST_PERSIST_TIMEOUT=1  test hook: in the persistent launch one
 *                         CTA never reports a finished pass, so the bounded
 *                         waits of its neighbours give up after 2 s and
 *                         steps fail with GLEMUR_ERR_TIMEOUT
 *   GLEMUR_TEST_TMA_TIMEOUT=1 or 2  test hook: the TMA stage kernels' first
 *                         tile wait (1) or first wait inside their plane loop
 *                         (2, CTAs of at least two z-planes) also waits on a
 *                         barrier that no copy completes, so the bounded wait
 *                         gives up and steps fail with GLEMUR_ERR_TIMEOUT
 * and, read at each call with a host buffer:
 *   GLEMUR_HOST_STAGING=1 copy page-locked host buffers through the staging
 *                         buffer instead of reading and writing them in
 *                         place from the conversion kernels
 * and, read once per process, for every launch of the library:
 *   GLEMUR_PDL=0          ordinary kernel launches instead of programmatic
 *                         dependent launches (each kernel of an attempt or
 *                         reverse step may otherwise be scheduled while the
 *                         previous one drains; it waits for that kernel's
 *                         completion before it touches memory) */
int glemur_init_grid(glemur_ctx** out, int nx, int ny, int nz,
                     const double lo[3], const double hi[3],
                     const glemur_opts* opts, void* stream, void* workspace,
                     size_t ws_bytes);

/* Set the node positions x(X) (float64 field, layout above; `mem` says
 * where it lives).  Boundary nodes keep these positions for ever.  Resets
 * the step counters, the time and the error status, and sets dt = dt0.
 * Section "Initial Configuration" (the initial grid), eq. "x integration"
 * (x(X,0) = X unless pre-distorted). */
int glemur_set_x(glemur_ctx* ctx, const double* x, int mem);

/* Set the initial field B(X, 0) on the nodes (float64 field).  Eq. "B
 * transformation" uses it at every step; it is not modified. */
int glemur_set_B0(glemur_ctx* ctx, const double* B0, int mem);

/* Copy the current accepted positions x into `x` (float64 field). */
int glemur_get_x(glemur_ctx* ctx, double* x, int mem);

/* Bytes of the raw relaxation state (the displacement x - X of every node
 * in the context's storage precision: 3N doubles, or 3N floats in mixed
 * precision); 0 for NULL. */
size_t glemur_state_bytes(const glemur_ctx* ctx);

/* Copy the raw state into dev_buf (device memory of glemur_state_bytes()):
 * an exact checkpoint, unlike glemur_get_x whose float64 x = X + d rounds. */
int glemur_get_state(glemur_ctx* ctx, void* dev_buf);

/* Restore a raw state taken by glemur_get_state from a context of the same
 * grid and precision.  Like glemur_set_x it resets the counters, the time,
 * the error status and dt = dt0. */
int glemur_set_state(glemur_ctx* ctx, const void* dev_buf);

/* Frictional velocity u = J x B of the current state at every node (0 on
 * the boundary) into `u` (float64 field): the right-hand side of eq. "x
 * integration" (eq. "magneto friction"). */
int glemur_velocity(glemur_ctx* ctx, double* u, int mem);

/* Advance by n_accept accepted steps (n_accept >= 0) of the Cash-Karp
 * 5(4) scheme with the error-controlled step of section "Time Stepping":
 * Lambda = max over nodes and components of the embedded error in x;
 * accept iff Lambda <= Lambda_0; dt' = dt (Lambda_0/Lambda)^0.2 when
 * rejecting (redo) or when Lambda < Lambda_0/2 (grow), clamped by
 * shrink_min/grow_max.  An attempt whose trial stage input folds the grid
 * (det dx/dX <= 0) is rejected with the largest shrink; a folded accepted
 * state stops with COLLAPSED.  Synchronises; fills *stats when non-NULL.
 * Errors: BADARG, CUDA, COLLAPSED, NONFINITE, DT_UNDERFLOW. */
int glemur_step(glemur_ctx* ctx, int n_accept, glemur_stats* stats);

/* Enqueue exactly n_attempts Cash-Karp attempts with the same control law
 * (each either accepted or rejected) without synchronising.  Throughput
 * harnesses time this; read the outcome with glemur_get_stats. */
int glemur_attempts(glemur_ctx* ctx, int n_attempts);

/* One attempt of the given size that is always accepted (replays a
 * recorded step-size schedule; section "Time Stepping" without the
 * control).  The next automatic step starts from dt.  Synchronises. */
int glemur_step_fixed(glemur_ctx* ctx, double dt, glemur_stats* stats);

/* Magnetic energy E_M = 1/2 sum zeta B^2 Delta dX dY dZ of the current
 * state (eq. "magnetic energy"; zeta = 1, 1/2, 1/4, 1/8 inside, on faces,
 * edges, corners).  FP64 accumulation.  Synchronises. */
int glemur_energy(glemur_ctx* ctx, double* E);

/* Force-free errors of the current state over interior nodes:
 * *xi = max |J x B| / B^2 (section "Evolution of Diagnostic Parameters")
 * and *xi_sin = max |J x B| / (|J| |B|) (nodes with |J||B| = 0 skipped),
 * with the context's current.  Synchronises. */
int glemur_forcefree_err(glemur_ctx* ctx, double* xi, double* xi_sin);

/* Accepted step sizes kept on the device: the last GLEMUR_DT_LOG accepted
 * steps since glemur_set_x / glemur_set_state (a ring in the workspace,
 * written by the device-side step control, so recording a schedule costs no
 * host synchronisation per step). */
#define GLEMUR_DT_LOG 65536

/* Copy the sizes of accepted steps first .. first+count-1 (numbered from 0
 * since glemur_set_x or glemur_set_state) into host memory dts[count], in
 * order: the step-size schedule of section "Time Stepping"'s control, for
 * replaying a run with glemur_step_fixed (parity checks, the adjoint).
 * BADARG if some of those steps have not been accepted yet or have left the
 * ring (first < accepted - GLEMUR_DT_LOG).  Synchronises. */
int glemur_get_dt_schedule(glemur_ctx* ctx, long long first, int count, double* dts);

/* ---- validation diagnostics (section "Diagnostics") --------------------
 * On the current accepted state, FP64 arithmetic in either precision,
 * deterministic sums; each synchronises the stream. */

/* Section "Deviation from the Exact Known Equilibrium": *sigma_x and
 * *sigma_B, the root mean square over all N nodes of |x - x_ref| and of
 * |B - B_ref| (B the pull-back of eq. "B transformation").  x_ref and B_ref
 * are device float64 fields (layout above), e.g. the IsoHelix field's
 * closed-form relaxed state (eqs. "x analytical relaxed", "B relaxed").
 * Errors: BADARG, CUDA. */
int glemur_deviation(glemur_ctx* ctx, const double* x_ref, const double* B_ref,
                     double* sigma_x, double* sigma_B);

/* Section "Force-Freeness": alpha* = J.B / B^2 at the nodes (i, j, k) of the
 * node line through (i, j) (1 <= i <= nx-2, 1 <= j <= ny-2), with the
 * context's current, into host alpha[nz] when non-NULL (the two boundary
 * entries, where the current is not defined, are NaN), and eq. "epsilon
 * star": *eps_star = max over pairs of its interior nodes of
 * a_r (alpha*_k - alpha*_l) / |X_k - X_l| (a_r > 0; |X_k - X_l| =
 * |k - l| h_z).  nz <= 6144.  Errors: BADARG, CUDA. */
int glemur_alpha_line(glemur_ctx* ctx, int i, int j, double a_r, double* alpha,
                      double* eps_star);

/* Section "Convexity", eq. "convexity": kappa = +1 at a node when each
 * trihedron of its index neighbours x(i+di,j,k) - x, x(i,j+dj,k) - x,
 * x(i,j,k+dk) - x (di, dj, dk = +-1, the neighbours inside the grid) has a
 * determinant of sign di dj dk, else -1.  *n_concave receives the number of
 * nodes with kappa = -1; kappa (device, N int8 values) may be NULL.
 * Errors: BADARG, CUDA. */
int glemur_convexity(glemur_ctx* ctx, long long* n_concave, signed char* kappa);

/* Counters and last-attempt values (see glemur_stats).  Synchronises. */
int glemur_get_stats(glemur_ctx* ctx, glemur_stats* stats);

/* Number of CUDA kernels one attempt launches (for launch accounting): the
 * stage kernels (two per stage for the FP64 two-pass stages) and the
 * step-control kernel; 1 with the persistent launch (GLEMUR_PERSIST=1, one
 * launch for any number of attempts). */
int glemur_kernels_per_attempt(const glemur_ctx* ctx);

/* Enqueue one attempt as glemur_attempts(ctx, 1) does (a target-reset
 * kernel, then the attempt's kernels, stage by stage -- also where
 * glemur_attempts would use the persistent launch), with a CUDA event
 * recorded on the context's stream before each Cash-Karp stage, before the
 * step control and after it; synchronise and write the 7 intervals in
 * milliseconds to ms[0..6]: stages 1..6 (each interval covers all kernels
 * of its stage: two for the FP64 two-pass stages), then the control.
 * Returns 7, or a negative error (BADARG if cap < 7). */
int glemur_profile_attempt(glemur_ctx* ctx, float* ms, int cap);

/* ---- adjoint (reverse mode) of the relaxation, mimetic current ---------
 * The step of section "Time Stepping" at a fixed step size is a smooth map
 * x_{n+1} = Phi(x_n; B0); these calls give its vector-Jacobian products so
 * that gradients of a loss of the final state with respect to B0 (and hence
 * to any parameters of B0) follow by running the steps backwards with
 * recomputation.  The paper relaxes fields and does not differentiate the
 * relaxation; these entry points are this library's addition.  All fields
 * are float64 device arrays (layout above); the adjoint workspace is
 * caller-owned device memory (256-byte aligned) of
 * glemur_adjoint_workspace_bytes().  They synchronise the stream and leave
 * the context's pending step size set to the dt they used. */

enum glemur_loss { GLEMUR_LOSS_ENERGY = 0, GLEMUR_LOSS_XI = 1 };

/* Adjoint workspace bytes for an nx*ny*nz grid (0 for invalid sizes). */
size_t glemur_adjoint_workspace_bytes(int nx, int ny, int nz, int precision);

/* With the context at state x_n: lam = (d x_{n+1} / d x_n)^T lam_next and
 * mu_B0 += (d x_{n+1} / d B0)^T lam_next for one Cash-Karp step of size dt
 * (the stages are recomputed from x_n).  Boundary entries of lam are zero
 * (line-tied nodes are not variables).  lam and lam_next may not alias.
 * Errors: BADARG (also for the direct current), WORKSPACE, CUDA. */
int glemur_vjp_step(glemur_ctx* ctx, double dt, const double* lam_next, double* lam,
                    double* mu_B0, void* adj_ws, size_t adj_bytes);

/* Loss of the current state -- GLEMUR_LOSS_ENERGY: E_M (eq. "magnetic
 * energy"); GLEMUR_LOSS_XI: xi = max |J x B| / B^2, differentiated at its
 * argmax node -- into *value (host), its gradient with respect to the
 * positions into lam (overwritten) and with respect to B0 added to mu_B0. */
int glemur_loss_grad(glemur_ctx* ctx, int loss, double* value, double* lam, double* mu_B0,
                     void* adj_ws, size_t adj_bytes);

/* Device bytes of the segment workspace glemur_adjoint_segment needs for
 * n_steps steps with a checkpoint every `every` steps: ceil(n_steps/every)
 * state checkpoints, the states of one segment (min(n_steps, every)) and
 * one adjoint field, each rounded up to 256 bytes (0 for invalid
 * arguments). */
size_t glemur_adjoint_segment_bytes(glemur_ctx* ctx, int n_steps, int every);

/* The reverse pass over a recorded segment, natively: the loss (as in
 * glemur_loss_grad) of the state reached from the positions x0 by n_steps
 * fixed steps of the sizes dts[0..n_steps-1] (host array; the schedule a
 * controlled run recorded, glemur_get_dt_schedule), into *value, and its
 * gradients: with respect to x0 into lam_x0 and with respect to B0 into
 * mu_B0 (device float64 fields, overwritten).  Forward: glemur_set_x(x0),
 * then the steps, keeping the raw state every `every` steps in seg_ws;
 * backward: each segment recomputed forwards from its checkpoint with its
 * states kept, the loss gradient seeded at the final state, and the steps'
 * glemur_vjp_step in reverse -- checkpointing with recompute, memory
 * O(n_steps/every + every) states.  x0 must not alias the workspaces (it
 * may be lam_x0 or mu_B0: it is read before they are written);
 * seg_ws (256-byte aligned, glemur_adjoint_segment_bytes) and adj_ws (as
 * for glemur_vjp_step) are caller-owned.  Leaves the context at state x0
 * and synchronises its stream.  Errors: BADARG, WORKSPACE, CUDA and those
 * of the steps (e.g. COLLAPSED). */
int glemur_adjoint_segment(glemur_ctx* ctx, const double* x0, const double* dts, int n_steps,
                           int every, int loss, double* value, double* lam_x0, double* mu_B0,
                           void* adj_ws, size_t adj_bytes, void* seg_ws, size_t seg_bytes);

/* out[p] = sum_m dB0[p*m_len + m] * mu[m] for p < n_params (device arrays):
 * the gradient with respect to parameters theta of B0(theta) from the
 * field adjoint mu_B0 and dB0/dtheta.  Asynchronous on `stream`. */
int glemur_param_contract(int n_params, long long m_len, const double* dB0, const double* mu,
                          double* out, void* stream);

/* Largest grid (nodes) glemur_energy_static accepts: 256^3. */
#define GLEMUR_STATIC_MAX_NODES (1LL << 24)

/* Magnetic energy E_M of positions x with initial field B0, allocating
 * nothing: for callers that cannot allocate device memory (a host framework
 * that owns the whole device pool and forbids foreign allocations, or code
 * that must not trigger the implicit device synchronisation of
 * cudaMalloc/cudaFree).  The paper has no counterpart; this is the energy
 * reduction of glemur_energy without a context or workspace.
 * x and B0 are device float64 fields (layout above) of an nx*ny*nz grid
 * with labels on [lo, hi]; *E (device memory, one double) receives E_M,
 * computed as glemur_energy does (FP64, fixed-order sums).  The per-CTA
 * partial sums live in a static device array of GLEMUR_STATIC_MAX_NODES/256
 * doubles (512 KiB) that every GPU loading this library holds until the
 * process exits; grids of more than GLEMUR_STATIC_MAX_NODES nodes return
 * GLEMUR_ERR_TOO_LARGE.  The first call on each device resolves that
 * array's device address (cudaGetSymbolAddress, with the device current);
 * the address belongs to the CUDA context that is current then, and a later
 * call from another context (after cudaDeviceReset, or from a framework's
 * own non-primary context) resolves it again.  Make the first call from
 * each context before any stream capture.  All calls share the array:
 * calls that overlap on the GPU (different streams or threads) race.  Asynchronous on `stream` (a
 * cudaStream_t or NULL).  Errors: BADARG, TOO_LARGE, CUDA. */
int glemur_energy_static(int nx, int ny, int nz, const double lo[3],
                         const double hi[3], const double* x, const double* B0,
                         double* E, void* stream);

/* Release the context (host memory only; the workspace stays the
 * caller's). NULL is ignored. */
void glemur_destroy(glemur_ctx* ctx);

/* Static description of a status code. */
const char* glemur_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* GLEMUR_H */
