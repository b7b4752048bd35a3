// Device-side definitions shared by the GB300 kernels of the relaxation step.
//
// Storage.  The library keeps the displacement d = x - X (X the label grid)
// rather than x: every stencil only needs differences of x, and
// x(m + e_a) - x(m - e_a) = d(m + e_a) - d(m - e_a) + 2 h_a e_a, so X never
// has to be formed and FP32 storage (mixed mode) keeps its precision in the
// part that moves.  B0 is stored pre-scaled, B0s_a = B0_a * 4 h_{a+1} h_{a+2},
// so that with the index-space differences g_a = 2 h_a dx/dX_a the pull-back
// of eq. "B transformation" is B = (g_0 B0s_0 + g_1 B0s_1 + g_2 B0s_2)/det G
// (the h factors cancel), and E_M = sum zeta |B|^2 det G / 16.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace glemur {

// CTA tile: TX x TY output columns, marching in z.
constexpr int TX = 32;
constexpr int TY = 8;
constexpr int NT = TX * TY;
// Displacement tile with a halo of 2 (the mimetic current needs B at the
// six neighbours, and B at a node needs x at its own neighbours).
constexpr int XW = TX + 4, XH = TY + 4, XP = XW * XH;
// B tile with a halo of 1.
constexpr int BW = TX + 2, BH = TY + 2, BP = BW * BH;
// Displacement tile with a halo of 1 (direct current).
constexpr int DW = TX + 2, DH = TY + 2, DP = DW * DH;
// TMA boxes of the mixed-precision mimetic stages (FP32 SoA fields, all
// three components per box).  A box must start on a 16-byte boundary, so it
// starts 4 columns left of the tile (2 of them unused) and is YW wide.
constexpr int YW = TX + 8;            // box width (floats)
constexpr int YH = TY + 4;            // stage-input box height (halo 2)
constexpr int YCS = YW * YH;          // floats per component
constexpr int YPL = 3 * YCS;          // floats per stage-input plane
constexpr int ZH = TY + 2;            // B0 box height (halo 1)
constexpr int ZCS = YW * ZH;          // floats per component
constexpr int ZPL = 3 * ZCS;          // floats per B0 plane
constexpr int ZSTRIDE = (ZPL * 4 + 127) / 128 * 32;  // B0 slot stride (floats), 128-byte aligned
constexpr unsigned YBYTES = YPL * 4, ZBYTES = ZPL * 4;

// Error flags raised by the stage kernels: det G <= 0 in the accepted state
// (stage 1 input: fatal) or in a trial stage input (the attempt is
// rejected with the largest shrink).
constexpr unsigned FLAG_COLLAPSED = 1u;
constexpr unsigned FLAG_FOLDED_TRIAL = 2u;
// A bounded wait for a tile load gave up (the attempt's results are void).
constexpr unsigned FLAG_TIMEOUT = 4u;

// Device status codes (same values as glemur_status).
constexpr int ST_OK = 0;
constexpr int ST_COLLAPSED = -3;
constexpr int ST_NONFINITE = -4;
constexpr int ST_DT_UNDERFLOW = -5;
constexpr int ST_TIMEOUT = -8;

// Control state of the time integration, resident in the workspace.  The
// step-control kernel updates it after every attempt, so the host never has
// to synchronise between attempts.
struct DevState {
  double dt;          // step size of the next attempt
  double dt_last;     // step size of the last accepted attempt
  double t;           // time of the accepted state
  double lambda;      // error estimate of the last attempt
  double lambda0, dt_min, grow_max, shrink_min, safety;
  long long n_accept, n_reject;
  long long target;   // attempts stop (no-op) once n_accept reaches this
  int consec;         // consecutive rejections
  int cur;            // which displacement buffer holds the accepted state
  int status;         // ST_OK or an error status
  unsigned flags;     // FLAG_* raised by stage kernels in this attempt
  int max_rejects;
  int replay;         // 1: accept the next attempt whatever its error
  // dt-scaled Cash-Karp coefficients of the pending attempt
  double dta[6][6];
  double dtb[6];
  double dte[6];
  float dtaf[6][6];
  float dtbf[6];
  float dtef[6];
  // diagnostics reduced from the state the last diagnostic launch saw
  double E, xi, xi_sin;
};

// Partial-result slots per CTA (see StageArgs::part).
enum { PART_LAMBDA = 0, PART_E = 1, PART_XI2 = 2, PART_XIS2 = 3, NPART = 4 };

template <typename T>
struct StageArgs {
  int nx, ny, nz;
  int kz;              // planes per CTA along z
  double h2[3];        // 2 h_a
  float h2f[3];        // 2 h_a rounded to float (mixed precision)
  const T* d[2];       // ping-pong displacement buffers (3N each)
  const T* B0s;        // pre-scaled B0 (3N)
  T* k[5];             // stage derivatives k1..k5 (3N each)
  T* k6;               // if set, the last stage also stores k6 here
  T* ys[2];            // stage inputs: y_s in ys[s & 1] (s >= 1), 3N each;
                       // boundary entries hold the fixed boundary positions
  int stage;           // 0..5 (stage s+1 of Cash-Karp)
  int diag;            // reduce E_M / xi partials in this launch
  int force;           // run even if the step target is reached
  DevState* st;
  double* part;        // [NPART][nblocks] per-CTA partials
  int nblocks;
  // test hook of the bounded tile waits: 0 (off); 1 or 2 make the TMA
  // stage kernels also wait, at the prologue (1) or at the first wait
  // inside the plane loop (2), on a barrier that no copy completes, so that
  // wait gives up and the attempt fails without any fault
  int tma_test;
};

// Programmatic dependent launch.  The kernels of an attempt are launched
// with launch_pdl: the next kernel of the stream may then be scheduled onto
// SMs that the current one has left while its last CTAs still run.  Each
// such kernel calls pdl_trigger() (its own successor may be scheduled once
// all of its CTAs have started) and pdl_wait() before it reads or writes
// anything an earlier kernel of the stream touches, DevState included:
// griddepcontrol.wait returns once the preceding grids have completed and
// their memory operations are visible.  Every path through such a kernel
// passes pdl_wait(), so completion stays transitive along the stream.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Host side: launch `k` on stream s, programmatic serialisation allowed
// unless the environment sets GLEMUR_PDL=0 (then an ordinary launch).  A
// grid launched this way is placed on SMs as slots free up, not spread
// evenly at launch: the one-wave FP64 passes therefore size their grid to
// exactly the CTAs per SM that each of them can hold.
bool pdl_enabled();
template <typename... Exp, typename... Act>
cudaError_t launch_pdl(void (*k)(Exp...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                       Act&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k, static_cast<Act&&>(args)...);
}

// Arguments of the FP64 two-pass stages (pass B: B and 1/det G at every
// node; pass C: current, k_s and the next stage input).
struct SplitArgs {
  int nx, ny, nz;
  double h2[3];        // 2 h_a
  const double* d[2];  // ping-pong displacements
  const double* B0s;   // pre-scaled B0 (3N)
  double* k[6];        // k1..k5 (k[5] = optional k6)
  double* ys[2];       // stage inputs: y_s in ys[s & 1] (s >= 1), 3N each;
                       // boundary entries hold the fixed boundary positions
  double* Bb;          // B, 3N
  double* rb;          // 1/det G, N, or null (then written to Gb only)
  double* Gb;          // per interior node n, 10 doubles at Gb + 10 n
                       // (16-byte aligned): g_0, g_1, g_2 (index-space
                       // differences, 3 components each) and 1/det G --
                       // written by pass B, read by pass C
  int diag, force;
  int periodic;        // periodic in z: planes 0, nz-1 are ghosts of nz-2, 1
  DevState* st;
  double* part;        // [NPART][nblocks] per-CTA partials
  int nblocks;         // partial stride: the largest of the grids
  int grid_b[6];       // CTAs of pass B of each stage
  int grid_c[6];       // CTAs of pass C of each stage
};

// The persistent FP64 attempt kernel's plan and synchronisation state
// (workspace memory): per node plane, completion counters of pass B and
// pass C and how many CTAs contribute to each; per CTA, the plane
// intervals its pass-B work touches (at most 6: interior planes and the
// boundary face blocks) and its pass-C interval (interior planes); an
// arrival counter and a release generation for the end of each attempt.
constexpr int PERSIST_BI = 6;  // pass-B intervals per CTA
struct PersistArgs {
  int* cntB;            // [nz]
  int* cntC;            // [nz]
  const int* touchB;    // [nz] contributions per plane and pass-B phase
  const int* touchC;    // [nz]
  const int* ivB;       // [G][PERSIST_BI][2] (lo, hi) inclusive, lo > hi: empty
  const int* ivC;       // [G][2]
  unsigned* bar;        // [2] arrivals, released generation
  double* dtlog;        // accepted step-size ring
  int n_attempts;       // attempts this launch
  int test_withhold;    // test hook: this CTA never publishes pass B of
                        // stage 3, so waits on it give up (-1: off)
};

// What the on-demand diagnostics (diagnostics.cu) need of a context.
struct DiagCtx {
  int nx, ny, nz;
  double lo[3], h[3];
  int precision, curl, periodic;
  const void* const* dbuf_dev;  // device copy of the two displacement buffers
  const void* B0s;              // pre-scaled B0 in storage precision
  const DevState* st;           // .cur selects the accepted displacement
  double* part;                 // NPART * max_blocks doubles of scratch
  int max_blocks;
  double* stage;                // 3N doubles of scratch
  cudaStream_t s;
};

__device__ __forceinline__ long long nidx(int i, int j, int k, int nx, int ny) {
  return ((long long)k * ny + j) * nx + i;
}

// max of two non-negative doubles that propagates NaN (of either sign),
// on the integer pipes: the bit patterns of non-negative doubles order like
// unsigned integers and every NaN pattern lies above +inf.  (All maxima of
// the step -- error norms, xi^2 -- are of non-negative values; -0 must not
// occur.)  GB300's FP64 pipe is 1/64 of its FP32 rate, so FP64 compares in
// reductions and per-node maxima are worth avoiding.
__device__ __forceinline__ double nanmax(double a, double b) {
  const unsigned long long ua = (unsigned long long)__double_as_longlong(a);
  const unsigned long long ub = (unsigned long long)__double_as_longlong(b);
  return __longlong_as_double((long long)(ua > ub ? ua : ub));
}

// a > b for non-negative doubles (a NaN a counts as larger), on the integer
// pipes (see nanmax); the float overload is the plain compare.
__device__ __forceinline__ bool gt_nonneg(double a, double b) {
  return (unsigned long long)__double_as_longlong(a) > (unsigned long long)__double_as_longlong(b);
}
__device__ __forceinline__ bool gt_nonneg(float a, float b) { return a > b || a != a; }
// not a NaN (integer test for doubles)
__device__ __forceinline__ bool not_nan(double a) {
  return ((unsigned long long)__double_as_longlong(a) & 0x7fffffffffffffffull) <=
         0x7ff0000000000000ull;
}
__device__ __forceinline__ bool not_nan(float a) { return a == a; }
// a <= 0 (false for NaN), integer test for doubles
__device__ __forceinline__ bool le_zero(double a) {
  return __double_as_longlong(a) <= 0 && not_nan(a);  // sign bit set, or +0
}
__device__ __forceinline__ bool le_zero(float a) { return a <= 0.0f; }

}  // namespace glemur
