// Step-size control of the relaxation (section "Time Stepping"): the
// Cash-Karp table, the control law of eq. "time stepping" with the
// acceptance rule around it, and the fixed-order reductions of the per-CTA
// partials (error norm, E_M, xi).  Run by one CTA after each attempt --
// as the control kernel, or inside the persistent attempt kernel by the
// CTA that finishes an attempt last.  Loads go through a policy: plain
// loads in the control kernel (a launch of its own), L2 loads where other
// CTAs of the same launch wrote the data.
#pragma once

#include <cuda_runtime.h>

#include "glemur.h"
#include "glemur_dev.cuh"

namespace glemur {

struct LdPlain {
  __device__ static __forceinline__ double ld(const double* p) { return *p; }
  __device__ static __forceinline__ int ldi(const int* p) { return *p; }
  __device__ static __forceinline__ unsigned ldu(const unsigned* p) { return *p; }
  __device__ static __forceinline__ long long ldll(const long long* p) { return *p; }
};
struct LdCoherent {
  __device__ static __forceinline__ double ld(const double* p) { return __ldcg(p); }
  __device__ static __forceinline__ int ldi(const int* p) { return __ldcg(p); }
  __device__ static __forceinline__ unsigned ldu(const unsigned* p) { return __ldcg(p); }
  __device__ static __forceinline__ long long ldll(const long long* p) { return __ldcg(p); }
};

// Cash-Karp embedded 5(4) pair (Cash & Karp, ACM TOMS 16, 1990), the scheme
// of section "Time Stepping".
static __constant__ double CK_A[6][6] = {
    {0, 0, 0, 0, 0, 0},
    {1.0 / 5.0, 0, 0, 0, 0, 0},
    {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0},
    {3.0 / 10.0, -9.0 / 10.0, 6.0 / 5.0, 0, 0, 0},
    {-11.0 / 54.0, 5.0 / 2.0, -70.0 / 27.0, 35.0 / 27.0, 0, 0},
    {1631.0 / 55296.0, 175.0 / 512.0, 575.0 / 13824.0, 44275.0 / 110592.0,
     253.0 / 4096.0, 0}};
static __constant__ double CK_B5[6] = {37.0 / 378.0, 0.0, 250.0 / 621.0, 125.0 / 594.0, 0.0,
                                512.0 / 1771.0};
static __constant__ double CK_B4[6] = {2825.0 / 27648.0, 0.0, 18575.0 / 48384.0,
                                13525.0 / 55296.0, 277.0 / 14336.0, 1.0 / 4.0};

// Sum and max reductions of the per-CTA diagnostic partials (fixed order).
template <class LD>
__device__ void finalize_diag(DevState* st, const double* part, int nb, double* sh) {
  double e = 0.0, x2 = 0.0, xs2 = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    e += LD::ld(&part[PART_E * nb + b]);
    x2 = nanmax(x2, LD::ld(&part[PART_XI2 * nb + b]));
    xs2 = nanmax(xs2, LD::ld(&part[PART_XIS2 * nb + b]));
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    e += __shfl_xor_sync(0xffffffffu, e, o);
    x2 = nanmax(x2, __shfl_xor_sync(0xffffffffu, x2, o));
    xs2 = nanmax(xs2, __shfl_xor_sync(0xffffffffu, xs2, o));
  }
  __syncthreads();
  if (lane == 0) {
    sh[w] = e;
    sh[32 + w] = x2;
    sh[64 + w] = xs2;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double E = 0.0, X = 0.0, XS = 0.0;
    for (int i = 0; i < nw; ++i) {
      E += sh[i];
      X = nanmax(X, sh[32 + i]);
      XS = nanmax(XS, sh[64 + i]);
    }
    st->E = E / 16.0;  // eq. "magnetic energy" in index-space units
    st->xi = sqrt(X);
    st->xi_sin = sqrt(XS);
  }
}

// r^0.2 for the step-size law of eq. "time stepping": one Newton step on
// y^5 = r (Newton's method for the n-th root, y <- ((n-1) y + r / y^(n-1))
// / n, which converges quadratically) from an FP32 estimate: ~1e-7 -> ~1e-14
// relative, with a handful of FP64 operations instead of a double pow on
// GB300's narrow FP64 pipe.  Outside the estimate's float range, pow.
__device__ __forceinline__ double fifth_root(double r) {
  if (!(r > 1e-30 && r < 1e30)) return pow(r, 0.2);
  const double y = (double)powf((float)r, 0.2f);
  const double y2 = y * y;
  return 0.2 * (4.0 * y + r / (y2 * y2));
}

// dt-scaled coefficients for step size dt, one entry per thread (the 36
// a_sj and the 6 b_j, b_j - b*_j; threads >= 42 idle).
__device__ __forceinline__ void set_coeffs_parallel(DevState* st, double dt) {
  const int t = threadIdx.x;
  if (t < 36) {
    const int s = t / 6, j = t % 6;
    const double v = dt * CK_A[s][j];
    st->dta[s][j] = v;
    st->dtaf[s][j] = (float)v;
  } else if (t < 42) {
    const int s = t - 36;
    const double b = dt * CK_B5[s], e = dt * (CK_B5[s] - CK_B4[s]);
    st->dtb[s] = b;
    st->dte[s] = e;
    st->dtbf[s] = (float)b;
    st->dtef[s] = (float)e;
  }
}

// Eq. "time stepping" and the acceptance rule around it, after an attempt
// (one whole CTA; returns at once when stepping has stopped).  Thread 0
// takes the decision from a snapshot of the control state (all loads
// independent, then all stores); the block then writes the dt-scaled
// coefficients of the next attempt in parallel.  `sh` holds 96 doubles.
template <class LD>
__device__ void control_block(DevState* st, const double* part, int nb, int diag,
                              double* dtlog, double* sh) {
  __shared__ double dt_next;
  __shared__ int go_on;
  if (LD::ldi(&st->status) != ST_OK ||
      LD::ldll(&st->n_accept) >= LD::ldll(&st->target))
    return;
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x)
    m = nanmax(m, LD::ld(&part[PART_LAMBDA * nb + b]));
  for (int o = 16; o > 0; o >>= 1) m = nanmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) m = nanmax(m, sh[i]);
    sh[95] = m;
  }
  __syncthreads();
  if (diag) finalize_diag<LD>(st, part, nb, sh);
  if (threadIdx.x == 0) {
    const double lam = sh[95];
    const double dt = LD::ld(&st->dt), lambda0 = LD::ld(&st->lambda0),
                 safety = LD::ld(&st->safety);
    const double shrink_min = LD::ld(&st->shrink_min), grow_max = LD::ld(&st->grow_max),
                 dt_min = LD::ld(&st->dt_min);
    const double t = LD::ld(&st->t);
    const unsigned flags = LD::ldu(&st->flags);
    const int replay = LD::ldi(&st->replay), consec = LD::ldi(&st->consec),
              max_rejects = LD::ldi(&st->max_rejects);
    const int cur = LD::ldi(&st->cur);
    const long long n_acc = LD::ldll(&st->n_accept), n_rej = LD::ldll(&st->n_reject);
    int status = ST_OK;
    bool accept = false;
    double dtn = dt;
    const bool folded = (flags & FLAG_FOLDED_TRIAL) != 0;
    double lam_out = lam;
    if (flags & FLAG_TIMEOUT) {
      status = ST_TIMEOUT;
    } else if (flags & FLAG_COLLAPSED) {
      status = ST_COLLAPSED;
    } else if (!folded && !isfinite(lam)) {
      status = ST_NONFINITE;
    } else if (folded) {
      // a trial stage folded the grid: reject with the largest shrink
      dtn = dt * shrink_min;
      lam_out = INFINITY;
      if (consec + 1 > max_rejects || dtn < dt_min) status = ST_DT_UNDERFLOW;
    } else if (replay) {
      accept = true;
    } else if (lam > lambda0) {
      double fac = safety * fifth_root(lambda0 / lam);
      if (fac < shrink_min) fac = shrink_min;
      dtn = dt * fac;
      if (consec + 1 > max_rejects || dtn < dt_min) status = ST_DT_UNDERFLOW;
    } else {
      accept = true;
      double fac = 1.0;
      if (lam < 0.5 * lambda0) {
        fac = lam > 0.0 ? safety * fifth_root(lambda0 / lam) : grow_max;
        if (fac > grow_max) fac = grow_max;
      }
      dtn = dt * fac;
    }
    st->lambda = lam_out;
    if (status != ST_OK) {
      // the attempt ends the run: counted as a rejection, state untouched
      st->status = status;
      st->n_reject = n_rej + 1;
      if (status == ST_DT_UNDERFLOW) st->consec = consec + 1;
      go_on = 0;
    } else {
      if (replay) st->replay = 0;
      if (accept) {
        // the step-size log: accepted step n_acc in slot n_acc mod the ring
        dtlog[n_acc % GLEMUR_DT_LOG] = dt;
        st->dt_last = dt;
        st->t = t + dt;
        st->cur = cur ^ 1;
        st->n_accept = n_acc + 1;
        st->consec = 0;
      } else {
        st->n_reject = n_rej + 1;
        st->consec = consec + 1;
      }
      st->dt = dtn;
      st->flags = 0;
      dt_next = dtn;
      go_on = 1;
    }
  }
  __syncthreads();
  if (go_on) set_coeffs_parallel(st, dt_next);
}

}  // namespace glemur
