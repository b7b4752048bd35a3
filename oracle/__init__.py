"""FP64 CPU oracle (test infrastructure only).

Python view of ``glemur_oracle.c``: a plain, slow restatement of the paper's
method that the CUDA library is checked against.  Only ``tests/``, the
package smoke check and the benchmark's CPU-baseline leg import this module;
the library itself never does, and this module imports nothing from it.

Fields are float64 arrays of shape (3, nz, ny, nx) (SoA, C order); ``grid``
is any object with ``nx, ny, nz`` and ``h`` (label spacings).
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

MIMETIC, DIRECT, NNN = 0, 1, 2
OK, ERR_BADARG, ERR_COLLAPSED, ERR_NONFINITE, ERR_DT_UNDERFLOW = 0, -1, -3, -4, -5

_dp = C.POINTER(C.c_double)


class _Grid(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("h", C.c_double * 3), ("periodic_z", C.c_int)]


class _Opts(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("dt_min", C.c_double),
                ("grow_max", C.c_double), ("shrink_min", C.c_double),
                ("max_rejects", C.c_int), ("safety", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("accepted", C.c_int), ("rejected", C.c_int), ("dt", C.c_double),
                ("t", C.c_double), ("lambda_", C.c_double)]


RHS_FN = C.CFUNCTYPE(C.c_int, C.c_void_p, _dp, _dp)


@dataclass
class ControlOpts:
    """Step-size control: the tolerance Lambda_0 and the library's defaults
    for the choices the paper leaves open."""
    lambda0: float = 1e-7
    dt_min: float = 1e-14
    grow_max: float = 5.0
    shrink_min: float = 0.1
    max_rejects: int = 64
    safety: float = 1.0

    def _c(self):
        return _Opts(self.lambda0, self.dt_min, self.grow_max, self.shrink_min,
                     self.max_rejects, self.safety)


_lib = None


def lib():
    global _lib
    if _lib is None:
        import os
        L = C.CDLL(os.environ.get("GLEMUR_ORACLE_LIB") or _build.build())
        L.ora_jacobian_at.argtypes = [C.POINTER(_Grid), _dp, C.c_int, C.c_int, C.c_int, _dp]
        L.ora_pullback.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp, _dp]
        L.ora_curl_mimetic.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp, _dp]
        L.ora_mimetic_loops_at.argtypes = [C.POINTER(_Grid), _dp, _dp, C.c_int, C.c_int,
                                           C.c_int, _dp, _dp, _dp]
        L.ora_curl_direct.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp]
        L.ora_curl_nnn.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp]
        L.ora_lorentz_velocity.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp]
        L.ora_lorentz_velocity.restype = None
        L.ora_velocity.argtypes = [C.POINTER(_Grid), C.c_int, _dp, _dp, _dp]
        L.ora_velocity_at.argtypes = [C.POINTER(_Grid), C.c_int, _dp, _dp, C.c_int,
                                      C.c_int, C.c_int, _dp]
        L.ora_cash_karp_tableau.argtypes = [_dp, _dp, _dp, _dp]
        L.ora_cash_karp_tableau.restype = None
        L.ora_ck_attempt.argtypes = [C.c_long, _dp, C.c_double, RHS_FN, C.c_void_p,
                                     _dp, _dp, _dp]
        L.ora_step_control.argtypes = [C.POINTER(_Opts), C.c_double, C.c_double, C.c_int,
                                       _dp, C.POINTER(C.c_int)]
        L.ora_relax.argtypes = [C.POINTER(_Grid), C.c_int, C.POINTER(_Opts), _dp, _dp,
                                C.c_int, _dp, _dp, C.POINTER(_Stats)]
        L.ora_step_fixed.argtypes = [C.POINTER(_Grid), C.c_int, _dp, _dp, C.c_double, _dp]
        L.ora_energy.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp]
        L.ora_forcefree.argtypes = [C.POINTER(_Grid), C.c_int, _dp, _dp, _dp, _dp]
        L.ora_deviation.argtypes = [C.POINTER(_Grid), _dp, _dp, _dp, _dp, _dp, _dp]
        L.ora_alpha_line.argtypes = [C.POINTER(_Grid), C.c_int, _dp, _dp, C.c_int, C.c_int,
                                     C.c_double, _dp, _dp]
        L.ora_convexity.argtypes = [C.POINTER(_Grid), _dp, C.c_void_p, C.POINTER(C.c_long)]
        L.orc_velocity.argtypes = [C.POINTER(_Grid), C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_relax_loss.argtypes = [C.POINTER(_Grid), C.c_void_p, C.c_void_p, _dp, C.c_int,
                                     C.c_int, C.c_void_p]
        _lib = L
    return _lib


def _g(grid) -> _Grid:
    return _Grid(grid.nx, grid.ny, grid.nz, (C.c_double * 3)(*grid.h),
                 int(getattr(grid, "periodic_z", False)))


def _p(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _f(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def _field(grid):
    return np.zeros((3, grid.nz, grid.ny, grid.nx))


def jacobian_at(grid, x, i, j, k) -> np.ndarray:
    x = _f(x)
    F = np.zeros(9)
    lib().ora_jacobian_at(C.byref(_g(grid)), _p(x), i, j, k, _p(F))
    return F.reshape(3, 3)


def pullback(grid, x, B0):
    x, B0 = _f(x), _f(B0)
    B = _field(grid)
    D = np.zeros((grid.nz, grid.ny, grid.nx))
    rc = lib().ora_pullback(C.byref(_g(grid)), _p(x), _p(B0), _p(B), _p(D))
    return B, D, rc


def curl_mimetic(grid, x, B):
    x, B = _f(x), _f(B)
    J = _field(grid)
    gap = np.zeros(1)
    rc = lib().ora_curl_mimetic(C.byref(_g(grid)), _p(x), _p(B), _p(J), _p(gap))
    return J, float(gap[0]), rc


def mimetic_loops_at(grid, x, B, i, j, k):
    x, B = _f(x), _f(B)
    c, M, J = np.zeros(3), np.zeros(9), np.zeros(3)
    rc = lib().ora_mimetic_loops_at(C.byref(_g(grid)), _p(x), _p(B), i, j, k,
                                    _p(c), _p(M), _p(J))
    return c, M.reshape(3, 3), J, rc


def curl_direct(grid, x, B0):
    x, B0 = _f(x), _f(B0)
    J = _field(grid)
    rc = lib().ora_curl_direct(C.byref(_g(grid)), _p(x), _p(B0), _p(J))
    return J, rc


def curl_nnn(grid, x, B):
    x, B = _f(x), _f(B)
    J = _field(grid)
    rc = lib().ora_curl_nnn(C.byref(_g(grid)), _p(x), _p(B), _p(J))
    return J, rc


def lorentz_velocity(grid, J, B):
    J, B = _f(J), _f(B)
    u = _field(grid)
    lib().ora_lorentz_velocity(C.byref(_g(grid)), _p(J), _p(B), _p(u))
    return u


def velocity(grid, x, B0, curl=MIMETIC):
    x, B0 = _f(x), _f(B0)
    u = _field(grid)
    rc = lib().ora_velocity(C.byref(_g(grid)), curl, _p(x), _p(B0), _p(u))
    return u, rc


def velocity_at(grid, x, B0, i, j, k, curl=MIMETIC):
    x, B0 = _f(x), _f(B0)
    u = np.zeros(3)
    rc = lib().ora_velocity_at(C.byref(_g(grid)), curl, _p(x), _p(B0), i, j, k, _p(u))
    return u, rc


def cash_karp_tableau():
    c, a, b5, b4 = np.zeros(6), np.zeros(36), np.zeros(6), np.zeros(6)
    lib().ora_cash_karp_tableau(_p(c), _p(a), _p(b5), _p(b4))
    return c, a.reshape(6, 6), b5, b4


def ck_attempt(y, dt, rhs):
    """One Cash-Karp attempt of the generic stepper on y' = rhs(y)."""
    y = _f(y).ravel().copy()
    n = y.size

    def cb(_ctx, yp, dp):
        yy = np.ctypeslib.as_array(yp, shape=(n,))
        d = np.ctypeslib.as_array(dp, shape=(n,))
        d[:] = rhs(yy.copy())
        return 0

    f = RHS_FN(cb)
    ynew, yerr, k = np.zeros(n), np.zeros(n), np.zeros(6 * n)
    rc = lib().ora_ck_attempt(n, _p(y), dt, f, None, _p(ynew), _p(yerr), _p(k))
    return ynew, yerr, k.reshape(6, n), rc


def step_control(opts: ControlOpts, lam, dt, consecutive_rejects=0):
    dtn = np.zeros(1)
    acc = C.c_int(0)
    o = opts._c()
    rc = lib().ora_step_control(C.byref(o), lam, dt, consecutive_rejects, _p(dtn),
                                C.byref(acc))
    return rc, float(dtn[0]), int(acc.value)


def relax(grid, x, B0, n_accept, dt, curl=MIMETIC, opts: ControlOpts | None = None,
          t=0.0):
    """n_accept error-controlled steps; returns (x, dt_next, dt_log, stats, rc)."""
    opts = opts or ControlOpts()
    x = _f(x).copy()
    B0 = _f(B0)
    d = np.array([dt], dtype=np.float64)
    log = np.zeros(max(n_accept, 1))
    st = _Stats(0, 0, 0.0, t, 0.0)
    o = opts._c()
    rc = lib().ora_relax(C.byref(_g(grid)), curl, C.byref(o), _p(x), _p(B0), n_accept,
                         _p(d), _p(log), C.byref(st))
    stats = dict(accepted=st.accepted, rejected=st.rejected, dt=st.dt, t=st.t,
                 lam=st.lambda_)
    return x, float(d[0]), log[:st.accepted].copy(), stats, rc


def step_fixed(grid, x, B0, dt, curl=MIMETIC):
    x = _f(x).copy()
    B0 = _f(B0)
    lam = np.zeros(1)
    rc = lib().ora_step_fixed(C.byref(_g(grid)), curl, _p(x), _p(B0), dt, _p(lam))
    return x, float(lam[0]), rc


def energy(grid, x, B0):
    x, B0 = _f(x), _f(B0)
    E = np.zeros(1)
    rc = lib().ora_energy(C.byref(_g(grid)), _p(x), _p(B0), _p(E))
    return float(E[0]), rc


def forcefree(grid, x, B0, curl=MIMETIC):
    x, B0 = _f(x), _f(B0)
    a, b = np.zeros(1), np.zeros(1)
    rc = lib().ora_forcefree(C.byref(_g(grid)), curl, _p(x), _p(B0), _p(a), _p(b))
    return float(a[0]), float(b[0]), rc


def deviation(grid, x, B0, x_ref, B_ref):
    """(sigma_x, sigma_B, rc): RMS over nodes of |x - x_ref| and |B - B_ref|."""
    x, B0, x_ref, B_ref = _f(x), _f(B0), _f(x_ref), _f(B_ref)
    a, b = np.zeros(1), np.zeros(1)
    rc = lib().ora_deviation(C.byref(_g(grid)), _p(x), _p(B0), _p(x_ref), _p(B_ref),
                             _p(a), _p(b))
    return float(a[0]), float(b[0]), rc


def alpha_line(grid, x, B0, i, j, a_r, curl=MIMETIC):
    """(alpha* along the node line (i, j, .) -- NaN at its two boundary
    nodes --, epsilon*, rc)."""
    x, B0 = _f(x), _f(B0)
    alpha = np.zeros(grid.nz)
    e = np.zeros(1)
    rc = lib().ora_alpha_line(C.byref(_g(grid)), curl, _p(x), _p(B0), i, j, a_r,
                              _p(alpha), _p(e))
    return alpha, float(e[0]), rc


def convexity(grid, x):
    """(kappa per node as int32 (nz, ny, nx), number of concave nodes)."""
    x = _f(x)
    kappa = np.zeros((grid.nz, grid.ny, grid.nx), dtype=np.int32)
    n = C.c_long(0)
    lib().ora_convexity(C.byref(_g(grid)), _p(x), kappa.ctypes.data, C.byref(n))
    return kappa, int(n.value)


# ---------------------------------------------------------------- complex step
# Complex-analytic evaluation of the same method (glemur_oracle_cstep.c):
# with an input perturbed by i*h, Im(output)/h is its exact derivative.

CSTEP_H = 1e-30
LOSS_ENERGY, LOSS_XI = 0, 1


def _c(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.complex128)


def cs_velocity(grid, y, B0):
    """u(y; B0) with complex positions and field (mimetic current)."""
    y, B0 = _c(y), _c(B0)
    u = np.zeros((3, grid.nz, grid.ny, grid.nx), dtype=np.complex128)
    rc = lib().orc_velocity(C.byref(_g(grid)), y.ctypes.data, B0.ctypes.data, u.ctypes.data)
    return u, rc


def cs_relax_loss(grid, x0, B0, dts, loss=LOSS_ENERGY):
    """Cash-Karp steps at the schedule `dts` from x0, then the loss
    (E_M or xi) of the final state; complex in, complex out."""
    x = _c(x0).copy()
    B0 = _c(B0)
    d = np.ascontiguousarray(dts, dtype=np.float64)
    val = np.zeros(1, dtype=np.complex128)
    rc = lib().orc_relax_loss(C.byref(_g(grid)), x.ctypes.data, B0.ctypes.data,
                              d.ctypes.data_as(_dp), len(d), loss, val.ctypes.data)
    return complex(val[0]), x, rc
